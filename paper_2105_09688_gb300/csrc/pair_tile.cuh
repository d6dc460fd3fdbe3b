// pair_tile.cuh -- device code of the O(N^2) pair sums, shared by the
// single-context kernels (k_pair.cu) and the batched kernels (batch.cu).
//
// Every integral against an empirical measure in the SSM (§2.3, eq.
// SSTM:scheme 1 and 2) is a sum over all N particles j (self term included,
// weight 1/N).  One tile computes, for THREADS * R target particles and the
// sources [j0, j1), the partial sums
//
//   PK_DRIFT1 : sum_j (y_j - y_i) 2^(-(y'_i - y'_j)^2)                      (d = 1)
//   PK_DRIFT3 : sum_j (y_j - y_i) 2^(-|y'_i - y'_j|^2)                      (d = 3)
//   PK_NEWTON3: sum_j (x_j - y_i) / (1 + |x_j - y_i|^2),  sum_j 1/(1 + |x_j - y_i|^2)
//   PK_NEWTON1: the same at d = 1
//
// (y' = scale * y turns the Gaussian kernels exp(-c r^2) of the drift into base-2
// exponentials; the FP64 forms use exp directly).  The results go to
// part[c * Np + t] for target slot t (the caller offsets part by chunk).
//
// A pairwise nonlinear kernel is not a contraction, so it runs on the FP32 (or
// FP64) CUDA-core pipes: each thread holds R targets in registers; sources are
// staged SUB at a time in shared memory from the FP64 state (converted and
// scaled while staging) and read back with broadcast loads.  FP32 forms use
// rcp.approx / ex2.approx and accumulate in FP32 within a SUB-source sub-tile;
// sub-tile sums are folded into a (hi, lo) pair by two-sum, so a chunk sum is
// accurate to ~2^-46 relative.  The packed form holds two targets per register
// pair and issues FFMA2/FADD2/FMUL2 (two FP32 lanes per instruction).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssm_device.cuh"

namespace ssm {

template <typename T> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4; };

template <int KIND> struct KindInfo;
template <> struct KindInfo<PK_DRIFT1> { static constexpr int D = 1, NC = 1; };
template <> struct KindInfo<PK_DRIFT3> { static constexpr int D = 3, NC = 3; };
template <> struct KindInfo<PK_NEWTON3> { static constexpr int D = 3, NC = 4; };
template <> struct KindInfo<PK_NEWTON1> { static constexpr int D = 1, NC = 2; };

// One pair interaction: accumulate into acc[NC].
template <int KIND, typename T>
__device__ __forceinline__ void pair(const typename V4<T>::t &s, T tx, T ty, T tz, T *acc);

template <> __device__ __forceinline__ void pair<PK_DRIFT1, float>(const float4 &s, float tx, float, float, float *acc) {
    const float dx = s.x - tx;
    const float e = ex2_approx(-dx * dx);
    acc[0] = fmaf(e, dx, acc[0]);
}
template <> __device__ __forceinline__ void pair<PK_DRIFT3, float>(const float4 &s, float tx, float ty, float tz, float *acc) {
    const float dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const float nq = fmaf(-dx, dx, fmaf(-dy, dy, -dz * dz));
    const float e = ex2_approx(nq);
    acc[0] = fmaf(e, dx, acc[0]);
    acc[1] = fmaf(e, dy, acc[1]);
    acc[2] = fmaf(e, dz, acc[2]);
}
template <> __device__ __forceinline__ void pair<PK_NEWTON3, float>(const float4 &s, float tx, float ty, float tz, float *acc) {
    const float dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const float q = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, 1.0f)));
    const float w = rcp_approx(q);
    acc[0] = fmaf(w, dx, acc[0]);
    acc[1] = fmaf(w, dy, acc[1]);
    acc[2] = fmaf(w, dz, acc[2]);
    acc[3] += w;
}
template <> __device__ __forceinline__ void pair<PK_NEWTON1, float>(const float4 &s, float tx, float, float, float *acc) {
    const float dx = s.x - tx;
    const float w = rcp_approx(fmaf(dx, dx, 1.0f));
    acc[0] = fmaf(w, dx, acc[0]);
    acc[1] += w;
}
template <> __device__ __forceinline__ void pair<PK_DRIFT1, double>(const double4 &s, double tx, double, double, double *acc) {
    const double dx = s.x - tx;
    acc[0] += dx * exp(-(dx * dx));
}
template <> __device__ __forceinline__ void pair<PK_DRIFT3, double>(const double4 &s, double tx, double ty, double tz, double *acc) {
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double e = exp(-(dx * dx + dy * dy + dz * dz) * 0.5);
    acc[0] += dx * e;
    acc[1] += dy * e;
    acc[2] += dz * e;
}
template <> __device__ __forceinline__ void pair<PK_NEWTON3, double>(const double4 &s, double tx, double ty, double tz, double *acc) {
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double w = 1.0 / (1.0 + dx * dx + dy * dy + dz * dz);
    acc[0] += dx * w;
    acc[1] += dy * w;
    acc[2] += dz * w;
    acc[3] += w;
}
template <> __device__ __forceinline__ void pair<PK_NEWTON1, double>(const double4 &s, double tx, double, double, double *acc) {
    const double dx = s.x - tx;
    const double w = 1.0 / (1.0 + dx * dx);
    acc[0] += dx * w;
    acc[1] += w;
}

template <typename T> __device__ __forceinline__ T cvt(double v, double scale);
template <> __device__ __forceinline__ float cvt<float>(double v, double scale) { return (float)(v * scale); }
template <> __device__ __forceinline__ double cvt<double>(double v, double scale) { return v * scale; }

// Scalar tile.  src, tgt: FP64 SoA state arrays [D][Np].  Targets t0 + r*THREADS +
// tid (r < R) below ntgt are particles act[t] (or t without a list).  Block-uniform:
// every thread of the block must call it with the same arguments.
template <int KIND, typename T, int THREADS, int R>
__device__ __forceinline__ void tile_scalar(const double *__restrict__ src, const double *__restrict__ tgt,
                                            const int *__restrict__ act, int64_t ntgt, int64_t Np, int64_t j0,
                                            int64_t j1, int64_t t0, double scale, double *__restrict__ part) {
    constexpr int D = KindInfo<KIND>::D, NC = KindInfo<KIND>::NC;
    using V = typename V4<T>::t;
    __shared__ V sm[SUB];
    const int tid = threadIdx.x;

    T tx[R], ty[R], tz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t t = t0 + r * THREADS + tid;
        int64_t i = 0;
        if (t < ntgt) i = act ? (int64_t)act[t] : t;
        tx[r] = cvt<T>(tgt[i], scale);
        ty[r] = D == 3 ? cvt<T>(tgt[Np + i], scale) : T(0);
        tz[r] = D == 3 ? cvt<T>(tgt[2 * Np + i], scale) : T(0);
    }
    T acc[R][NC];
    float hi[R][NC], lo[R][NC];   // compensated FP32 totals (FP32 forms only)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[r][c] = T(0); hi[r][c] = 0.f; lo[r][c] = 0.f; }

    for (int64_t base = j0; base < j1; base += SUB) {
        const int ns = (int)((j1 - base) < SUB ? (j1 - base) : SUB);
        __syncthreads();
        for (int s = tid; s < ns; s += THREADS) {
            const int64_t j = base + s;
            V v;
            v.x = cvt<T>(src[j], scale);
            v.y = D == 3 ? cvt<T>(src[Np + j], scale) : T(0);
            v.z = D == 3 ? cvt<T>(src[2 * Np + j], scale) : T(0);
            v.w = T(0);
            sm[s] = v;
        }
        __syncthreads();
        if (ns == SUB) {
#pragma unroll 4
            for (int s = 0; s < SUB; ++s) {
                const V v = sm[s];
#pragma unroll
                for (int r = 0; r < R; ++r) pair<KIND, T>(v, tx[r], ty[r], tz[r], acc[r]);
            }
        } else {
            for (int s = 0; s < ns; ++s) {
                const V v = sm[s];
#pragma unroll
                for (int r = 0; r < R; ++r) pair<KIND, T>(v, tx[r], ty[r], tz[r], acc[r]);
            }
        }
        if (sizeof(T) == 4) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < NC; ++c) { two_sum_acc(hi[r][c], lo[r][c], (float)acc[r][c]); acc[r][c] = T(0); }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t t = t0 + r * THREADS + tid;
        if (t < ntgt) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
                part[(int64_t)c * Np + t] = sizeof(T) == 4 ? (double)hi[r][c] + (double)lo[r][c] : (double)acc[r][c];
        }
    }
}

// ---- packed FP32 form (d = 3 kinds) -----------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int KIND>
__device__ __forceinline__ void pair2(float2 sx, float2 sy, float2 sz, float2 ntx, float2 nty, float2 ntz,
                                      float2 one, float2 *acc);
// The differences and the plain sums are issued as FFMA2 with a unit factor
// (fma(s, 1, -t) rounds exactly like s - t): FADD2 sustains only ~2/3 of the
// FFMA2 rate on this SM.  `one` comes from shared memory so the compiler cannot
// turn the fma back into an add.
template <> __device__ __forceinline__ void pair2<PK_NEWTON3>(float2 sx, float2 sy, float2 sz, float2 ntx,
                                                              float2 nty, float2 ntz, float2 one, float2 *acc) {
    const float2 dx = __ffma2_rn(sx, one, ntx), dy = __ffma2_rn(sy, one, nty), dz = __ffma2_rn(sz, one, ntz);
    float2 q = __ffma2_rn(dx, dx, one);
    q = __ffma2_rn(dy, dy, q);
    q = __ffma2_rn(dz, dz, q);
    const float2 w = f2(rcp_approx(q.x), rcp_approx(q.y));
    acc[0] = __ffma2_rn(w, dx, acc[0]);
    acc[1] = __ffma2_rn(w, dy, acc[1]);
    acc[2] = __ffma2_rn(w, dz, acc[2]);
    acc[3] = __ffma2_rn(w, one, acc[3]);
}
template <> __device__ __forceinline__ void pair2<PK_DRIFT3>(float2 sx, float2 sy, float2 sz, float2 ntx,
                                                             float2 nty, float2 ntz, float2 one, float2 *acc) {
    const float2 dx = __ffma2_rn(sx, one, ntx), dy = __ffma2_rn(sy, one, nty), dz = __ffma2_rn(sz, one, ntz);
    const float2 mdz = f2(-dz.x, -dz.y), mdy = f2(-dy.x, -dy.y), mdx = f2(-dx.x, -dx.y);
    const float2 nq = __ffma2_rn(mdx, dx, __ffma2_rn(mdy, dy, __fmul2_rn(mdz, dz)));
    const float2 e = f2(ex2_approx(nq.x), ex2_approx(nq.y));
    acc[0] = __ffma2_rn(e, dx, acc[0]);
    acc[1] = __ffma2_rn(e, dy, acc[1]);
    acc[2] = __ffma2_rn(e, dz, acc[2]);
}

// Packed tile: target 2k of a register pair in .x, 2k+1 in .y; a source coordinate
// is stored duplicated in shared memory so one packed instruction advances two
// pair interactions.  Same arithmetic as the scalar FP32 form, term for term.
template <int KIND, int THREADS, int R>
__device__ __forceinline__ void tile_packed(const double *__restrict__ src, const double *__restrict__ tgt,
                                            const int *__restrict__ act, int64_t ntgt, int64_t Np, int64_t j0,
                                            int64_t j1, int64_t t0, double scale, double *__restrict__ part) {
    static_assert(R % 2 == 0, "targets per thread come in pairs");
    constexpr int NC = KindInfo<KIND>::NC, R2 = R / 2;
    __shared__ float4 sxy[SUB];   // (x, x, y, y)
    __shared__ float2 szz[SUB];   // (z, z)
    __shared__ float2 s_one;
    const int tid = threadIdx.x;
    if (tid == 0) s_one = f2(1.0f, 1.0f);

    float2 ntx[R2], nty[R2], ntz[R2];
#pragma unroll
    for (int k = 0; k < R2; ++k) {
        float v[2][3];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t t = t0 + (2 * k + e) * THREADS + tid;
            int64_t i = 0;
            if (t < ntgt) i = act ? (int64_t)act[t] : t;
            v[e][0] = -(float)(tgt[i] * scale);
            v[e][1] = -(float)(tgt[Np + i] * scale);
            v[e][2] = -(float)(tgt[2 * Np + i] * scale);
        }
        ntx[k] = f2(v[0][0], v[1][0]);
        nty[k] = f2(v[0][1], v[1][1]);
        ntz[k] = f2(v[0][2], v[1][2]);
    }
    float2 acc[R2][NC], hi[R2][NC], lo[R2][NC];
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) { acc[k][c] = f2(0.f, 0.f); hi[k][c] = f2(0.f, 0.f); lo[k][c] = f2(0.f, 0.f); }

    for (int64_t base = j0; base < j1; base += SUB) {
        const int ns = (int)((j1 - base) < SUB ? (j1 - base) : SUB);
        __syncthreads();
        for (int s = tid; s < ns; s += THREADS) {
            const int64_t j = base + s;
            const float x = (float)(src[j] * scale), y = (float)(src[Np + j] * scale), z = (float)(src[2 * Np + j] * scale);
            sxy[s] = make_float4(x, x, y, y);
            szz[s] = f2(z, z);
        }
        __syncthreads();
        const float2 one = s_one;
        if (ns == SUB) {
#pragma unroll 4
            for (int s = 0; s < SUB; ++s) {
                const float4 a = sxy[s];
                const float2 b = szz[s];
#pragma unroll
                for (int k = 0; k < R2; ++k)
                    pair2<KIND>(f2(a.x, a.y), f2(a.z, a.w), b, ntx[k], nty[k], ntz[k], one, acc[k]);
            }
        } else {
            for (int s = 0; s < ns; ++s) {
                const float4 a = sxy[s];
                const float2 b = szz[s];
#pragma unroll
                for (int k = 0; k < R2; ++k)
                    pair2<KIND>(f2(a.x, a.y), f2(a.z, a.w), b, ntx[k], nty[k], ntz[k], one, acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < R2; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                two_sum_acc(hi[k][c].x, lo[k][c].x, acc[k][c].x);
                two_sum_acc(hi[k][c].y, lo[k][c].y, acc[k][c].y);
                acc[k][c] = f2(0.f, 0.f);
            }
    }
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t t = t0 + (2 * k + e) * THREADS + tid;
            if (t < ntgt) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    part[(int64_t)c * Np + t] =
                        e == 0 ? (double)hi[k][c].x + (double)lo[k][c].x : (double)hi[k][c].y + (double)lo[k][c].y;
            }
        }
}

}  // namespace ssm
