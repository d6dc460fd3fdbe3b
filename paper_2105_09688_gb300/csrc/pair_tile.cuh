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
// part[c * ps + t] for target slot t (the caller offsets part by chunk and gives
// the stride ps of the partial sums).
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
template <> struct V4<double> { using t = double4_32a; };

// Particle of target slot t (0 for slots past ntgt).  Debug builds check the list
// entry against the arrays' extent Np (SSM_CHECK_BOUNDS: recorded, slot 0 read instead).
__device__ __forceinline__ int64_t target_index(const int *__restrict__ act, int64_t t, int64_t ntgt, int64_t Np) {
    if (t >= ntgt) return 0;
    const int64_t i = act ? (int64_t)act[t] : t;
    return SSM_IN_BOUNDS(i >= 0 && i < Np) ? i : 0;
}

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
// PK_NEWTON1 with the reciprocal on the FMA pipe instead of the MUFU: a seed from
// the IEEE bit pattern (y0 = bits(K - bits(q)), K = 0x7ef311c2 found by a minimax
// search over q in [1, 2): max |q y0 - 1| = 0.0505) refined by three Newton steps
// y <- y + y (1 - q y) (error 0.0505^8 before rounding, ~1 ulp after).  The d = 1
// step-1 sums are MUFU-bound (1 reciprocal to 4 FP32 operations per pair) with the
// FMA pipe mostly idle, so one target in eight takes this form (timed at N = 2^18,
// 128 threads x 8 targets: 13.4 ms a pass against 14.5 ms with every reciprocal on
// the MUFU; one in four 14.1 ms, one in two 16.4 ms).
constexpr unsigned RCP_SEED = 0x7ef311c2u;
__device__ __forceinline__ float rcp_newton(float q) {
    float y = __uint_as_float(RCP_SEED - __float_as_uint(q));
#pragma unroll
    for (int k = 0; k < 3; ++k) y = fmaf(y, fmaf(-q, y, 1.0f), y);
    return y;
}
__device__ __forceinline__ void pair_newton1_fma(const float4 &s, float tx, float *acc) {
    const float dx = s.x - tx;
    const float w = rcp_newton(fmaf(dx, dx, 1.0f));
    acc[0] = fmaf(w, dx, acc[0]);
    acc[1] += w;
}
template <> __device__ __forceinline__ void pair<PK_DRIFT1, double>(const double4_32a &s, double tx, double, double, double *acc) {
    const double dx = s.x - tx;
    acc[0] += dx * exp(-(dx * dx));
}
template <> __device__ __forceinline__ void pair<PK_DRIFT3, double>(const double4_32a &s, double tx, double ty, double tz, double *acc) {
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double e = exp(-(dx * dx + dy * dy + dz * dz) * 0.5);
    acc[0] += dx * e;
    acc[1] += dy * e;
    acc[2] += dz * e;
}
template <> __device__ __forceinline__ void pair<PK_NEWTON3, double>(const double4_32a &s, double tx, double ty, double tz, double *acc) {
    const double dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    const double w = 1.0 / (1.0 + dx * dx + dy * dy + dz * dz);
    acc[0] += dx * w;
    acc[1] += dy * w;
    acc[2] += dz * w;
    acc[3] += w;
}
template <> __device__ __forceinline__ void pair<PK_NEWTON1, double>(const double4_32a &s, double tx, double, double, double *acc) {
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
                                            int64_t j1, int64_t t0, double scale, double *__restrict__ part,
                                            int64_t ps) {
    constexpr int D = KindInfo<KIND>::D, NC = KindInfo<KIND>::NC;
    using V = typename V4<T>::t;
    __shared__ V sm[SUB];
    const int tid = threadIdx.x;

    T tx[R], ty[R], tz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t t = t0 + r * THREADS + tid;
        int64_t i = 0;
        if (t < ntgt) i = target_index(act, t, ntgt, Np);
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
                for (int r = 0; r < R; ++r) {
                    if constexpr (KIND == PK_NEWTON1 && sizeof(T) == 4 && R >= 8) {
                        if (r % 8 == 7) {
                            pair_newton1_fma(v, tx[r], acc[r]);
                            continue;
                        }
                    }
                    pair<KIND, T>(v, tx[r], ty[r], tz[r], acc[r]);
                }
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
                part[(int64_t)c * ps + t] = sizeof(T) == 4 ? (double)hi[r][c] + (double)lo[r][c] : (double)acc[r][c];
        }
    }
}

// ---- packed FP32 forms (d = 3 kinds) ----------------------------------------
// Target 2k of a register pair in .x, 2k+1 in .y; a source value is stored
// duplicated in shared memory so one packed instruction advances two pair
// interactions.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Difference form: the scalar FP32 arithmetic, term for term.
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

// Centred expansion.  With s = scale (x_j - c) and t = scale (y_i - c) rounded to
// FP32, c a point near the block's targets (their centroid),
//   1 + |s - t|^2  = (1 + |s|^2) + |t|^2 - 2 s.t                  (step 1, scale 1)
//   2^(-|s - t|^2) = 2^(-|t|^2) * 2^(-|s|^2 + 2 s.t)                  (drift)
// and sum_j w_ij (s_j - t_i) = sum_j w_ij s_j - t_i sum_j w_ij.  So a pair costs the
// dot product and four accumulations -- 8 (step 1) and 7 (drift) packed
// instructions instead of 10 and 9 -- and the per-target factors (|t|^2, 2^(-|t|^2)
// and the linear t_i term) are applied once per target in FP64.  The source record
// is (s, k_j) with k_j = 1 + |s_j|^2 (step 1) or -|s_j|^2 (drift); the target
// registers hold u = -2t (step 1) or 2t (drift) and, for step 1, kb = |t|^2.
template <int KIND>
__device__ __forceinline__ void pair2x(float2 sx, float2 sy, float2 sz, float2 k, float2 ux, float2 uy, float2 uz,
                                       float2 kb, float2 one, float2 *acc);
template <> __device__ __forceinline__ void pair2x<PK_NEWTON3>(float2 sx, float2 sy, float2 sz, float2 k, float2 ux,
                                                               float2 uy, float2 uz, float2 kb, float2 one,
                                                               float2 *acc) {
    float2 q = __ffma2_rn(k, one, kb);
    q = __ffma2_rn(sz, uz, q);
    q = __ffma2_rn(sy, uy, q);
    q = __ffma2_rn(sx, ux, q);
    const float2 w = f2(rcp_approx(q.x), rcp_approx(q.y));
    acc[0] = __ffma2_rn(w, sx, acc[0]);
    acc[1] = __ffma2_rn(w, sy, acc[1]);
    acc[2] = __ffma2_rn(w, sz, acc[2]);
    acc[3] = __ffma2_rn(w, one, acc[3]);
}
template <> __device__ __forceinline__ void pair2x<PK_DRIFT3>(float2 sx, float2 sy, float2 sz, float2 k, float2 ux,
                                                              float2 uy, float2 uz, float2, float2 one, float2 *acc) {
    float2 g = __ffma2_rn(sz, uz, k);
    g = __ffma2_rn(sy, uy, g);
    g = __ffma2_rn(sx, ux, g);
    const float2 e = f2(ex2_approx(g.x), ex2_approx(g.y));
    acc[0] = __ffma2_rn(e, sx, acc[0]);
    acc[1] = __ffma2_rn(e, sy, acc[1]);
    acc[2] = __ffma2_rn(e, sz, acc[2]);
    acc[3] = __ffma2_rn(e, one, acc[3]);
}

// Cancellation in the expansion grows with |s|^2 + |t|^2 (the rounding of one
// pair term is ~2^-24 (1 + 2|s|^2 + 2|t|^2) / q relative), so a block takes the
// expansion only when every one of its targets has |t|^2 <= EXP_R2 (scaled units
// about the centre); a source far from all targets makes q or the exponent large
// itself and keeps ~2^-24 relative accuracy.  The bound also keeps the drift's
// 2^(-|s|^2 + 2 s.t) <= 2^|t|^2 far from FP32 overflow.
constexpr float EXP_R2 = 64.f;

// Accumulators per target (difference / expanded form) and sources per shared-memory
// sub-tile of the packed kinds: the step-1 sums stage 512 sources at a time (half the
// barriers and two-sum folds of 256: 19.90 against 20.15 ms a pass at N = 2^18), the
// drift 256 (17.91 against 18.02 ms).
template <int KIND> struct PackedInfo;
template <> struct PackedInfo<PK_NEWTON3> { static constexpr int NC = 4, NX = 4, SUBP = 512; };
template <> struct PackedInfo<PK_DRIFT3> { static constexpr int NC = 3, NX = 4, SUBP = 256; };



// The two-sum compensation accumulators (hi, lo) of a thread's R2 x NC float2 sums,
// folded once per sub-tile of sources: in registers, or in shared memory (SMEM), where they
// leave the registers to the inner loop's accumulators and targets (more resident
// blocks).  Shared layout slot-major, hl[(2 slot + {0: hi, 1: lo}) THREADS + tid],
// slot = (k NC + c) 2 + lane: a warp's accesses fall in distinct banks.
template <int R2, int NC, int THREADS, bool SMEM> struct Comp;
template <int R2, int NC, int THREADS> struct Comp<R2, NC, THREADS, false> {
    float2 hi[R2][NC], lo[R2][NC];
    __device__ __forceinline__ Comp(float *, int) {
#pragma unroll
        for (int k = 0; k < R2; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) { hi[k][c] = f2(0.f, 0.f); lo[k][c] = f2(0.f, 0.f); }
    }
    __device__ __forceinline__ void fold(float2 (&acc)[R2][NC]) {
#pragma unroll
        for (int k = 0; k < R2; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                two_sum_acc(hi[k][c].x, lo[k][c].x, acc[k][c].x);
                two_sum_acc(hi[k][c].y, lo[k][c].y, acc[k][c].y);
                acc[k][c] = f2(0.f, 0.f);
            }
    }
    __device__ __forceinline__ double value(int k, int c, int e) const {
        return e == 0 ? (double)hi[k][c].x + (double)lo[k][c].x : (double)hi[k][c].y + (double)lo[k][c].y;
    }
};
template <int R2, int NC, int THREADS> struct Comp<R2, NC, THREADS, true> {
    float *my;   // this thread's column: constant offsets from one base
    __device__ __forceinline__ Comp(float *p, int t) : my(p + t) {
#pragma unroll
        for (int s = 0; s < 4 * R2 * NC; ++s) my[s * THREADS] = 0.f;
    }
    __device__ __forceinline__ void acc1(int slot, float a) {
        float h = my[(2 * slot) * THREADS], l = my[(2 * slot + 1) * THREADS];
        two_sum_acc(h, l, a);
        my[(2 * slot) * THREADS] = h;
        my[(2 * slot + 1) * THREADS] = l;
    }
    __device__ __forceinline__ void fold(float2 (&acc)[R2][NC]) {
#pragma unroll
        for (int k = 0; k < R2; ++k)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                acc1((k * NC + c) * 2 + 0, acc[k][c].x);
                acc1((k * NC + c) * 2 + 1, acc[k][c].y);
                acc[k][c] = f2(0.f, 0.f);
            }
    }
    __device__ __forceinline__ double value(int k, int c, int e) const {
        const int slot = (k * NC + c) * 2 + e;
        return (double)my[(2 * slot) * THREADS] + (double)my[(2 * slot + 1) * THREADS];
    }
};
// Compensation in shared memory for the shapes of 4 targets a thread, where it was
// measured faster (128 x 4 at N = 2^18: step-1 pass 20.65 ms against 21.16 ms with
// it in registers); with 8 targets a thread it was slower (21.9 against 21.0 ms),
// so those keep it in registers.  At most 32 KB beside the source sub-tile.
__host__ __device__ constexpr bool comp_in_smem(int threads, int r) {
    return r <= 4 && threads * (r / 2) * 4 * 4 * 4 <= 32768;
}

// Difference form of a packed tile (buf: 2 SUBP float4 of shared memory).
template <int KIND, int THREADS, int R>
__device__ __forceinline__ void tile_packed_diff(float4 *buf, float *hl, const float2 *s_one, const double *__restrict__ src,
                                                 const double *__restrict__ tgt, const int *__restrict__ act,
                                                 int64_t ntgt, int64_t Np, int64_t j0, int64_t j1, int64_t t0,
                                                 double scale, double *__restrict__ part, int64_t ps) {
    constexpr int NC = PackedInfo<KIND>::NC, R2 = R / 2, SUBP = PackedInfo<KIND>::SUBP;
    float4 *sxy = buf;                              // (x, x, y, y)
    float2 *szz = reinterpret_cast<float2 *>(buf + SUBP);   // (z, z)
    const int tid = threadIdx.x;

    float2 ntx[R2], nty[R2], ntz[R2];
#pragma unroll
    for (int k = 0; k < R2; ++k) {
        float v[2][3];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t i = target_index(act, t0 + (2 * k + e) * THREADS + tid, ntgt, Np);
            v[e][0] = -(float)(tgt[i] * scale);
            v[e][1] = -(float)(tgt[Np + i] * scale);
            v[e][2] = -(float)(tgt[2 * Np + i] * scale);
        }
        ntx[k] = f2(v[0][0], v[1][0]);
        nty[k] = f2(v[0][1], v[1][1]);
        ntz[k] = f2(v[0][2], v[1][2]);
    }
    float2 acc[R2][NC];
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[k][c] = f2(0.f, 0.f);
    Comp<R2, NC, THREADS, comp_in_smem(THREADS, R)> comp(hl, tid);

    for (int64_t base = j0; base < j1; base += SUBP) {
        const int ns = (int)((j1 - base) < SUBP ? (j1 - base) : SUBP);
        __syncthreads();
        for (int s = tid; s < ns; s += THREADS) {
            const int64_t j = base + s;
            const float x = (float)(src[j] * scale), y = (float)(src[Np + j] * scale), z = (float)(src[2 * Np + j] * scale);
            sxy[s] = make_float4(x, x, y, y);
            szz[s] = f2(z, z);
        }
        __syncthreads();
        const float2 one = *s_one;
        if (ns == SUBP) {
#pragma unroll 4
            for (int s = 0; s < SUBP; ++s) {
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
        comp.fold(acc);
    }
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t t = t0 + (2 * k + e) * THREADS + tid;
            if (t < ntgt) {
#pragma unroll
                for (int c = 0; c < NC; ++c) part[(int64_t)c * ps + t] = comp.value(k, c, e);
            }
        }
}

// Expanded form of a packed tile about the point cc[3] (unscaled coordinates).
// The partial sums it writes mean what the difference form's mean:
//   step 1: sum_j w (s_j - fl(y_i)) and sum_j w, with s_j = fl(x_j - c) + c, so the
//           consumer's correction of the FP32 target, -(y - fl(y)) sum w, still
//           applies (the linear t_i term is taken in FP64 here);
//   drift : sum_j e_ij (s_j - t_i) in scaled units, t_i = scale (y_i - c) exact.
template <int KIND, int THREADS, int R, typename CC>
__device__ __forceinline__ void tile_packed_exp(float4 *buf, float *hl, const float2 *s_one, const double *__restrict__ src,
                                                const double *__restrict__ tgt, const int *__restrict__ act,
                                                int64_t ntgt, int64_t Np, int64_t j0, int64_t j1, int64_t t0,
                                                double scale, const CC &cc, double *__restrict__ part,
                                                int64_t ps) {
    constexpr bool NEWTON = KIND == PK_NEWTON3;
    constexpr int NX = PackedInfo<KIND>::NX, R2 = R / 2, SUBP = PackedInfo<KIND>::SUBP;
    const int tid = threadIdx.x;
    const float usign = NEWTON ? -2.f : 2.f;

    float2 ux[R2], uy[R2], uz[R2], kb[R2];
#pragma unroll
    for (int k = 0; k < R2; ++k) {
        float v[2][4];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t i = target_index(act, t0 + (2 * k + e) * THREADS + tid, ntgt, Np);
            const float a = (float)((tgt[i] - cc[0]) * scale), b = (float)((tgt[Np + i] - cc[1]) * scale),
                        d = (float)((tgt[2 * Np + i] - cc[2]) * scale);
            v[e][0] = usign * a;
            v[e][1] = usign * b;
            v[e][2] = usign * d;
            v[e][3] = (float)((double)a * a + (double)b * b + (double)d * d);
        }
        ux[k] = f2(v[0][0], v[1][0]);
        uy[k] = f2(v[0][1], v[1][1]);
        uz[k] = f2(v[0][2], v[1][2]);
        kb[k] = f2(v[0][3], v[1][3]);
    }
    float2 acc[R2][NX];
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int c = 0; c < NX; ++c) acc[k][c] = f2(0.f, 0.f);
    Comp<R2, NX, THREADS, comp_in_smem(THREADS, R)> comp(hl, tid);

    for (int64_t base = j0; base < j1; base += SUBP) {
        const int ns = (int)((j1 - base) < SUBP ? (j1 - base) : SUBP);
        __syncthreads();
        for (int s = tid; s < ns; s += THREADS) {
            const int64_t j = base + s;
            const float x = (float)((src[j] - cc[0]) * scale), y = (float)((src[Np + j] - cc[1]) * scale),
                        z = (float)((src[2 * Np + j] - cc[2]) * scale);
            const double n2 = (double)x * x + (double)y * y + (double)z * z;
            const float kj = NEWTON ? (float)(1.0 + n2) : (float)(-n2);
            buf[2 * s] = make_float4(x, x, y, y);
            buf[2 * s + 1] = make_float4(z, z, kj, kj);
        }
        __syncthreads();
        const float2 one = *s_one;
        if (ns == SUBP) {
// unroll timed at N = 2^18: 128 x 4 step-1 pass 20.35 ms unrolled 16 (20.53 ms at 8);
// 128 x 8 drift pass 17.50 ms unrolled 12 (17.67 ms at 8, 17.78 ms at 16)
#pragma unroll (NEWTON && R == 4 ? 16 : (!NEWTON && R == 8) ? 12 : 8)
            for (int s = 0; s < SUBP; ++s) {
                const float4 a = buf[2 * s], b = buf[2 * s + 1];
#pragma unroll
                for (int k = 0; k < R2; ++k)
                    pair2x<KIND>(f2(a.x, a.y), f2(a.z, a.w), f2(b.x, b.y), f2(b.z, b.w), ux[k], uy[k], uz[k], kb[k],
                                 one, acc[k]);
            }
        } else {
            for (int s = 0; s < ns; ++s) {
                const float4 a = buf[2 * s], b = buf[2 * s + 1];
#pragma unroll
                for (int k = 0; k < R2; ++k)
                    pair2x<KIND>(f2(a.x, a.y), f2(a.z, a.w), f2(b.x, b.y), f2(b.z, b.w), ux[k], uy[k], uz[k], kb[k],
                                 one, acc[k]);
            }
        }
        comp.fold(acc);
    }
#pragma unroll
    for (int k = 0; k < R2; ++k)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t t = t0 + (2 * k + e) * THREADS + tid;
            if (t < ntgt) {
                const int64_t i = target_index(act, t, ntgt, Np);
                double S[NX];
#pragma unroll
                for (int c = 0; c < NX; ++c) S[c] = comp.value(k, c, e);
                if (NEWTON) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const double yc = tgt[c * Np + i];
                        part[(int64_t)c * ps + t] = S[c] - ((double)(float)yc - cc[c]) * S[3];
                    }
                    part[(int64_t)3 * ps + t] = S[3];
                } else {
                    const float2 tu[3] = {ux[k], uy[k], uz[k]};
                    double b2 = 0.0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const double tc = 0.5 * (double)(e == 0 ? tu[c].x : tu[c].y);   // the FP32 t_i
                        b2 += tc * tc;
                    }
                    const double f = exp2(-b2);
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        part[(int64_t)c * ps + t] = f * (S[c] - (tgt[c * Np + i] - cc[c]) * scale * S[3]);
                }
            }
        }
}

// Resident blocks per SM that the expanded kernels are compiled for (the register
// budget ptxas schedules the loop under; chosen by timing the compiled shapes).
__host__ __device__ constexpr int packed_min_blocks(int threads, int r) {
    return threads == 128 ? (r == 8 ? 3 : 5) : (r == 8 ? 1 : 2);
}

// Packed tile.  EXPAND: the block centres the expansion on the centroid of its
// own targets and takes it when all of them are within EXP_R2 of that point,
// else it runs the difference form; the choice is block-uniform and depends only
// on the data (and the launch shape).
template <int KIND, int THREADS, int R, bool EXPAND>
__device__ __forceinline__ void tile_packed(const double *__restrict__ src, const double *__restrict__ tgt,
                                            const int *__restrict__ act, int64_t ntgt, int64_t Np, int64_t j0,
                                            int64_t j1, int64_t t0, double scale, double *__restrict__ part,
                                            int64_t ps) {
    static_assert(R % 2 == 0, "targets per thread come in pairs");
    static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
    __shared__ float4 buf[2 * PackedInfo<KIND>::SUBP];
    __shared__ float s_hl[comp_in_smem(THREADS, R) ? THREADS * (R / 2) * 4 * 4 : 1];
    __shared__ float2 s_one;
    __shared__ double s_red[THREADS / 32][4];
    const int tid = threadIdx.x;
    if (tid == 0) s_one = f2(1.0f, 1.0f);
    if (EXPAND) {
        // centroid of the valid targets (fixed-order FP64 reduction)
        double m[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t t = t0 + r * THREADS + tid;
            if (t < ntgt) {
                const int64_t i = target_index(act, t, ntgt, Np);
                m[0] += tgt[i];
                m[1] += tgt[Np + i];
                m[2] += tgt[2 * Np + i];
                m[3] += 1.0;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
        if ((tid & 31) == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) s_red[tid >> 5][k] = m[k];
        __syncthreads();
        double cc[3] = {0.0, 0.0, 0.0}, cnt = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) {
            cc[0] += s_red[w][0];
            cc[1] += s_red[w][1];
            cc[2] += s_red[w][2];
            cnt += s_red[w][3];
        }
        cc[0] /= cnt; cc[1] /= cnt; cc[2] /= cnt;   // cnt >= 1: the caller skips empty tiles
        int ok = 1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t t = t0 + r * THREADS + tid;
            if (t < ntgt) {
                const int64_t i = target_index(act, t, ntgt, Np);
                const double a = (tgt[i] - cc[0]) * scale, b = (tgt[Np + i] - cc[1]) * scale,
                             d = (tgt[2 * Np + i] - cc[2]) * scale;
                ok &= (a * a + b * b + d * d <= (double)EXP_R2) ? 1 : 0;   // false for NaN
            }
        }
        // The step-1 kind reads the centre from shared memory in its loop and the
        // drift kind from registers: the register allocations that time fastest.
        if constexpr (KIND == PK_NEWTON3) {
            __shared__ double s_cc[3];
            if (tid < 3) s_cc[tid] = cc[tid];
            if (__syncthreads_and(ok)) {
                tile_packed_exp<KIND, THREADS, R>(buf, s_hl, &s_one, src, tgt, act, ntgt, Np, j0, j1, t0, scale, s_cc,
                                                  part, ps);
                return;
            }
        } else if (__syncthreads_and(ok)) {
            tile_packed_exp<KIND, THREADS, R>(buf, s_hl, &s_one, src, tgt, act, ntgt, Np, j0, j1, t0, scale, cc, part,
                                              ps);
            return;
        }
    }
    tile_packed_diff<KIND, THREADS, R>(buf, s_hl, &s_one, src, tgt, act, ntgt, Np, j0, j1, t0, scale, part, ps);
}

}  // namespace ssm
