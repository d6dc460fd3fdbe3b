// k_pair.cu -- the O(N^2) pair sums of the split-step method.
//
// Every integral against an empirical measure in the SSM (§2.3, eq.
// SSTM:scheme 1 and 2) is a sum over all N particles j (self term included,
// weight 1/N).  One kernel computes, for a tile of target particles and one
// chunk of source particles, the partial sums
//
//   PK_DRIFT1 : sum_j (y_j - y_i) exp(-(y_i - y_j)^2)                      (d = 1)
//   PK_DRIFT3 : sum_j (y_j - y_i) exp(-|y_i - y_j|^2 / 2)                  (d = 3)
//   PK_NEWTON3: sum_j (x_j - y_i) / (1 + |x_j - y_i|^2),  sum_j 1/(1 + |x_j - y_i|^2)
//
// (the first two are b of step 2 at mu^Y; the third is the pair part of v in
// step 1 at mu^X and the scalar that its diagonal Jacobian approximation uses).
// Partial sums go to part[(chunk * NC + comp) * Np + t]; the O(N) kernel that
// consumes them adds the chunks in a fixed order in double.
//
// Design (GB300, sm_103a): a pairwise nonlinear kernel is not a contraction, so
// it runs on the FP32 (or FP64) CUDA-core pipes: each thread holds R targets in
// registers, sources are staged 256 at a time in shared memory from the FP64
// state (converted and scaled while staging) and read back as one broadcast
// 16-byte load per source.  The FP32 forms use rcp.approx / ex2.approx and
// accumulate in FP32 within a 256-source sub-tile; sub-tile sums are folded into
// a (hi, lo) pair by two-sum, so the chunk sum is accurate to ~2^-46 relative.
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

// One pair interaction: accumulate into acc[NC].
template <int KIND, typename T>
__device__ __forceinline__ void pair(const typename V4<T>::t &s, T tx, T ty, T tz, T *acc);

// FP32 forms (coordinates pre-scaled for the Gaussian kinds).
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
// FP64 forms (unscaled coordinates, IEEE division and exp).
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

template <typename T> __device__ __forceinline__ T cvt(double v, double scale);
template <> __device__ __forceinline__ float cvt<float>(double v, double scale) { return (float)(v * scale); }
template <> __device__ __forceinline__ double cvt<double>(double v, double) { return v; }

// src, tgt: FP64 SoA state arrays [D][Np].  act/cnt: optional compacted target
// list (targets t < *cnt are particles act[t]); without it targets are 0..N-1.
template <int KIND, typename T, int THREADS, int R>
__global__ void __launch_bounds__(THREADS)
k_pair(const double *__restrict__ src, const double *__restrict__ tgt, const int *__restrict__ act,
       const int *__restrict__ cnt, int64_t N, int64_t Np, int64_t chunk_len, double scale,
       double *__restrict__ part) {
    constexpr int D = KindInfo<KIND>::D, NC = KindInfo<KIND>::NC;
    using V = typename V4<T>::t;
    __shared__ V sm[SUB];

    const int64_t ntgt = act ? (int64_t)(*cnt) : N;
    const int64_t t0 = (int64_t)blockIdx.x * (THREADS * R);
    if (t0 >= ntgt) return;   // block-uniform
    const int tid = threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t j0 = (int64_t)chunk * chunk_len;
    const int64_t j1 = (j0 + chunk_len < N) ? j0 + chunk_len : N;

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
            for (int c = 0; c < NC; ++c) {
                const double v = sizeof(T) == 4 ? (double)hi[r][c] + (double)lo[r][c] : (double)acc[r][c];
                part[((int64_t)chunk * NC + c) * Np + t] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packed-FP32 form (sm_100+ FFMA2/FADD2/FMUL2: two FP32 lanes per instruction).
// Targets are held in pairs: target 2k in .x and 2k+1 in .y of a float2, and a
// source coordinate is broadcast to both halves (stored duplicated in shared
// memory), so one packed instruction advances two pair interactions.  Same
// arithmetic as the scalar FP32 form, term for term.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int KIND>
__device__ __forceinline__ void pair2(float2 sx, float2 sy, float2 sz, float2 ntx, float2 nty, float2 ntz,
                                      float2 *acc);
template <> __device__ __forceinline__ void pair2<PK_NEWTON3>(float2 sx, float2 sy, float2 sz, float2 ntx,
                                                              float2 nty, float2 ntz, float2 *acc) {
    const float2 dx = __fadd2_rn(sx, ntx), dy = __fadd2_rn(sy, nty), dz = __fadd2_rn(sz, ntz);
    float2 q = __ffma2_rn(dx, dx, f2(1.0f, 1.0f));
    q = __ffma2_rn(dy, dy, q);
    q = __ffma2_rn(dz, dz, q);
    const float2 w = f2(rcp_approx(q.x), rcp_approx(q.y));
    acc[0] = __ffma2_rn(w, dx, acc[0]);
    acc[1] = __ffma2_rn(w, dy, acc[1]);
    acc[2] = __ffma2_rn(w, dz, acc[2]);
    acc[3] = __fadd2_rn(acc[3], w);
}
template <> __device__ __forceinline__ void pair2<PK_DRIFT3>(float2 sx, float2 sy, float2 sz, float2 ntx,
                                                             float2 nty, float2 ntz, float2 *acc) {
    const float2 dx = __fadd2_rn(sx, ntx), dy = __fadd2_rn(sy, nty), dz = __fadd2_rn(sz, ntz);
    const float2 mdz = f2(-dz.x, -dz.y), mdy = f2(-dy.x, -dy.y), mdx = f2(-dx.x, -dx.y);
    const float2 nq = __ffma2_rn(mdx, dx, __ffma2_rn(mdy, dy, __fmul2_rn(mdz, dz)));
    const float2 e = f2(ex2_approx(nq.x), ex2_approx(nq.y));
    acc[0] = __ffma2_rn(e, dx, acc[0]);
    acc[1] = __ffma2_rn(e, dy, acc[1]);
    acc[2] = __ffma2_rn(e, dz, acc[2]);
}

template <int KIND, int THREADS, int R>
__global__ void __launch_bounds__(THREADS)
k_pair2(const double *__restrict__ src, const double *__restrict__ tgt, const int *__restrict__ act,
        const int *__restrict__ cnt, int64_t N, int64_t Np, int64_t chunk_len, double scale,
        double *__restrict__ part) {
    static_assert(R % 2 == 0, "targets per thread come in pairs");
    constexpr int NC = KindInfo<KIND>::NC, R2 = R / 2;
    __shared__ float4 sxy[SUB];   // (x, x, y, y)
    __shared__ float2 szz[SUB];   // (z, z)

    const int64_t ntgt = act ? (int64_t)(*cnt) : N;
    const int64_t t0 = (int64_t)blockIdx.x * (THREADS * R);
    if (t0 >= ntgt) return;
    const int tid = threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t j0 = (int64_t)chunk * chunk_len;
    const int64_t j1 = (j0 + chunk_len < N) ? j0 + chunk_len : N;

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
        if (ns == SUB) {
#pragma unroll 4
            for (int s = 0; s < SUB; ++s) {
                const float4 a = sxy[s];
                const float2 b = szz[s];
#pragma unroll
                for (int k = 0; k < R2; ++k) pair2<KIND>(f2(a.x, a.y), f2(a.z, a.w), b, ntx[k], nty[k], ntz[k], acc[k]);
            }
        } else {
            for (int s = 0; s < ns; ++s) {
                const float4 a = sxy[s];
                const float2 b = szz[s];
#pragma unroll
                for (int k = 0; k < R2; ++k) pair2<KIND>(f2(a.x, a.y), f2(a.z, a.w), b, ntx[k], nty[k], ntz[k], acc[k]);
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
                for (int c = 0; c < NC; ++c) {
                    const double v = e == 0 ? (double)hi[k][c].x + (double)lo[k][c].x : (double)hi[k][c].y + (double)lo[k][c].y;
                    part[((int64_t)chunk * NC + c) * Np + t] = v;
                }
            }
        }
}

// ---------------------------------------------------------------------------
// Host launchers.  Launch shapes (threads, targets per thread, packed or
// scalar FP32) are compiled-in candidates; the chunk count comes from the plan.
// ---------------------------------------------------------------------------
template <int KIND, typename T, int THREADS, int R>
static cudaError_t launch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                          int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
    const int64_t tiles = (N + THREADS * R - 1) / (THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)p.chunks);
    k_pair<KIND, T, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part);
    return cudaGetLastError();
}
template <int KIND, int THREADS, int R>
static cudaError_t launch2(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                           int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
    const int64_t tiles = (N + THREADS * R - 1) / (THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)p.chunks);
    k_pair2<KIND, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part);
    return cudaGetLastError();
}

// The (threads, targets per thread) shapes compiled for the scalar and the
// packed kernels.
#define SSM_PAIR_SHAPES(X) X(128, 2) X(128, 4) X(256, 2) X(256, 4) X(128, 8)
#define SSM_PAIR2_SHAPES(X) X(128, 4) X(128, 8) X(256, 4) X(256, 8)

template <int KIND, typename T>
static cudaError_t dispatch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                            int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
#define SSM_CASE(TH, RR) \
    if (p.threads == TH && p.rpt == RR) return launch<KIND, T, TH, RR>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    return cudaErrorInvalidValue;
}
template <int KIND>
static cudaError_t dispatch2(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                             int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
#define SSM_CASE(TH, RR) \
    if (p.threads == TH && p.rpt == RR) return launch2<KIND, TH, RR>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t pair_sums(int kind, bool fp32, const Plan &p, const double *src, const double *tgt, const int *act,
                      const int *cnt, int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
    if (fp32 && p.vec2) {
        if (kind == PK_NEWTON3) return dispatch2<PK_NEWTON3>(p, src, tgt, act, cnt, N, Np, scale, part, st);
        if (kind == PK_DRIFT3) return dispatch2<PK_DRIFT3>(p, src, tgt, act, cnt, N, Np, scale, part, st);
        return cudaErrorInvalidValue;
    }
    switch (kind) {
    case PK_DRIFT1:
        return fp32 ? dispatch<PK_DRIFT1, float>(p, src, tgt, act, cnt, N, Np, scale, part, st)
                    : dispatch<PK_DRIFT1, double>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    case PK_DRIFT3:
        return fp32 ? dispatch<PK_DRIFT3, float>(p, src, tgt, act, cnt, N, Np, scale, part, st)
                    : dispatch<PK_DRIFT3, double>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    case PK_NEWTON3:
        return fp32 ? dispatch<PK_NEWTON3, float>(p, src, tgt, act, cnt, N, Np, scale, part, st)
                    : dispatch<PK_NEWTON3, double>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    }
    return cudaErrorInvalidValue;
}

template <int KIND, typename T>
static int occ_dispatch(int threads, int rpt) {
    int nb = 0;
#define SSM_CASE(TH, RR) \
    if (threads == TH && rpt == RR) { \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair<KIND, T, TH, RR>, TH, 0) != cudaSuccess) nb = 0; \
        return nb; }
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    return 0;
}
template <int KIND>
static int occ_dispatch2(int threads, int rpt) {
    int nb = 0;
#define SSM_CASE(TH, RR) \
    if (threads == TH && rpt == RR) { \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pair2<KIND, TH, RR>, TH, 0) != cudaSuccess) nb = 0; \
        return nb; }
    SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    return 0;
}

// Resident blocks per SM of a pair kernel shape (0 if unknown / no device).
int pair_blocks_per_sm(int kind, bool fp32, bool vec2, int threads, int rpt) {
    if (fp32 && vec2) {
        if (kind == PK_NEWTON3) return occ_dispatch2<PK_NEWTON3>(threads, rpt);
        if (kind == PK_DRIFT3) return occ_dispatch2<PK_DRIFT3>(threads, rpt);
        return 0;
    }
    switch (kind) {
    case PK_DRIFT1: return fp32 ? occ_dispatch<PK_DRIFT1, float>(threads, rpt) : occ_dispatch<PK_DRIFT1, double>(threads, rpt);
    case PK_DRIFT3: return fp32 ? occ_dispatch<PK_DRIFT3, float>(threads, rpt) : occ_dispatch<PK_DRIFT3, double>(threads, rpt);
    case PK_NEWTON3: return fp32 ? occ_dispatch<PK_NEWTON3, float>(threads, rpt) : occ_dispatch<PK_NEWTON3, double>(threads, rpt);
    }
    return 0;
}

// Candidate launch shapes of a pair kind for the autotuner: {vec2, threads, rpt}.
int pair_shape_candidates(int kind, bool fp32, int (*out)[3], int max_out) {
    int n = 0;
    auto add = [&](int v, int th, int r) { if (n < max_out) { out[n][0] = v; out[n][1] = th; out[n][2] = r; ++n; } };
#define SSM_CASE(TH, RR) add(0, TH, RR);
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    if (fp32 && (kind == PK_NEWTON3 || kind == PK_DRIFT3)) {
#define SSM_CASE(TH, RR) add(1, TH, RR);
        SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    }
    return n;
}

}  // namespace ssm
