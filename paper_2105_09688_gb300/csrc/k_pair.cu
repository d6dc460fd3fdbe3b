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
// Host launchers.  Launch shapes (threads, targets per thread) are compiled-in
// candidates; the chunk count comes from the plan.
// ---------------------------------------------------------------------------
template <int KIND, typename T, int THREADS, int R>
static cudaError_t launch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                          int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
    const int64_t tiles = (N + THREADS * R - 1) / (THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)p.chunks);
    k_pair<KIND, T, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part);
    return cudaGetLastError();
}

// The (threads, rpt) shapes each kind is compiled for.
#define SSM_PAIR_SHAPES(X) X(128, 2) X(128, 4) X(256, 2) X(256, 4) X(128, 8)

template <int KIND, typename T>
static cudaError_t dispatch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                            int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
#define SSM_CASE(TH, RR) \
    if (p.threads == TH && p.rpt == RR) return launch<KIND, T, TH, RR>(p, src, tgt, act, cnt, N, Np, scale, part, st);
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t pair_sums(int kind, bool fp32, const Plan &p, const double *src, const double *tgt, const int *act,
                      const int *cnt, int64_t N, int64_t Np, double scale, double *part, cudaStream_t st) {
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

bool pair_shape_supported(int threads, int rpt) {
#define SSM_CASE(TH, RR) if (threads == TH && rpt == RR) return true;
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    return false;
}

}  // namespace ssm
