// k_mlp.cu -- learned initial guess for step 1 of the coupled workload.
//
// A small network predicts, from particle i's state and the moments of the
// empirical measure, the converged pair sum S(Y*_i) = (1/N) sum_j (X_j - Y*_i) /
// (1 + |X_j - Y*_i|^2) of step 1 (§2.3, eq. SSTM:scheme 1).  The start Y^0 is then
// the exact root of the per-particle cubic u = X + h(-u|u|^2 + 0.5 S_pred), so the
// network only has to learn the smooth measure-dependent part.  The Newton-type
// passes of k_newton_update run from that start; a particle whose residual still
// exceeds the tolerance after `ws_passes` passes restarts from the plain start
// Y = X (plain Newton judges the learned start).  The paper has no counterpart.
//
// Network: features f = (x_1, x_2, x_3, m_1..m_4 per coordinate (12), h) = 16,
// standardised with the training set's mean and standard deviation;
// 16 -> 64 -> 64 -> 64 -> 3, SiLU on the hidden layers, weights stored in BF16,
// biases and all arithmetic in FP32.  The whole forward is ~9.4k FMA per
// particle, ~0.2% of a step at N = 2^18, so it runs on CUDA-core FMAs with the
// weights broadcast from shared memory.
//
// Training (ssm_ws_train) is plain minibatch Adam on the mean squared error of
// the standardised outputs, with FP32 master weights and the forward run on the
// BF16-rounded weights; every step runs in the kernels below.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ssm.h"
#include "particle_ops.cuh"
#include "ssm_device.cuh"

namespace ssm {

constexpr int NI = 16, NH = 64, NO = 3;
// Blob layout, in 32-bit words.
constexpr uint32_t WS_MAGIC = 0x57534D53u, WS_VERSION = 1u;
constexpr int OFF_FMEAN = 8, OFF_FSTD = 24, OFF_YMEAN = 40, OFF_YSTD = 44;
constexpr int OFF_B1 = 48, OFF_B2 = 112, OFF_B3 = 176, OFF_B4 = 240;
constexpr int OFF_W = 244;                               // bf16 weights start here
constexpr int NW1 = NH * NI, NW2 = NH * NH, NW3 = NH * NH, NW4 = 4 * NH;   // W4 padded to 4 rows
constexpr int BLOB_WORDS = OFF_W + (NW1 + NW2 + NW3 + NW4) / 2;
constexpr size_t BLOB_BYTES = (size_t)BLOB_WORDS * 4;
// Master parameter vector (training): W1, b1, W2, b2, W3, b3, W4 (3 x 64), b4.
constexpr int P_W1 = 0, P_B1 = P_W1 + NW1, P_W2 = P_B1 + NH, P_B2 = P_W2 + NW2, P_W3 = P_B2 + NH, P_B3 = P_W3 + NW3,
              P_W4 = P_B3 + NH, P_B4 = P_W4 + NO * NH, NPARAM = P_B4 + NO;

struct Net {                    // FP32 view of the network in shared memory
    float W1[NW1], W2[NW2], W3[NW3], W4[NO * NH];
    float b1[NH], b2[NH], b3[NH], b4[4];
    float fm[NI], fs[NI], ym[4], ys[4];
};

__device__ __forceinline__ float silu(float s) { return s / (1.0f + __expf(-s)); }
__device__ __forceinline__ float dsilu(float s) {
    const float g = 1.0f / (1.0f + __expf(-s));
    return g * (1.0f + s * (1.0f - g));
}

// Cooperative load of a blob into shared memory (block-wide).
__device__ void load_net(const float *__restrict__ blob, Net &n) {
    const __nv_bfloat16 *w = reinterpret_cast<const __nv_bfloat16 *>(blob + OFF_W);
    for (int k = threadIdx.x; k < NW1; k += blockDim.x) n.W1[k] = __bfloat162float(w[k]);
    for (int k = threadIdx.x; k < NW2; k += blockDim.x) n.W2[k] = __bfloat162float(w[NW1 + k]);
    for (int k = threadIdx.x; k < NW3; k += blockDim.x) n.W3[k] = __bfloat162float(w[NW1 + NW2 + k]);
    for (int k = threadIdx.x; k < NO * NH; k += blockDim.x) n.W4[k] = __bfloat162float(w[NW1 + NW2 + NW3 + k]);
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        n.b1[k] = blob[OFF_B1 + k];
        n.b2[k] = blob[OFF_B2 + k];
        n.b3[k] = blob[OFF_B3 + k];
    }
    if (threadIdx.x < 4) {
        n.b4[threadIdx.x] = blob[OFF_B4 + threadIdx.x];
        n.ym[threadIdx.x] = blob[OFF_YMEAN + threadIdx.x];
        n.ys[threadIdx.x] = blob[OFF_YSTD + threadIdx.x];
    }
    if (threadIdx.x < NI) {
        n.fm[threadIdx.x] = blob[OFF_FMEAN + threadIdx.x];
        n.fs[threadIdx.x] = blob[OFF_FSTD + threadIdx.x];
    }
}

// Per-thread activation column in shared memory, after the Net: element k of
// thread t at col[k * blockDim.x] (col = base + t), so the outer loops over
// neurons need not be unrolled (registers hold only the current layer's input).
__device__ __forceinline__ float *act_column() {
    extern __shared__ float smem[];
    return smem + sizeof(Net) / sizeof(float) + threadIdx.x;
}

// One dense layer: out[j] = act(b[j] + sum_k W[j*NIN + k] in[k]) into the column.
template <int NIN, bool STORE>
__device__ __forceinline__ void dense_silu(const float *W, const float *bias, const float *in, float *col, float *zs,
                                           float *as) {
    const int T = blockDim.x;
    for (int j = 0; j < NH; ++j) {
        float s = bias[j];
#pragma unroll
        for (int k = 0; k < NIN; ++k) s = fmaf(W[j * NIN + k], in[k], s);
        const float a = silu(s);
        col[j * T] = a;
        if (STORE) { zs[j] = s; as[j] = a; }
    }
}

// Forward pass of one sample (standardised features in f, standardised outputs).
// With STORE, pre-activations z and activations a of the three hidden layers go
// to zs/as ([3][64] each).
template <bool STORE>
__device__ __forceinline__ void forward(const Net &n, const float *f, float *out, float *zs, float *as) {
    float *col = act_column();
    const int T = blockDim.x;
    float a[NH];
    dense_silu<NI, STORE>(n.W1, n.b1, f, col, zs, as);
#pragma unroll
    for (int k = 0; k < NH; ++k) a[k] = col[k * T];
    dense_silu<NH, STORE>(n.W2, n.b2, a, col, STORE ? zs + NH : nullptr, STORE ? as + NH : nullptr);
#pragma unroll
    for (int k = 0; k < NH; ++k) a[k] = col[k * T];
    dense_silu<NH, STORE>(n.W3, n.b3, a, col, STORE ? zs + 2 * NH : nullptr, STORE ? as + 2 * NH : nullptr);
#pragma unroll
    for (int k = 0; k < NH; ++k) a[k] = col[k * T];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        float s = n.b4[o];
#pragma unroll
        for (int k = 0; k < NH; ++k) s = fmaf(n.W4[o * NH + k], a[k], s);
        out[o] = s;
    }
}


// The prediction used for the start: the network's S_pred, plus -- when the previous
// step of this run converged from a prediction of this particle -- that step's error
// S(Y*) - S_pred, kept per particle.  The network sees the particle and the moments
// of the measure, not the particular sample of N particles; the part of S it cannot
// predict, the sample's fluctuation about its law (~1/sqrt(N)), is a smooth field
// that moves little in one step, so the previous error removes most of it (at
// N = 2^18 the start's error falls from ~6e-7 to ~4e-8, below the ~1e-7 at which one
// pass and the residual bound suffice).  The raw prediction is kept for the next step.
__device__ __forceinline__ void corrected_start(const double (&X)[3], const float (&S)[3], double h, double *y,
                                                const double *__restrict__ sconv, float *__restrict__ spred,
                                                bool corr, int64_t i, int64_t Np) {
    float Su[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Su[c] = S[c];
        if (corr) Su[c] += f64_to_f32_fast(sconv[c * Np + i] - (double)spred[c * Np + i]);
        spred[c * Np + i] = S[c];
    }
    cubic_start<3>(X, Su, h, y + i, Np);
}

// Learned start of step 1 on the CUDA cores (FFMA, weights broadcast from shared memory).
__global__ void __launch_bounds__(128)
k_ws_start(const double *__restrict__ x, double *__restrict__ y, const float *__restrict__ blob,
           const double *__restrict__ mom, int64_t N, int64_t Np, double h, const double *__restrict__ sconv,
           float *__restrict__ spred, const int *__restrict__ ws_prev) {
    extern __shared__ float smem[];
    Net &n = *reinterpret_cast<Net *>(smem);
    load_net(blob, n);
    __syncthreads();
    const bool corr = *ws_prev != 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double X[3];
        float f[NI];
#pragma unroll
        for (int c = 0; c < 3; ++c) { X[c] = x[c * Np + i]; f[c] = (float)X[c]; }
#pragma unroll
        for (int k = 0; k < 12; ++k) f[3 + k] = (float)mom[k];
        f[15] = (float)h;
#pragma unroll
        for (int k = 0; k < NI; ++k) f[k] = (f[k] - n.fm[k]) / n.fs[k];
        float o[NO];
        forward<false>(n, f, o, nullptr, nullptr);
        float S[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) S[c] = o[c] * n.ys[c] + n.ym[c];
        corrected_start(X, S, h, y, sconv, spred, corr, i, Np);
    }
}

// ---- the same start on the tensor cores: mma.sync m16n8k16, BF16 operands, FP32
// accumulate -------------------------------------------------------------------------
// A warp takes 32 particles at a time and pushes each 16-particle half through the four
// layers: activations [16 x K] are the A operand, the stored BF16 weights (row-major
// [out][in], i.e. the B operand in column order) are read from shared memory, the
// FP32 accumulators get bias and SiLU and become, register for register, the A operand
// of the next layer (the m16n8 accumulator layout of two adjacent n-tiles is the
// m16k16 operand layout).  Each activation enters as two BF16 parts, hi = bf16(a) and
// lo = bf16(a - hi), with two products per tile: the weights are exact in BF16, so
// the layer is computed to ~2^-16 relative of the activations instead of 2^-8 -- the
// start carries the previous step's error forward, which cancels only the smooth part
// of the prediction error, not rounding that jumps from step to step.  Rows of W are
// padded by 8 elements so that the fragment loads of a warp fall in distinct banks.
constexpr int MW_LD1 = NI + 8, MW_LD = NH + 8;
constexpr int MW_W2 = NH * MW_LD1, MW_W3 = MW_W2 + NH * MW_LD, MW_W4 = MW_W3 + NH * MW_LD, MW_TOT = MW_W4 + 8 * MW_LD;
constexpr int MMA_WARPS = 4;
struct MmaNet {
    __nv_bfloat16 w[MW_TOT];                          // W1 | W2 | W3 | W4 (8 rows; rows 3..7 zero)
    float b1[NH], b2[NH], b3[NH], b4[8];
    float fm[NI], fsi[NI], ym[4], ys[4];
    __nv_bfloat16 feat[MMA_WARPS][2][32][NI + 8];     // a warp's staged, standardised features (hi, lo)
    float out[MMA_WARPS][32][4];                      // a warp's network outputs
};

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float silu_fast(float s) { return s * rcp_approx(1.0f + ex2_approx(-1.4426950408889634f * s)); }

// hi = bf16(v), lo = bf16(v - hi) for a pair of values, packed as two BF16 pairs.
__device__ __forceinline__ void split_bf16(float v0, float v1, unsigned &hi, unsigned &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
    hi = *reinterpret_cast<const unsigned *>(&h);
    lo = *reinterpret_cast<const unsigned *>(&l);
}

// One hidden layer: d[j] = (A_hi + A_lo) . W^T for the 8 n-tiles of 64 outputs (KT
// k-tiles of input), then bias + SiLU, split and repacked in place as the next
// layer's 4 k-tiles.
template <int KT>
__device__ __forceinline__ void mma_hidden(const __nv_bfloat16 *W, int ld, const float *bias, unsigned (&ah)[4][4],
                                           unsigned (&al)[4][4], int g, int t) {
    float d[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.0f;
        const __nv_bfloat16 *row = W + (8 * j + g) * ld + 2 * t;
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const unsigned b0 = lds32(row + 16 * kk), b1 = lds32(row + 16 * kk + 8);
            mma_bf16(d[j], al[kk], b0, b1);
            mma_bf16(d[j], ah[kk], b0, b1);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float c0 = bias[8 * j + 2 * t], c1 = bias[8 * j + 2 * t + 1];
        split_bf16(silu_fast(d[j][0] + c0), silu_fast(d[j][1] + c1), ah[j >> 1][(j & 1) * 2 + 0],
                   al[j >> 1][(j & 1) * 2 + 0]);
        split_bf16(silu_fast(d[j][2] + c0), silu_fast(d[j][3] + c1), ah[j >> 1][(j & 1) * 2 + 1],
                   al[j >> 1][(j & 1) * 2 + 1]);
    }
}

__global__ void __launch_bounds__(MMA_WARPS * 32)
k_ws_start_mma(const double *__restrict__ x, double *__restrict__ y, const float *__restrict__ blob,
               const double *__restrict__ mom, int64_t N, int64_t Np, double h, const double *__restrict__ sconv,
               float *__restrict__ spred, const int *__restrict__ ws_prev) {
    __shared__ MmaNet sm;
    const bool corr = *ws_prev != 0;
    const __nv_bfloat16 *wg = reinterpret_cast<const __nv_bfloat16 *>(blob + OFF_W);
    for (int k = threadIdx.x; k < NW1; k += blockDim.x) sm.w[(k / NI) * MW_LD1 + k % NI] = wg[k];
    for (int k = threadIdx.x; k < NW2; k += blockDim.x) sm.w[MW_W2 + (k / NH) * MW_LD + k % NH] = wg[NW1 + k];
    for (int k = threadIdx.x; k < NW3; k += blockDim.x) sm.w[MW_W3 + (k / NH) * MW_LD + k % NH] = wg[NW1 + NW2 + k];
    for (int k = threadIdx.x; k < 8 * NH; k += blockDim.x)
        sm.w[MW_W4 + (k / NH) * MW_LD + k % NH] = k < NO * NH ? wg[NW1 + NW2 + NW3 + k] : __float2bfloat16_rn(0.0f);
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        sm.b1[k] = blob[OFF_B1 + k];
        sm.b2[k] = blob[OFF_B2 + k];
        sm.b3[k] = blob[OFF_B3 + k];
    }
    if (threadIdx.x < 8) sm.b4[threadIdx.x] = threadIdx.x < NO ? blob[OFF_B4 + threadIdx.x] : 0.0f;
    if (threadIdx.x < 4) {
        sm.ym[threadIdx.x] = blob[OFF_YMEAN + threadIdx.x];
        sm.ys[threadIdx.x] = blob[OFF_YSTD + threadIdx.x];
    }
    if (threadIdx.x < NI) {
        sm.fm[threadIdx.x] = blob[OFF_FMEAN + threadIdx.x];
        sm.fsi[threadIdx.x] = 1.0f / blob[OFF_FSTD + threadIdx.x];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16(*feat)[NI + 8] = sm.feat[warp][0];
    __nv_bfloat16(*featl)[NI + 8] = sm.feat[warp][1];
    float(*out)[4] = sm.out[warp];
    for (int64_t base = ((int64_t)blockIdx.x * MMA_WARPS + warp) * 32; base < N;
         base += (int64_t)gridDim.x * MMA_WARPS * 32) {
        const int64_t i = base + lane;
        double X[3] = {0.0, 0.0, 0.0};
        if (i < N)
#pragma unroll
            for (int c = 0; c < 3; ++c) X[c] = x[c * Np + i];
        float f[NI];
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] = f64_to_f32_fast(X[c]);
#pragma unroll
        for (int k = 0; k < 12; ++k) f[3 + k] = (float)mom[k];
        f[15] = (float)h;
#pragma unroll
        for (int k = 0; k < NI; k += 2)
            split_bf16((f[k] - sm.fm[k]) * sm.fsi[k], (f[k + 1] - sm.fm[k + 1]) * sm.fsi[k + 1],
                       *reinterpret_cast<unsigned *>(&feat[lane][k]), *reinterpret_cast<unsigned *>(&featl[lane][k]));
        __syncwarp();
#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = 16 * mt + g, r1 = r0 + 8;
            unsigned ah[4][4], al[4][4];
            ah[0][0] = lds32(&feat[r0][2 * t]);
            ah[0][1] = lds32(&feat[r1][2 * t]);
            ah[0][2] = lds32(&feat[r0][2 * t + 8]);
            ah[0][3] = lds32(&feat[r1][2 * t + 8]);
            al[0][0] = lds32(&featl[r0][2 * t]);
            al[0][1] = lds32(&featl[r1][2 * t]);
            al[0][2] = lds32(&featl[r0][2 * t + 8]);
            al[0][3] = lds32(&featl[r1][2 * t + 8]);
            mma_hidden<1>(sm.w, MW_LD1, sm.b1, ah, al, g, t);
            mma_hidden<4>(sm.w + MW_W2, MW_LD, sm.b2, ah, al, g, t);
            mma_hidden<4>(sm.w + MW_W3, MW_LD, sm.b3, ah, al, g, t);
            float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const __nv_bfloat16 *row = sm.w + MW_W4 + g * MW_LD + 2 * t;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const unsigned b0 = lds32(row + 16 * kk), b1 = lds32(row + 16 * kk + 8);
                mma_bf16(o, al[kk], b0, b1);
                mma_bf16(o, ah[kk], b0, b1);
            }
            if (t < 2) {   // columns 2t, 2t + 1 of rows r0, r1 (outputs 0..2; column 3 is padding)
                out[r0][2 * t] = o[0] + sm.b4[2 * t];
                out[r0][2 * t + 1] = o[1] + sm.b4[2 * t + 1];
                out[r1][2 * t] = o[2] + sm.b4[2 * t];
                out[r1][2 * t + 1] = o[3] + sm.b4[2 * t + 1];
            }
        }
        __syncwarp();
        if (i < N) {
            float S[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) S[c] = out[lane][c] * sm.ys[c] + sm.ym[c];
            corrected_start(X, S, h, y, sconv, spred, corr, i, Np);
        }
        __syncwarp();
    }
}

// Network outputs (unstandardised) for raw feature rows (ssm_ws_predict).
__global__ void __launch_bounds__(128)
k_ws_predict(const float *__restrict__ blob, const float *__restrict__ feat, int64_t n_rows, float *__restrict__ out) {
    extern __shared__ float smem[];
    Net &n = *reinterpret_cast<Net *>(smem);
    load_net(blob, n);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += (int64_t)gridDim.x * blockDim.x) {
        float f[NI], o[NO];
#pragma unroll
        for (int k = 0; k < NI; ++k) f[k] = (feat[r * NI + k] - n.fm[k]) / n.fs[k];
        forward<false>(n, f, o, nullptr, nullptr);
#pragma unroll
        for (int c = 0; c < NO; ++c) out[r * NO + c] = o[c] * n.ys[c] + n.ym[c];
    }
}

// Training-data rows from the last step: X_n rebuilt from its converged root
// (X = Y* - h v(Y*), exact up to the residual tolerance), the moments of X_n,
// h, and the label S(Y*).
__global__ void k_ws_collect(const double *__restrict__ y, const double *__restrict__ sconv,
                             const double *__restrict__ mom_prev, int64_t N, int64_t Np, double h, int64_t stride,
                             int64_t offset, int64_t rows, float *__restrict__ feat, float *__restrict__ label) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = offset + r * stride;
        double Y[3], S[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) { Y[c] = y[c * Np + i]; S[c] = sconv[c * Np + i]; }
        const double yy = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            feat[r * NI + c] = (float)(Y[c] - h * (-Y[c] * yy + 0.5 * S[c]));
            label[r * NO + c] = (float)S[c];
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) feat[r * NI + 3 + k] = (float)mom_prev[k];
        feat[r * NI + 15] = (float)h;
    }
}

// ---- training kernels -------------------------------------------------------
// Per-sample buffers (row b of the batch): fz = standardised features [16],
// Z = pre-activations [192], A = activations [192], D = deltas [192 + 3].

__global__ void __launch_bounds__(128)
k_train_fwd(const float *__restrict__ blob, const float *__restrict__ feat, const float *__restrict__ label,
            const int *__restrict__ perm, int64_t b0, int B, float *__restrict__ FZ, float *__restrict__ Z,
            float *__restrict__ A, float *__restrict__ D, double *__restrict__ loss) {
    extern __shared__ float smem[];
    Net &n = *reinterpret_cast<Net *>(smem);
    load_net(blob, n);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const int64_t r = perm ? (int64_t)perm[b0 + b] : b0 + b;
        float f[NI], o[NO];
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            f[k] = (feat[r * NI + k] - n.fm[k]) / n.fs[k];
            FZ[(int64_t)b * NI + k] = f[k];
        }
        forward<true>(n, f, o, Z + (int64_t)b * 3 * NH, A + (int64_t)b * 3 * NH);
#pragma unroll
        for (int c = 0; c < NO; ++c) {
            const float t = (label[r * NO + c] - n.ym[c]) / n.ys[c];
            const float e = o[c] - t;
            l += (double)e * e;
            D[(int64_t)b * (3 * NH + NO) + 3 * NH + c] = 2.0f * e / (float)(B * NO);   // d loss / d out
        }
    }
    // block sum of the squared errors
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    __shared__ double ws[4];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, ws[0] + ws[1] + ws[2] + ws[3]);
}

__global__ void __launch_bounds__(128)
k_train_bwd(const float *__restrict__ blob, int B, const float *__restrict__ Z, float *__restrict__ D) {
    extern __shared__ float smem[];
    Net &n = *reinterpret_cast<Net *>(smem);
    load_net(blob, n);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *z = Z + (int64_t)b * 3 * NH;
    float *dl = D + (int64_t)b * (3 * NH + NO);
    float g[NO], dv[NH];
#pragma unroll
    for (int c = 0; c < NO; ++c) g[c] = dl[3 * NH + c];
    // delta of hidden layer 3: (W4^T g) * silu'(z3)
    for (int k = 0; k < NH; ++k) {
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) s = fmaf(n.W4[o * NH + k], g[o], s);
        dl[2 * NH + k] = s * dsilu(z[2 * NH + k]);
    }
    // delta of layer 2 from layer 3 (through W3), then layer 1 from layer 2 (W2)
#pragma unroll
    for (int k = 0; k < NH; ++k) dv[k] = dl[2 * NH + k];
    for (int k = 0; k < NH; ++k) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < NH; ++j) s = fmaf(n.W3[j * NH + k], dv[j], s);
        dl[NH + k] = s * dsilu(z[NH + k]);
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) dv[k] = dl[NH + k];
    for (int k = 0; k < NH; ++k) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < NH; ++j) s = fmaf(n.W2[j * NH + k], dv[j], s);
        dl[k] = s * dsilu(z[k]);
    }
}

// Gradient of every parameter over the batch, in two deterministic stages: block
// (x, c) sums samples [c Bc, (c + 1) Bc) of its 128 parameters in sample order
// into part[c][p] (one thread per parameter and chunk, WG_CHUNKS chunks: enough
// blocks to fill the device), then k_train_wgrad_sum adds the chunks in order.
constexpr int WG_CHUNKS = 64;
__global__ void __launch_bounds__(128)
k_train_wgrad(int B, const float *__restrict__ FZ, const float *__restrict__ A, const float *__restrict__ D,
              float *__restrict__ part) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const int bc = (B + WG_CHUNKS - 1) / WG_CHUNKS;
    const int b0 = blockIdx.y * bc, b1 = b0 + bc < B ? b0 + bc : B;
    constexpr int DS = 3 * NH + NO;
    int dj, in_k = -1, in_layer = -1;   // delta column, input column (-1: bias), input kind
    if (p < P_B1) { dj = (p - P_W1) / NI; in_k = (p - P_W1) % NI; in_layer = 0; }
    else if (p < P_W2) { dj = p - P_B1; }
    else if (p < P_B2) { dj = NH + (p - P_W2) / NH; in_k = (p - P_W2) % NH; in_layer = 1; }
    else if (p < P_W3) { dj = NH + (p - P_B2); }
    else if (p < P_B3) { dj = 2 * NH + (p - P_W3) / NH; in_k = (p - P_W3) % NH; in_layer = 2; }
    else if (p < P_W4) { dj = 2 * NH + (p - P_B3); }
    else if (p < P_B4) { dj = 3 * NH + (p - P_W4) / NH; in_k = (p - P_W4) % NH; in_layer = 3; }
    else { dj = 3 * NH + (p - P_B4); }
    float s = 0.f;
    for (int b = b0; b < b1; ++b) {
        const float dv = D[(int64_t)b * DS + dj];
        float av = 1.0f;
        if (in_layer == 0) av = FZ[(int64_t)b * NI + in_k];
        else if (in_layer > 0) av = A[(int64_t)b * 3 * NH + (in_layer - 1) * NH + in_k];
        s = fmaf(dv, av, s);
    }
    part[(int64_t)blockIdx.y * NPARAM + p] = s;
}
__global__ void k_train_wgrad_sum(const float *__restrict__ part, float *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float s = 0.f;
    for (int c = 0; c < WG_CHUNKS; ++c) s += part[(int64_t)c * NPARAM + p];
    grad[p] = s;
}
static cudaError_t launch_wgrad(int B, const float *fz, const float *a, const float *d, float *part, float *grad) {
    k_train_wgrad<<<dim3((NPARAM + 127) / 128, WG_CHUNKS), 128>>>(B, fz, a, d, part);
    k_train_wgrad_sum<<<(NPARAM + 127) / 128, 128>>>(part, grad);
    return cudaGetLastError();
}

// Adam on the FP32 master weights; writes the BF16-rounded blob used by the forward.
__global__ void k_adam(const float *__restrict__ grad, float *__restrict__ m, float *__restrict__ v,
                       float *__restrict__ w, float *__restrict__ blob, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float g = grad[p];
    const float mn = 0.9f * m[p] + 0.1f * g, vn = 0.999f * v[p] + 0.001f * g * g;
    m[p] = mn;
    v[p] = vn;
    const float wn = w[p] - lr * (mn * c1) / (sqrtf(vn * c2) + 1e-8f);
    w[p] = wn;
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(blob + OFF_W);
    if (p < P_B1) wb[p - P_W1] = __float2bfloat16_rn(wn);
    else if (p < P_W2) blob[OFF_B1 + (p - P_B1)] = wn;
    else if (p < P_B2) wb[NW1 + (p - P_W2)] = __float2bfloat16_rn(wn);
    else if (p < P_W3) blob[OFF_B2 + (p - P_B2)] = wn;
    else if (p < P_B3) wb[NW1 + NW2 + (p - P_W3)] = __float2bfloat16_rn(wn);
    else if (p < P_W4) blob[OFF_B3 + (p - P_B3)] = wn;
    else if (p < P_B4) wb[NW1 + NW2 + NW3 + (p - P_W4)] = __float2bfloat16_rn(wn);
    else blob[OFF_B4 + (p - P_B4)] = wn;
}

constexpr size_t NET_SMEM = sizeof(Net) + sizeof(float) * NH * 128;   // net + activation columns (128 threads)

bool blob_ok(const void *blob, size_t bytes) {
    if (!blob || bytes < BLOB_BYTES) return false;
    uint32_t h[2];
    memcpy(h, blob, sizeof h);
    return h[0] == WS_MAGIC && h[1] == WS_VERSION;
}

cudaError_t set_smem_limits() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_ws_start, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NET_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ws_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NET_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NET_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NET_SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

// Start of step 1 from the previous step's converged pair sums (ssm_opts.carry_start;
// no counterpart in the paper, a warm start of the same solve): from the second step
// of a run on, Y_i starts at the root of u = X_i + h(-u|u|^2 + S*_i / 2), S*_i the
// particle's converged pair sum of the previous step (sconv), which the step's own sum
// differs from by how far the particle and the measure moved in one step -- O(sqrt h),
// so the start is ~1e-5 from the root instead of h|v(X_i)| ~ 1e-2 for Y = X, and
// step 1 needs one pass less.  *valid == 0 (the first step, or a state that was set)
// keeps the plain start that k_newton_begin wrote.
template <int D>
__global__ void k_carry_start(const double *__restrict__ x, double *__restrict__ y, const double *__restrict__ sconv,
                              int64_t N, int64_t Np, double h, const int *__restrict__ valid) {
    if (*valid == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double X[D];
        float S[D];
#pragma unroll
        for (int c = 0; c < D; ++c) { X[c] = x[c * Np + i]; S[c] = f64_to_f32_fast(sconv[c * Np + i]); }
        cubic_start<D>(X, S, h, y + i, Np);
    }
}

cudaError_t launch_carry_start(ssm_ctx *c) {
    int64_t blocks = (c->N + 255) / 256;
    if (blocks > (int64_t)c->sms * 8) blocks = (int64_t)c->sms * 8;
    if (c->d == 1)
        k_carry_start<1><<<(unsigned)blocks, 256, 0, c->st>>>(c->x, c->y, c->sconv, c->N, c->Np, c->h, c->ws_prev);
    else
        k_carry_start<3><<<(unsigned)blocks, 256, 0, c->st>>>(c->x, c->y, c->sconv, c->N, c->Np, c->h, c->ws_prev);
    return cudaGetLastError();
}

// The learned start on the form the context selects (ssm_opts.ws_forward): 0 =
// tensor-core mma.sync, 1 = CUDA-core FFMA.
cudaError_t ws_forward_start(ssm_ctx *c) {
    if (c->opt.ws_forward == 1) {
        cudaError_t e = set_smem_limits();
        if (e != cudaSuccess) return e;
        int64_t blocks = (c->N + 127) / 128;
        if (blocks > (int64_t)c->sms * 8) blocks = (int64_t)c->sms * 8;
        k_ws_start<<<(unsigned)blocks, 128, NET_SMEM, c->st>>>(c->x, c->y, c->ws_w, c->mom, c->N, c->Np, c->h,
                                                              c->sconv, c->spred, c->ws_prev);
    } else {
        int64_t blocks = (c->N + MMA_WARPS * 32 - 1) / (MMA_WARPS * 32);
        if (blocks > (int64_t)c->sms * 8) blocks = (int64_t)c->sms * 8;
        k_ws_start_mma<<<(unsigned)blocks, MMA_WARPS * 32, 0, c->st>>>(c->x, c->y, c->ws_w, c->mom, c->N, c->Np,
                                                                       c->h, c->sconv, c->spred, c->ws_prev);
    }
    return cudaGetLastError();
}

// splitmix64, for the host-side shuffles and initial weights of training.
static uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double unit(uint64_t &s) { return ((splitmix(s) >> 11) + 0.5) * 0x1p-53; }

static uint16_t bf16_bits(float f) {   // round to nearest even
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Host: fill a blob from master parameters and statistics.
static void pack_blob(const std::vector<float> &w, const float *fm, const float *fs, const float *ym, const float *ys,
                      std::vector<uint32_t> &blob) {
    blob.assign(BLOB_WORDS, 0u);
    blob[0] = WS_MAGIC; blob[1] = WS_VERSION; blob[2] = NI; blob[3] = NH; blob[4] = NO;
    float *fb = reinterpret_cast<float *>(blob.data());
    for (int k = 0; k < NI; ++k) { fb[OFF_FMEAN + k] = fm[k]; fb[OFF_FSTD + k] = fs[k]; }
    for (int k = 0; k < 4; ++k) { fb[OFF_YMEAN + k] = k < NO ? ym[k] : 0.f; fb[OFF_YSTD + k] = k < NO ? ys[k] : 1.f; }
    for (int k = 0; k < NH; ++k) { fb[OFF_B1 + k] = w[P_B1 + k]; fb[OFF_B2 + k] = w[P_B2 + k]; fb[OFF_B3 + k] = w[P_B3 + k]; }
    for (int k = 0; k < NO; ++k) fb[OFF_B4 + k] = w[P_B4 + k];
    uint16_t *wb = reinterpret_cast<uint16_t *>(fb + OFF_W);
    for (int k = 0; k < NW1; ++k) wb[k] = bf16_bits(w[P_W1 + k]);
    for (int k = 0; k < NW2; ++k) wb[NW1 + k] = bf16_bits(w[P_W2 + k]);
    for (int k = 0; k < NW3; ++k) wb[NW1 + NW2 + k] = bf16_bits(w[P_W3 + k]);
    for (int k = 0; k < NO * NH; ++k) wb[NW1 + NW2 + NW3 + k] = bf16_bits(w[P_W4 + k]);
}

// Host: master parameters of a blob (weights as their BF16 values).
static void unpack_blob(const void *src, std::vector<float> &w) {
    const float *fb = reinterpret_cast<const float *>(src);
    const uint16_t *wb = reinterpret_cast<const uint16_t *>(fb + OFF_W);
    auto f = [](uint16_t h) { uint32_t u = (uint32_t)h << 16; float v; memcpy(&v, &u, 4); return v; };
    w.assign(NPARAM, 0.f);
    for (int k = 0; k < NW1; ++k) w[P_W1 + k] = f(wb[k]);
    for (int k = 0; k < NW2; ++k) w[P_W2 + k] = f(wb[NW1 + k]);
    for (int k = 0; k < NW3; ++k) w[P_W3 + k] = f(wb[NW1 + NW2 + k]);
    for (int k = 0; k < NO * NH; ++k) w[P_W4 + k] = f(wb[NW1 + NW2 + NW3 + k]);
    for (int k = 0; k < NH; ++k) { w[P_B1 + k] = fb[OFF_B1 + k]; w[P_B2 + k] = fb[OFF_B2 + k]; w[P_B3 + k] = fb[OFF_B3 + k]; }
    for (int k = 0; k < NO; ++k) w[P_B4 + k] = fb[OFF_B4 + k];
}

}  // namespace ssm

using namespace ssm;

namespace {
ssm_status cst(cudaError_t e) {
    return e == cudaSuccess ? SSM_OK : (e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA);
}
struct DevBuf {   // scoped device allocation for the training / checking entry points
    void *p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, n ? n : 1); }
    ~DevBuf() { if (p) cudaFree(p); }
    template <typename T> T *as() { return reinterpret_cast<T *>(p); }
};
}  // namespace

extern "C" {

size_t ssm_ws_blob_bytes(void) { return BLOB_BYTES; }

ssm_status ssm_ws_load(ssm_ctx *c, const void *blob, size_t bytes) {
    if (!c || !blob_ok(blob, bytes)) return SSM_EINVAL;
    if (c->coef != SSM_COEF_COUPLED3D) return SSM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->ws_w, blob, BLOB_BYTES, cudaMemcpyHostToDevice, c->st);
    // a new network: no previous prediction error to carry over
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws_prev, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cst(e);
    c->ws_loaded = 1;
    if (c->graph_ready) { cudaGraphExecDestroy(c->gexec); c->graph_ready = false; }
    return SSM_OK;
}

ssm_status ssm_ws_collect(ssm_ctx *c, int64_t stride, int64_t offset, float *feat, float *label, int64_t *rows_out) {
    if (!c || !feat || !label || stride < 1 || offset < 0 || c->coef != SSM_COEF_COUPLED3D) return SSM_EINVAL;
    if (c->n < 1) return SSM_ESTATE;
    const int64_t rows = offset < c->N ? (c->N - offset + stride - 1) / stride : 0;
    if (rows_out) *rows_out = rows;
    if (rows == 0) return SSM_OK;
    DevBuf df, dl;
    cudaError_t e = df.alloc(sizeof(float) * NI * rows);
    if (e == cudaSuccess) e = dl.alloc(sizeof(float) * NO * rows);
    if (e == cudaSuccess) {
        const int64_t blocks = (rows + 255) / 256 < 1216 ? (rows + 255) / 256 : 1216;
        k_ws_collect<<<(unsigned)blocks, 256, 0, c->st>>>(c->y, c->sconv, c->mom_prev, c->N, c->Np, c->h, stride,
                                                          offset, rows, df.as<float>(), dl.as<float>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(feat, df.p, sizeof(float) * NI * rows, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(label, dl.p, sizeof(float) * NO * rows, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return cst(e);
}

ssm_status ssm_ws_predict(const void *blob, size_t bytes, const float *feat, int64_t n, float *out) {
    if (!blob_ok(blob, bytes) || !feat || !out || n < 0) return SSM_EINVAL;
    if (n == 0) return SSM_OK;
    DevBuf db, df, dout;
    cudaError_t e = set_smem_limits();
    if (e == cudaSuccess) e = db.alloc(BLOB_BYTES);
    if (e == cudaSuccess) e = df.alloc(sizeof(float) * NI * n);
    if (e == cudaSuccess) e = dout.alloc(sizeof(float) * NO * n);
    if (e == cudaSuccess) e = cudaMemcpy(db.p, blob, BLOB_BYTES, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(df.p, feat, sizeof(float) * NI * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int64_t blocks = (n + 127) / 128 < 1216 ? (n + 127) / 128 : 1216;
        k_ws_predict<<<(unsigned)blocks, 128, NET_SMEM>>>(db.as<float>(), df.as<float>(), n, dout.as<float>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout.p, sizeof(float) * NO * n, cudaMemcpyDeviceToHost);
    return cst(e);
}

// One forward + backward over n rows with the blob's weights: the gradient of the
// mean squared error of the standardised outputs w.r.t. the parameters, in the
// order W1 [64x16], b1, W2 [64x64], b2, W3 [64x64], b3, W4 [3x64], b4.
ssm_status ssm_ws_grad(const void *blob, size_t bytes, const float *feat, const float *label, int64_t n,
                       float *grad, double *loss) {
    if (!blob_ok(blob, bytes) || !feat || !label || !grad || n < 1 || n > (1 << 20)) return SSM_EINVAL;
    DevBuf db, df, dl, fz, z, a, d, g, gp, ls;
    const int B = (int)n;
    cudaError_t e = set_smem_limits();
    if (e == cudaSuccess) e = db.alloc(BLOB_BYTES);
    if (e == cudaSuccess) e = df.alloc(sizeof(float) * NI * n);
    if (e == cudaSuccess) e = dl.alloc(sizeof(float) * NO * n);
    if (e == cudaSuccess) e = fz.alloc(sizeof(float) * NI * n);
    if (e == cudaSuccess) e = z.alloc(sizeof(float) * 3 * NH * n);
    if (e == cudaSuccess) e = a.alloc(sizeof(float) * 3 * NH * n);
    if (e == cudaSuccess) e = d.alloc(sizeof(float) * (3 * NH + NO) * n);
    if (e == cudaSuccess) e = g.alloc(sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = gp.alloc(sizeof(float) * NPARAM * WG_CHUNKS);
    if (e == cudaSuccess) e = ls.alloc(sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(db.p, blob, BLOB_BYTES, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(df.p, feat, sizeof(float) * NI * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dl.p, label, sizeof(float) * NO * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ls.p, 0, sizeof(double));
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        k_train_fwd<<<blocks, 128, NET_SMEM>>>(db.as<float>(), df.as<float>(), dl.as<float>(), nullptr, 0, B,
                                               fz.as<float>(), z.as<float>(), a.as<float>(), d.as<float>(), ls.as<double>());
        k_train_bwd<<<blocks, 128, NET_SMEM>>>(db.as<float>(), B, z.as<float>(), d.as<float>());
        launch_wgrad(B, fz.as<float>(), a.as<float>(), d.as<float>(), gp.as<float>(), g.as<float>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(grad, g.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpy(&l, ls.p, sizeof(double), cudaMemcpyDeviceToHost);
    if (loss) *loss = l / (double)(n * NO);
    return cst(e);
}

// Train the network on n rows (features [n][16], labels [n][3], host arrays):
// minibatch Adam, `epochs` passes over a fresh random order each, learning rate
// lr decayed by a cosine to lr/20, initial weights N(0, 1/fan_in) from `seed`.
// Writes the blob (ssm_ws_blob_bytes() bytes) and, if loss_curve != NULL, the
// mean training loss of each epoch.  Synchronous; allocates its own device buffers.
ssm_status ssm_ws_train(const float *feat, const float *label, int64_t n, int epochs, int batch, float lr,
                        uint64_t seed, void *blob_out, size_t bytes, double *loss_curve) {
    if (!feat || !label || !blob_out || bytes < BLOB_BYTES || n < 2 || epochs < 1 || batch < 1 ||
        batch > (1 << 16) || n > ((int64_t)1 << 28) || !(lr > 0.f))
        return SSM_EINVAL;
    // feature / label statistics (host, double)
    float fm[NI], fs[NI], ym[NO], ys[NO];
    for (int k = 0; k < NI; ++k) {
        double s = 0, s2 = 0;
        for (int64_t r = 0; r < n; ++r) { const double v = feat[r * NI + k]; s += v; s2 += v * v; }
        const double m = s / n, var = s2 / n - m * m;
        fm[k] = (float)m;
        fs[k] = (float)(var > 1e-20 ? sqrt(var) : 1.0);
    }
    for (int k = 0; k < NO; ++k) {
        double s = 0, s2 = 0;
        for (int64_t r = 0; r < n; ++r) { const double v = label[r * NO + k]; s += v; s2 += v * v; }
        const double m = s / n, var = s2 / n - m * m;
        ym[k] = (float)m;
        ys[k] = (float)(var > 1e-20 ? sqrt(var) : 1.0);
    }
    // initial weights
    uint64_t rs = seed ^ 0x5353574E45540001ull;
    std::vector<float> w(NPARAM, 0.f);
    auto gauss = [&]() { const double u1 = unit(rs), u2 = unit(rs); return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2); };
    for (int k = 0; k < NW1; ++k) w[P_W1 + k] = (float)(gauss() / sqrt((double)NI));
    for (int k = 0; k < NW2; ++k) w[P_W2 + k] = (float)(gauss() / sqrt((double)NH));
    for (int k = 0; k < NW3; ++k) w[P_W3 + k] = (float)(gauss() / sqrt((double)NH));
    for (int k = 0; k < NO * NH; ++k) w[P_W4 + k] = (float)(gauss() / sqrt((double)NH));
    std::vector<uint32_t> blob;
    pack_blob(w, fm, fs, ym, ys, blob);

    const int B = batch;
    DevBuf db, df, dl, dperm, fz, z, a, d, g, gp, m, v, dw, ls;
    cudaError_t e = set_smem_limits();
    if (e == cudaSuccess) e = db.alloc(BLOB_BYTES);
    if (e == cudaSuccess) e = df.alloc(sizeof(float) * NI * n);
    if (e == cudaSuccess) e = dl.alloc(sizeof(float) * NO * n);
    if (e == cudaSuccess) e = dperm.alloc(sizeof(int) * n);
    if (e == cudaSuccess) e = fz.alloc(sizeof(float) * NI * B);
    if (e == cudaSuccess) e = z.alloc(sizeof(float) * 3 * NH * B);
    if (e == cudaSuccess) e = a.alloc(sizeof(float) * 3 * NH * B);
    if (e == cudaSuccess) e = d.alloc(sizeof(float) * (3 * NH + NO) * B);
    if (e == cudaSuccess) e = g.alloc(sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = gp.alloc(sizeof(float) * NPARAM * WG_CHUNKS);
    if (e == cudaSuccess) e = m.alloc(sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = v.alloc(sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = dw.alloc(sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = ls.alloc(sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(db.p, blob.data(), BLOB_BYTES, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(df.p, feat, sizeof(float) * NI * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dl.p, label, sizeof(float) * NO * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dw.p, w.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m.p, 0, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMemset(v.p, 0, sizeof(float) * NPARAM);
    std::vector<int> perm((size_t)n);
    const int64_t nb = n / B > 0 ? n / B : 1;
    const int Bl = n < B ? (int)n : B;
    int64_t step = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t r = 0; r < n; ++r) perm[r] = (int)r;
        for (int64_t r = n - 1; r > 0; --r) {   // Fisher-Yates
            const int64_t j = (int64_t)(splitmix(rs) % (uint64_t)(r + 1));
            const int t = perm[r]; perm[r] = perm[j]; perm[j] = t;
        }
        e = cudaMemcpy(dperm.p, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(ls.p, 0, sizeof(double));
        for (int64_t bi = 0; bi < nb && e == cudaSuccess; ++bi, ++step) {
            const double prog = (double)(ep * nb + bi) / (double)(epochs * nb);
            const float lr_t = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + cos(3.141592653589793 * prog))));
            const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)(step + 1))));
            const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)(step + 1))));
            const unsigned blocks = (unsigned)((Bl + 127) / 128);
            k_train_fwd<<<blocks, 128, NET_SMEM>>>(db.as<float>(), df.as<float>(), dl.as<float>(), dperm.as<int>(),
                                                   bi * Bl, Bl, fz.as<float>(), z.as<float>(), a.as<float>(),
                                                   d.as<float>(), ls.as<double>());
            k_train_bwd<<<blocks, 128, NET_SMEM>>>(db.as<float>(), Bl, z.as<float>(), d.as<float>());
            launch_wgrad(Bl, fz.as<float>(), a.as<float>(), d.as<float>(), gp.as<float>(), g.as<float>());
            k_adam<<<(NPARAM + 127) / 128, 128>>>(g.as<float>(), m.as<float>(), v.as<float>(), dw.as<float>(),
                                                  db.as<float>(), lr_t, c1, c2);
            e = cudaGetLastError();
        }
        double l = 0.0;
        if (e == cudaSuccess) e = cudaMemcpy(&l, ls.p, sizeof(double), cudaMemcpyDeviceToHost);
        if (loss_curve) loss_curve[ep] = l / (double)(nb * Bl * NO);
    }
    if (e == cudaSuccess) e = cudaMemcpy(blob_out, db.p, BLOB_BYTES, cudaMemcpyDeviceToHost);
    return cst(e);
}

// Host helper for tests: the parameter vector (weights at their BF16 values) of a blob.
ssm_status ssm_ws_params(const void *blob, size_t bytes, float *params) {
    if (!blob_ok(blob, bytes) || !params) return SSM_EINVAL;
    std::vector<float> w;
    unpack_blob(blob, w);
    memcpy(params, w.data(), sizeof(float) * NPARAM);
    return SSM_OK;
}

int ssm_ws_num_params(void) { return NPARAM; }

}  // extern "C"
