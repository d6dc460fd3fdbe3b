// batch.cu -- many independent SSM ensembles (uneven N, different h, d = 1 and 3)
// advanced together by one CUDA graph whose device-side loops run every step of
// every ensemble: one cudaGraphLaunch for a whole batch run.
//
// Each ensemble is the coupled coefficient set (v = -y|y|^2 + 0.5 int (z - y)/(1 +
// |y - z|^2) mu(dz), b = int (z - y) exp(-|y - z|^2 / 2) mu(dz), sigma = 0.3 y + 0.2
// componentwise) at d = 1 or d = 3, stepped by the SSM of §2.3 (eq.
// SSTM:scheme 1 and 2) exactly as a single context steps it; only the scheduling
// differs.  Per batch step every unfinished ensemble advances one step:
//
//   kb_begin -> WHILE(any particle unconverged) { kb_pair<step 1> -> kb_update }
//            -> kb_pair<drift> -> kb_euler -> kb_finish      (inside WHILE(any ensemble unfinished))
//
// Every kernel is persistent-style: a grid sized to the device's resident slots
// walks a list of work items built, inside the kernel, from a prefix sum over the
// ensembles (pair items = (ensemble, target tile, source chunk); O(N) items =
// particles or 256-particle segments), so large and small ensembles share the
// GPU in every phase.  Loop conditions are set on the device
// (cudaGraphSetConditional) by the last block of kb_update / kb_finish, which is
// found with an atomic ticket; no kernel ever waits for another block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "pair_tile.cuh"
#include "particle_ops.cuh"
#include "ssm.h"
#include "ssm_device.cuh"

namespace ssm {
cudaError_t launch_init_x0_raw(int d, double *x, int64_t N, int64_t Np, uint64_t seed, double mean, double sd,
                               double *mpart, unsigned *ticket, double *mom, int *err, cudaStream_t st);
SSM_BOUNDS_READER(bounds_hits_batch)
}

using namespace ssm;

namespace {

constexpr int MAX_ENS = 1024;
constexpr int BT = 128;      // threads of the pair kernels
constexpr int SEGT = 256;    // threads (and particles per segment) of the O(N) kernels
constexpr int64_t NMAX_ENS = (int64_t)1 << 24;

struct BEns {                // one ensemble, in device memory
    int d, active, fine_r, chunks, fp32, carry;   // carry: ssm_opts.carry_start
    int64_t N, Np, M, chunk_len, seg0, nseg;
    long long n;
    uint64_t seed;
    double h, sqrt_h, sqrt_hf, scale, bscale, tol;
    double *x, *y, *part, *mom;
    double *sconv;            // converged step-1 pair sums of the last step (carry only)
    int *act0, *act1, *cnt;
    float *rprev;
};

struct BGlobal {             // batch-wide device state
    int pass, any_active, err, pad;
    long long bstep, stop_at;
    unsigned ticket_upd, ticket_fin;
    long long counters[CNT_N];
};

struct BShape { int r1, r3, packed; };   // targets per thread (d = 1, d = 3); d = 3 form: 0 scalar,
                                         // 1 packed difference form, 2 packed centred expansion

// ---- block-wide prefix sum over ensembles (every block computes the same) ----
template <typename F>
__device__ __forceinline__ void block_prefix(long long *pref, int n_ens, F count) {
    __shared__ long long carry;
    if (threadIdx.x == 0) { pref[0] = 0; carry = 0; }
    __syncthreads();
    for (int base = 0; base < n_ens; base += blockDim.x) {
        const int e = base + threadIdx.x;
        long long v = e < n_ens ? count(e) : 0;
        // inclusive scan within the block (Hillis-Steele in shared memory)
        __shared__ long long tmp[SEGT];
        tmp[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            const long long a = threadIdx.x >= off ? tmp[threadIdx.x - off] : 0;
            __syncthreads();
            tmp[threadIdx.x] += a;
            __syncthreads();
        }
        if (e < n_ens) pref[e + 1] = carry + tmp[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) carry += tmp[blockDim.x - 1];
        __syncthreads();
    }
}

// Ensemble e with pref[e] <= it < pref[e + 1] (pref non-decreasing, it < pref[n]).
__device__ __forceinline__ int find_ens(const long long *pref, int n_ens, long long it) {
    int lo = 0, hi = n_ens - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pref[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool last_block_of(unsigned *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) *ticket = 0u;
    return last;
}

// ---- phase kernels ----------------------------------------------------------

// Start of step 1 (every target active) for every unfinished ensemble: Y = X, or with
// ssm_opts.carry_start from its second step on the carried start of the single
// contexts (the root of u = X + h(-u|u|^2 + S*/2) with the particle's converged pair
// sum S* of the previous step).
__device__ __forceinline__ void plain_start(BEns *ens, int n_ens, BGlobal *g, int kmax) {
    __shared__ long long pref[MAX_ENS + 1];
    block_prefix(pref, n_ens, [&](int e) -> long long { return ens[e].active ? ens[e].N : 0; });
    const long long total = pref[n_ens];
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int e = find_ens(pref, n_ens, idx);
        const BEns &E = ens[e];
        const int64_t i = idx - pref[e];
        for (int c = 0; c < E.d; ++c) E.y[c * E.Np + i] = E.x[c * E.Np + i];
        if (E.carry && E.n > 0) {
            if (E.d == 1) {
                const double X[1] = {E.x[i]};
                const float Sc[1] = {f64_to_f32_fast(E.sconv[i])};
                cubic_start<1>(X, Sc, E.h, E.y + i, E.Np);
            } else {
                double X[3];
                float Sc[3];
                for (int c = 0; c < 3; ++c) {
                    X[c] = E.x[c * E.Np + i];
                    Sc[c] = f64_to_f32_fast(E.sconv[c * E.Np + i]);
                }
                cubic_start<3>(X, Sc, E.h, E.y + i, E.Np);
            }
        }
        E.act0[i] = (int)i;
        if (i == 0) {
            E.cnt[0] = (int)E.N;
            for (int k = 1; k <= kmax; ++k) E.cnt[k] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) g->pass = 0;
}

// Graph node: plain start, then open the pass loop.
__global__ void __launch_bounds__(SEGT)
kb_begin(BEns *ens, int n_ens, BGlobal *g, int kmax, cudaGraphConditionalHandle hpass) {
    plain_start(ens, n_ens, g, kmax);
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hpass, 1u);
}

// The same start outside any graph (launch-shape tuning).
__global__ void __launch_bounds__(SEGT) kb_plain_start(BEns *ens, int n_ens, BGlobal *g, int kmax) {
    plain_start(ens, n_ens, g, kmax);
}

// Pair sums of all ensembles: step-1 sums (NEWTON) at the active targets of the
// current pass, or the drift sums at all particles.
template <bool NEWTON, typename T, int R1, int R3, int PK3>
__global__ void __launch_bounds__(BT)
kb_pair(BEns *ens, int n_ens, const BGlobal *g) {
    __shared__ long long pref[MAX_ENS + 1];
    const int pass = NEWTON ? g->pass : 0;
    block_prefix(pref, n_ens, [&](int e) -> long long {
        const BEns &E = ens[e];
        if (!E.active) return 0;
        const int64_t ntgt = NEWTON ? (int64_t)E.cnt[pass] : E.N;
        const int64_t tile = (int64_t)BT * (E.d == 1 ? R1 : R3);
        return ((ntgt + tile - 1) / tile) * E.chunks;
    });
    const long long total = pref[n_ens];
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        const int e = find_ens(pref, n_ens, it);
        const BEns &E = ens[e];
        const long long local = it - pref[e];
        const int chunk = (int)(local % E.chunks);
        const long long tile = local / E.chunks;
        const int64_t j0 = (int64_t)chunk * E.chunk_len;
        const int64_t j1 = j0 + E.chunk_len < E.N ? j0 + E.chunk_len : E.N;
        const int nc = NEWTON ? E.d + 1 : E.d;
        double *part = E.part + (int64_t)chunk * nc * E.Np;
        const int *act = NEWTON ? ((pass & 1) ? E.act1 : E.act0) : nullptr;
        int64_t ntgt = NEWTON ? (int64_t)E.cnt[pass] : E.N;
        if (!SSM_IN_BOUNDS(ntgt >= 0 && ntgt <= E.Np)) ntgt = 0;
        const double *src = NEWTON ? E.x : E.y;
        const double sc = NEWTON ? 1.0 : E.scale;
        if (E.d == 1) {
            tile_scalar<NEWTON ? PK_NEWTON1 : PK_DRIFT1, T, BT, R1>(src, E.y, act, ntgt, E.Np, j0, j1,
                                                                     tile * BT * R1, sc, part, E.Np);
        } else if (PK3) {
            tile_packed<NEWTON ? PK_NEWTON3 : PK_DRIFT3, BT, R3, PK3 == 2>(src, E.y, act, ntgt, E.Np, j0, j1,
                                                                           tile * BT * R3, sc, part, E.Np);
        } else {
            tile_scalar<NEWTON ? PK_NEWTON3 : PK_DRIFT3, T, BT, R3>(src, E.y, act, ntgt, E.Np, j0, j1,
                                                                     tile * BT * R3, sc, part, E.Np);
        }
    }
}

template <int D>
__device__ __forceinline__ int update_one(const BEns &E, int pass, int64_t t, int i, bool fp32, int kmax) {
    constexpr int NC = D + 1;
    double S[D], Sw = 0.0, Y[D], X[D];
#pragma unroll
    for (int c = 0; c < D; ++c) S[c] = 0.0;
    for (int k = 0; k < E.chunks; ++k) {
        const double *pk = E.part + (int64_t)k * NC * E.Np + t;
#pragma unroll
        for (int c = 0; c < D; ++c) S[c] += pk[c * E.Np];
        Sw += pk[D * E.Np];
    }
    const double invN = 1.0 / (double)E.N;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        S[c] *= invN;
        Y[c] = E.y[c * E.Np + i];
        X[c] = E.x[c * E.Np + i];
    }
    Sw *= invN;
    const int r = newton_update_particle<D>(S, Sw, Y, X, E.h, E.tol, fp32, pass, kmax, -1, &E.rprev[i]);
    if (r == UPD_CONTINUE || r == UPD_CONVERGED || r == UPD_FLOOR)
#pragma unroll
        for (int c = 0; c < D; ++c) E.y[c * E.Np + i] = Y[c];
    if (E.carry && (r == UPD_CONVERGED || r == UPD_FLOOR))
#pragma unroll
        for (int c = 0; c < D; ++c) E.sconv[c * E.Np + i] = S[c];
    return r;
}

// Step-1 updates of every active target; the last block advances the pass and
// decides whether the pass loop runs again.
__global__ void __launch_bounds__(SEGT)
kb_update(BEns *ens, int n_ens, BGlobal *g, int kmax, int fp32, cudaGraphConditionalHandle hpass) {
    __shared__ long long pref[MAX_ENS + 1];
    const int pass = g->pass;
    block_prefix(pref, n_ens, [&](int e) -> long long { return ens[e].active ? ens[e].cnt[pass] : 0; });
    const long long total = pref[n_ens];
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += (long long)gridDim.x * blockDim.x) {
        const long long idx = base + threadIdx.x;
        bool keep = false;
        int e = 0, i = 0;
        if (idx < total && SSM_IN_BOUNDS(find_ens(pref, n_ens, idx) < n_ens)) {
            e = find_ens(pref, n_ens, idx);
            const BEns &E = ens[e];
            const int64_t t = idx - pref[e];
            i = ((pass & 1) ? E.act1 : E.act0)[t];
            if (SSM_IN_BOUNDS(i >= 0 && i < E.N)) {
                const int r = E.d == 1 ? update_one<1>(E, pass, t, i, fp32 != 0, kmax)
                                       : update_one<3>(E, pass, t, i, fp32 != 0, kmax);
                if (r == UPD_CONTINUE) keep = true;
                else if (r == UPD_FLOOR) atomicAdd((unsigned long long *)&g->counters[CNT_FLOOR], 1ull);
                else if (r == UPD_NOCONV) atomicOr(&g->err, ERR_NOCONV);
                else if (r == UPD_NONFINITE) atomicOr(&g->err, ERR_NONFINITE);
            }
        }
        // append survivors to their ensemble's next list; lanes of one ensemble
        // share one atomic
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const unsigned grp = __match_any_sync(km, e);
            const int leader = __ffs(grp) - 1;
            const BEns &E = ens[e];
            int slot = 0;
            if (lane == leader) slot = atomicAdd(&E.cnt[pass + 1], __popc(grp));
            slot = __shfl_sync(grp, slot, leader);
            ((pass & 1) ? E.act0 : E.act1)[slot + __popc(grp & ((1u << lane) - 1u))] = i;
        }
    }
    if (last_block_of(&g->ticket_upd) && threadIdx.x == 0) {
        long long next = 0;
        for (int e = 0; e < n_ens; ++e)
            if (ens[e].active) next += __ldcg(&ens[e].cnt[pass + 1]);
        g->counters[CNT_NEWTON_ROWS] += total;
        if (total > 0) g->counters[CNT_NEWTON_PASSES] += 1;
        g->pass = pass + 1;
        cudaGraphSetConditional(hpass, (next > 0 && pass + 1 < kmax) ? 1u : 0u);
    }
}

// Step 2 per 256-particle segment, with that segment's moment partial sums.
// Step 2 of one particle; the FP32C form draws dW from the FP32 transform and forms
// the increment in FP32, exactly as the single-context kernel does.
template <int D>
__device__ __forceinline__ void euler_segment(const BEns &E, int64_t i, double (&m)[12]) {
    double yv[D], b[D], inc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        yv[c] = E.y[c * E.Np + i];
        double s = 0.0;
        for (int k = 0; k < E.chunks; ++k) s += E.part[((int64_t)k * D + c) * E.Np + i];
        b[c] = s * E.bscale;
    }
    if (E.fp32) {
        float dw[D];
        brownian32<D>(E.seed, i, E.n, (float)E.sqrt_h, E.fine_r, (float)E.sqrt_hf, dw);
#pragma unroll
        for (int c = 0; c < D; ++c)
            inc[c] = (double)fmaf(sigma_of32(SSM_COEF_COUPLED3D, (float)yv[c], 0.0f), dw[c], (float)E.h * (float)b[c]);
    } else {
        double dw[D];
        brownian<D>(E.seed, i, E.n, E.sqrt_h, E.fine_r, E.sqrt_hf, dw);
#pragma unroll
        for (int c = 0; c < D; ++c) inc[c] = E.h * b[c] + sigma_of(SSM_COEF_COUPLED3D, yv[c], 0.0) * dw[c];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double xn = yv[c] + inc[c];
        E.x[c * E.Np + i] = xn;
        const double x2 = xn * xn;
        m[0 * 3 + c] += xn;
        m[1 * 3 + c] += x2;
        m[2 * 3 + c] += x2 * xn;
        m[3 * 3 + c] += x2 * x2;
    }
}

__global__ void __launch_bounds__(SEGT)
kb_euler(BEns *ens, int n_ens, const long long *seg_pref, double *mseg, BGlobal *g) {
    __shared__ long long pref[MAX_ENS + 1];
    for (int e = threadIdx.x; e <= n_ens; e += blockDim.x) pref[e] = seg_pref[e];
    __syncthreads();
    const long long total = pref[n_ens];
    __shared__ double red[SEGT / 32][12];
    for (long long seg = blockIdx.x; seg < total; seg += gridDim.x) {
        const int e = find_ens(pref, n_ens, seg);
        const BEns &E = ens[e];
        if (!E.active) continue;   // block-uniform
        const int64_t i = (seg - pref[e]) * SEGT + threadIdx.x;
        double m[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) m[k] = 0.0;
        if (i < E.N) {
            if (E.d == 1) euler_segment<1>(E, i, m);
            else euler_segment<3>(E, i, m);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k)
            for (int off = 16; off > 0; off >>= 1) m[k] += __shfl_down_sync(0xffffffffu, m[k], off);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 12; ++k) red[threadIdx.x >> 5][k] = m[k];
        __syncthreads();
        if (threadIdx.x < 12) {
            double s = 0.0;
            for (int w = 0; w < SEGT / 32; ++w) s += red[w][threadIdx.x];
            if (!isfinite(s)) atomicOr(&g->err, ERR_NONFINITE);
            mseg[seg * 12 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// Per ensemble (block e): moments from the segment partials in segment order,
// advance the step; the last block decides whether the step loop runs again.
__global__ void kb_finish(BEns *ens, int n_ens, const long long *seg_pref, const double *mseg, BGlobal *g,
                          cudaGraphConditionalHandle hstep) {
    for (int e = blockIdx.x; e < n_ens; e += gridDim.x) {
        BEns &E = ens[e];
        if (!E.active) continue;
        if (threadIdx.x < 4 * E.d) {
            const int k = threadIdx.x / E.d, c = threadIdx.x % E.d;
            double s = 0.0;
            for (long long sg = seg_pref[e]; sg < seg_pref[e + 1]; ++sg) s += mseg[sg * 12 + k * 3 + c];
            E.mom[threadIdx.x] = s / (double)E.N;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd((unsigned long long *)&g->counters[CNT_STEPS], 1ull);
            atomicAdd((unsigned long long *)&g->counters[CNT_DRIFT_ROWS], (unsigned long long)E.N);
            E.n += 1;
            if (E.n >= E.M) E.active = 0;
        }
        __syncthreads();
    }
    if (last_block_of(&g->ticket_fin) && threadIdx.x == 0) {
        int any = 0;
        for (int e = 0; e < n_ens; ++e) any |= __ldcg(&ens[e].active);
        g->any_active = any;
        g->bstep += 1;
        cudaGraphSetConditional(hstep, (any && g->bstep < g->stop_at) ? 1u : 0u);
    }
}

__global__ void kb_set_stop(BGlobal *g, long long k) { g->stop_at = g->bstep + k; }

constexpr BShape SHAPES_F32[] = { {8, 4, 1}, {8, 8, 1}, {8, 4, 2}, {8, 8, 2}, {8, 4, 0}, {4, 4, 0} };
constexpr BShape SHAPE_F64 = {2, 2, 0};

template <bool NEWTON>
void *pair_kernel(bool f32, const BShape &s) {
    if (!f32) return (void *)kb_pair<NEWTON, double, 2, 2, 0>;
    if (s.packed == 1 && s.r3 == 4) return (void *)kb_pair<NEWTON, float, 8, 4, 1>;
    if (s.packed == 1 && s.r3 == 8) return (void *)kb_pair<NEWTON, float, 8, 8, 1>;
    if (s.packed == 2 && s.r3 == 4) return (void *)kb_pair<NEWTON, float, 8, 4, 2>;
    if (s.packed == 2 && s.r3 == 8) return (void *)kb_pair<NEWTON, float, 8, 8, 2>;
    if (s.r1 == 8) return (void *)kb_pair<NEWTON, float, 8, 4, 0>;
    return (void *)kb_pair<NEWTON, float, 4, 4, 0>;
}

}  // namespace

struct ssm_batch {
    int n;
    bool f32;
    double tol;
    int kmax;
    cudaStream_t st;
    bool own_stream;
    char *mem;
    BEns *d_ens;
    BGlobal *d_g;
    long long *d_seg_pref;
    double *d_mseg, *d_mpart;
    unsigned *d_ticket;
    int *d_err;
    std::vector<BEns> h_ens;
    std::vector<int64_t> M;
    BShape shape;
    int64_t chunk_len;
    int grid_pair[2], grid_small;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    bool graph_ready;
    int status;
};

namespace {

ssm_status cuda_st(cudaError_t e) {
    return e == cudaSuccess ? SSM_OK : (e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA);
}

// Chunking of each ensemble for a given chunk length (sources per chunk).
void set_chunks(ssm_batch *b, int64_t chunk_len) {
    b->chunk_len = chunk_len;
    for (auto &E : b->h_ens) {
        const int64_t len = chunk_len < E.N ? chunk_len : (E.N + SUB - 1) / SUB * SUB;
        E.chunk_len = len;
        E.chunks = (int)((E.N + len - 1) / len);
    }
}

cudaError_t kernel_node(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *dep, size_t ndep, void *func,
                        unsigned grid, unsigned block, void **args) {
    cudaKernelNodeParams p = {};
    p.func = func;
    p.gridDim = dim3(grid);
    p.blockDim = dim3(block);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    return cudaGraphAddKernelNode(node, g, dep, ndep, &p);
}

// The batch graph: WHILE(step) { begin; WHILE(pass) { pair<1>; update }; pair<0>; euler; finish }.
cudaError_t build_graph(ssm_batch *b) {
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->gexec);
        cudaGraphDestroy(b->graph);
        b->graph_ready = false;
    }
    cudaGraph_t g;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle hstep, hpass;
    e = cudaGraphConditionalHandleCreate(&hstep, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hstep;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t nstep;
    if (e == cudaSuccess) e = cudaGraphAddNode(&nstep, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return e; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaGraphConditionalHandleCreate(&hpass, body, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return e; }

    // kernel arguments (copied into the nodes at creation)
    BEns *ens = b->d_ens;
    int n = b->n;
    BGlobal *gl = b->d_g;
    int kmax = b->kmax;
    int fp32 = b->f32 ? 1 : 0;
    long long *segp = b->d_seg_pref;
    double *mseg = b->d_mseg;
    const BGlobal *glc = gl;

    cudaGraphNode_t nb, npass, nd, ne, nf;
    void *a_begin[] = { &ens, &n, &gl, &kmax, &hpass };
    e = kernel_node(body, &nb, nullptr, 0, (void *)kb_begin, b->grid_small, SEGT, a_begin);
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hpass;
    ip.conditional.type = cudaGraphCondTypeWhile;
    ip.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&npass, body, &nb, nullptr, 1, &ip);
    if (e == cudaSuccess) {
        cudaGraph_t pbody = ip.conditional.phGraph_out[0];
        cudaGraphNode_t np, nu;
        void *a_pair[] = { &ens, &n, &glc };
        e = kernel_node(pbody, &np, nullptr, 0, pair_kernel<true>(b->f32, b->shape), b->grid_pair[0], BT, a_pair);
        void *a_upd[] = { &ens, &n, &gl, &kmax, &fp32, &hpass };
        if (e == cudaSuccess) e = kernel_node(pbody, &nu, &np, 1, (void *)kb_update, b->grid_small, SEGT, a_upd);
    }
    void *a_drift[] = { &ens, &n, &glc };
    if (e == cudaSuccess) e = kernel_node(body, &nd, &npass, 1, pair_kernel<false>(b->f32, b->shape), b->grid_pair[1], BT, a_drift);
    void *a_eul[] = { &ens, &n, &segp, &mseg, &gl };
    if (e == cudaSuccess) e = kernel_node(body, &ne, &nd, 1, (void *)kb_euler, b->grid_small, SEGT, a_eul);
    const long long *segc = segp;
    const double *msegc = mseg;
    void *a_fin[] = { &ens, &n, &segc, &msegc, &gl, &hstep };
    unsigned fin_grid = (unsigned)(n < 1024 ? n : 1024);
    if (e == cudaSuccess) e = kernel_node(body, &nf, &ne, 1, (void *)kb_finish, fin_grid, 32, a_fin);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return e; }
    b->graph = g;
    b->graph_ready = true;
    return cudaSuccess;
}

int resident_grid(void *func, int threads) {
    int nb = 0;
    int sms = device_sms();
    if (sms <= 0) sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, 0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return sms * nb;
}

void set_grids(ssm_batch *b) {
    b->grid_pair[0] = resident_grid(pair_kernel<true>(b->f32, b->shape), BT);
    b->grid_pair[1] = resident_grid(pair_kernel<false>(b->f32, b->shape), BT);
    b->grid_small = resident_grid((void *)kb_update, SEGT);
}

// Refresh the host copy of the ensemble descriptors from the device (the step
// counters and active flags advance there) before editing and re-uploading it.
cudaError_t pull_ens(ssm_batch *b) {
    cudaError_t e = cudaMemcpyAsync(b->h_ens.data(), b->d_ens, sizeof(BEns) * b->n, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    return e;
}

ssm_status harvest_batch(ssm_batch *b) {
    if (b->status != SSM_OK) return (ssm_status)b->status;
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, &b->d_g->err, sizeof(int), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) { b->status = SSM_ECUDA; return SSM_ECUDA; }
    if (err & ERR_NONFINITE) b->status = SSM_ENONFINITE;
    else if (err & ERR_NOCONV) b->status = SSM_ENOCONV;
    else if (bounds_hits_all()) b->status = SSM_EBOUNDS;
    return (ssm_status)b->status;
}

}  // namespace

extern "C" {

ssm_status ssm_batch_create(int n, const ssm_ens_desc *desc, const ssm_opts *opts, ssm_batch **out) {
    if (!out || !desc || n < 1 || n > MAX_ENS) return SSM_EINVAL;
    *out = nullptr;
    ssm_opts o;
    if (opts) o = *opts; else ssm_opts_default(&o);
    if (o.precision != SSM_FP64 && o.precision != SSM_FP32C) return SSM_EINVAL;
    if (o.measure_y != 0) return SSM_EINVAL;   // the batched form steps the SSM (mu^X in step 1)
    if (o.carry_start != 0 && o.carry_start != 1) return SSM_EINVAL;
    if (o.newton_kmax <= 0) o.newton_kmax = 12;
    if (o.newton_kmax > 64) return SSM_EINVAL;
    for (int e = 0; e < n; ++e) {
        const ssm_ens_desc &D = desc[e];
        if ((D.d != 1 && D.d != 3) || D.N < 1 || D.N > NMAX_ENS || !(D.h > 0.0) || !(D.T > 0.0) || D.h > D.T)
            return SSM_EINVAL;
        if (D.h > 1.0 / (1.0 + 2.0 / 16.0)) return SSM_EINVAL;   // Theorem 2.3 with L_v = 1/16
        const double M = nearbyint(D.T / D.h);
        if (M < 1.0 || fabs(M * D.h - D.T) > 1e-12 * D.T) return SSM_EINVAL;
        if (D.fine_log2 < 0 || D.fine_log2 > 30) return SSM_EINVAL;
        if (D.fine_log2 > 0) {
            const double r = D.h / (D.T / (double)(1ll << D.fine_log2));
            if (r < 1.0 || fabs(nearbyint(r) - r) > 1e-9) return SSM_EINVAL;
        }
    }
    ssm_batch *b = new (std::nothrow) ssm_batch();
    if (!b) return SSM_ENOMEM;
    b->n = n;
    b->f32 = o.precision == SSM_FP32C;
    b->tol = o.newton_tol > 0.0 ? o.newton_tol : (b->f32 ? 1e-10 : 1e-13);
    b->kmax = o.newton_kmax;
    b->shape = b->f32 ? SHAPES_F32[0] : SHAPE_F64;
    b->h_ens.resize(n);
    b->M.resize(n);
    cudaError_t e = cudaSuccess;
    if (o.stream) { b->st = (cudaStream_t)o.stream; b->own_stream = false; }
    else { e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking); b->own_stream = true; }
    if (e != cudaSuccess) { delete b; return cuda_st(e); }

    // layout: per ensemble x, y [d][Np], part (sized for 4096-source chunks), mom,
    // act0, act1 [Np], cnt [kmax + 2]; then the tables
    const int64_t min_chunk = 4096;
    std::vector<int64_t> off(n);
    size_t o8 = 0;
    auto take = [&](size_t bytes) { size_t at = o8; o8 = (o8 + bytes + 255) & ~(size_t)255; return at; };
    struct Offs { size_t x, y, part, mom, a0, a1, cnt, rp, sc; };
    std::vector<Offs> of(n);
    long long nseg_total = 0;
    for (int k = 0; k < n; ++k) {
        const ssm_ens_desc &D = desc[k];
        const int64_t Np = (D.N + 127) / 128 * 128;
        const int64_t chunks_max = (D.N + min_chunk - 1) / min_chunk;
        of[k].x = take(sizeof(double) * D.d * Np);
        of[k].y = take(sizeof(double) * D.d * Np);
        of[k].part = take(sizeof(double) * chunks_max * (D.d + 1) * Np);
        of[k].mom = take(sizeof(double) * 12);
        of[k].a0 = take(sizeof(int) * Np);
        of[k].a1 = take(sizeof(int) * Np);
        of[k].rp = take(sizeof(float) * Np);
        of[k].cnt = take(sizeof(int) * (b->kmax + 2));
        of[k].sc = take(o.carry_start ? sizeof(double) * D.d * Np : 0);
        nseg_total += (D.N + SEGT - 1) / SEGT;
    }
    const size_t o_ens = take(sizeof(BEns) * n), o_g = take(sizeof(BGlobal)), o_seg = take(sizeof(long long) * (n + 1));
    const size_t o_mseg = take(sizeof(double) * 12 * (size_t)nseg_total), o_mpart = take(sizeof(double) * RED_MAX_BLOCKS * 12);
    const size_t o_tk = take(sizeof(unsigned)), o_err = take(sizeof(int));
    e = cudaMalloc((void **)&b->mem, o8);
    if (e != cudaSuccess) { if (b->own_stream) cudaStreamDestroy(b->st); delete b; return cuda_st(e); }
    e = cudaMemsetAsync(b->mem, 0, o8, b->st);
    std::vector<long long> segp(n + 1, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const ssm_ens_desc &D = desc[k];
        BEns &E = b->h_ens[k];
        E.d = D.d;
        E.fp32 = b->f32 ? 1 : 0;
        E.N = D.N;
        E.Np = (D.N + 127) / 128 * 128;
        E.M = (int64_t)nearbyint(D.T / D.h);
        E.n = 0;
        E.active = 1;
        E.seed = D.seed;
        E.h = D.h;
        E.tol = o.newton_tol > 0.0 ? o.newton_tol : default_tol(b->f32, D.h, D.N);
        E.sqrt_h = sqrt(D.h);
        E.fine_r = 1;
        E.sqrt_hf = 0.0;
        if (D.fine_log2 > 0) {
            const double hf = D.T / (double)(1ll << D.fine_log2);
            E.fine_r = (int)llround(D.h / hf);
            E.sqrt_hf = sqrt(hf);
        }
        // exp(-r^2 / 2) = 2^(-|scale r|^2) in FP32; in FP64 the d = 1 kernel
        // evaluates exp(-r^2) (scale 1/sqrt(2)) and the d = 3 kernel has the 1/2 built in
        E.scale = b->f32 ? sqrt(0.5 * LOG2E) : (D.d == 1 ? sqrt(0.5) : 1.0);
        E.bscale = 1.0 / ((double)D.N * E.scale);
        E.x = (double *)(b->mem + of[k].x);
        E.y = (double *)(b->mem + of[k].y);
        E.part = (double *)(b->mem + of[k].part);
        E.mom = (double *)(b->mem + of[k].mom);
        E.act0 = (int *)(b->mem + of[k].a0);
        E.act1 = (int *)(b->mem + of[k].a1);
        E.rprev = (float *)(b->mem + of[k].rp);
        E.cnt = (int *)(b->mem + of[k].cnt);
        E.carry = o.carry_start;
        E.sconv = o.carry_start ? (double *)(b->mem + of[k].sc) : nullptr;
        E.seg0 = segp[k];
        E.nseg = (D.N + SEGT - 1) / SEGT;
        segp[k + 1] = segp[k] + E.nseg;
        b->M[k] = E.M;
    }
    set_chunks(b, 8192);
    b->d_ens = (BEns *)(b->mem + o_ens);
    b->d_g = (BGlobal *)(b->mem + o_g);
    b->d_seg_pref = (long long *)(b->mem + o_seg);
    b->d_mseg = (double *)(b->mem + o_mseg);
    b->d_mpart = (double *)(b->mem + o_mpart);
    b->d_ticket = (unsigned *)(b->mem + o_tk);
    b->d_err = (int *)(b->mem + o_err);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ens, b->h_ens.data(), sizeof(BEns) * n, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_seg_pref, segp.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, b->st);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const BEns &E = b->h_ens[k];
        e = launch_init_x0_raw(E.d, E.x, E.N, E.Np, E.seed, o.x0_mean, o.x0_std, b->d_mpart, b->d_ticket, E.mom,
                               b->d_err, b->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e == cudaSuccess) { set_grids(b); e = build_graph(b); }
    if (e != cudaSuccess) { ssm_batch_destroy(b); return cuda_st(e); }
    *out = b;
    return SSM_OK;
}

ssm_status ssm_batch_run_steps(ssm_batch *b, int64_t k) {
    if (!b || k < 0) return SSM_EINVAL;
    if (b->status != SSM_OK) return (ssm_status)b->status;
    if (k == 0) return SSM_OK;
    kb_set_stop<<<1, 1, 0, b->st>>>(b->d_g, (long long)k);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphLaunch(b->gexec, b->st);
    if (e != cudaSuccess) { b->status = cuda_st(e); return (ssm_status)b->status; }
    return SSM_OK;
}

ssm_status ssm_batch_run(ssm_batch *b) {
    if (!b) return SSM_EINVAL;
    return ssm_batch_run_steps(b, (int64_t)1 << 40);
}

ssm_status ssm_batch_sync(ssm_batch *b) {
    if (!b) return SSM_EINVAL;
    return harvest_batch(b);
}

ssm_status ssm_batch_get_state(ssm_batch *b, int e, double *x, int64_t *n) {
    if (!b || e < 0 || e >= b->n) return SSM_EINVAL;
    ssm_status s = harvest_batch(b);
    if (s != SSM_OK) return s;
    BEns E;
    cudaError_t ce = cudaMemcpy(&E, b->d_ens + e, sizeof(BEns), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess && x) {
        std::vector<double> soa((size_t)E.d * E.Np);
        ce = cudaMemcpy(soa.data(), E.x, sizeof(double) * E.d * E.Np, cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < E.N && ce == cudaSuccess; ++i)
            for (int c = 0; c < E.d; ++c) x[i * E.d + c] = soa[(size_t)c * E.Np + i];
    }
    if (n) *n = E.n;
    return cuda_st(ce);
}

ssm_status ssm_batch_moments(ssm_batch *b, int e, double *out) {
    if (!b || !out || e < 0 || e >= b->n) return SSM_EINVAL;
    ssm_status s = harvest_batch(b);
    if (s != SSM_OK) return s;
    return cuda_st(cudaMemcpy(out, b->h_ens[e].mom, sizeof(double) * 4 * b->h_ens[e].d, cudaMemcpyDeviceToHost));
}

ssm_status ssm_batch_stats(ssm_batch *b, ssm_stats_t *out) {
    if (!b || !out) return SSM_EINVAL;
    BGlobal g;
    cudaError_t e = cudaMemcpyAsync(&g, b->d_g, sizeof g, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return cuda_st(e);
    memset(out, 0, sizeof *out);
    out->steps = g.counters[CNT_STEPS];
    out->newton_passes = g.counters[CNT_NEWTON_PASSES];
    out->newton_rows = g.counters[CNT_NEWTON_ROWS];
    out->drift_rows = g.counters[CNT_DRIFT_ROWS];
    out->max_passes = g.bstep;   // batch steps taken
    out->floor_accepts = g.counters[CNT_FLOOR];
    return harvest_batch(b);
}

// Time every compiled launch shape and chunk length on one batch step's pair
// phases (the state is restored afterwards) and keep the fastest.
ssm_status ssm_batch_autotune(ssm_batch *b, double *best_ms) {
    if (!b) return SSM_EINVAL;
    if (b->status != SSM_OK) return (ssm_status)b->status;
    // the pair kernels read cnt[pass] and the active lists: set up a plain start
    // of step 1 for every ensemble (Y = X, all targets active), which changes no state
    std::vector<BShape> cands;
    if (b->f32) for (const BShape &s : SHAPES_F32) cands.push_back(s);
    else cands.push_back(SHAPE_F64);
    const int64_t lens[3] = { 4096, 8192, 16384 };
    cudaError_t err = pull_ens(b);
    if (err != cudaSuccess) { b->status = cuda_st(err); return (ssm_status)b->status; }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SSM_ECUDA;
    float best = 1e30f;
    BShape best_s = b->shape;
    int64_t best_len = b->chunk_len;
    const int n = b->n;
    for (const int64_t len : lens) {
        set_chunks(b, len);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(b->d_ens, b->h_ens.data(), sizeof(BEns) * n, cudaMemcpyHostToDevice, b->st);
        if (err == cudaSuccess) {
            kb_plain_start<<<b->grid_small, SEGT, 0, b->st>>>(b->d_ens, n, b->d_g, b->kmax);
            err = cudaGetLastError();
        }
        for (const BShape &s : cands) {
            if (err != cudaSuccess) break;
            b->shape = s;
            set_grids(b);
            float ms = 0.f;
            void *fn = pair_kernel<true>(b->f32, s), *fd = pair_kernel<false>(b->f32, s);
            BEns *ens = b->d_ens;
            const BGlobal *gl = b->d_g;
            void *args[] = { &ens, (void *)&b->n, &gl };
            err = cudaLaunchKernel(fd, dim3(b->grid_pair[1]), dim3(BT), args, 0, b->st);   // warm
            if (err == cudaSuccess) err = cudaEventRecord(e0, b->st);
            if (err == cudaSuccess) err = cudaLaunchKernel(fn, dim3(b->grid_pair[0]), dim3(BT), args, 0, b->st);
            if (err == cudaSuccess) err = cudaLaunchKernel(fd, dim3(b->grid_pair[1]), dim3(BT), args, 0, b->st);
            if (err == cudaSuccess) err = cudaEventRecord(e1, b->st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < best) { best = ms; best_s = s; best_len = len; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->shape = best_s;
    set_chunks(b, best_len);
    if (err == cudaSuccess) err = cudaMemcpyAsync(b->d_ens, b->h_ens.data(), sizeof(BEns) * n, cudaMemcpyHostToDevice, b->st);
    if (err == cudaSuccess) { set_grids(b); err = build_graph(b); }
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->st);
    if (err != cudaSuccess) { b->status = cuda_st(err); return (ssm_status)b->status; }
    if (best_ms) *best_ms = best;
    return SSM_OK;
}

ssm_status ssm_batch_set_plan(ssm_batch *b, const int *in) {
    if (!b || !in) return SSM_EINVAL;
    if (b->status != SSM_OK) return (ssm_status)b->status;
    bool ok = false;
    BShape shape = SHAPE_F64;
    if (b->f32) {
        for (const BShape &s : SHAPES_F32)
            if (s.packed == in[0] && s.r1 == in[1] && s.r3 == in[2]) { ok = true; shape = s; }
    } else {
        ok = SHAPE_F64.packed == in[0] && SHAPE_F64.r1 == in[1] && SHAPE_F64.r3 == in[2];
    }
    if (!ok || (in[3] != 4096 && in[3] != 8192 && in[3] != 16384)) return SSM_EINVAL;
    cudaError_t err = pull_ens(b);
    if (err == cudaSuccess) {
        b->shape = shape;
        set_chunks(b, in[3]);
        err = cudaMemcpyAsync(b->d_ens, b->h_ens.data(), sizeof(BEns) * b->n, cudaMemcpyHostToDevice, b->st);
    }
    if (err == cudaSuccess) { set_grids(b); err = build_graph(b); }
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->st);
    if (err != cudaSuccess) { b->status = cuda_st(err); return (ssm_status)b->status; }
    return SSM_OK;
}

ssm_status ssm_batch_get_plan(ssm_batch *b, int *out) {
    if (!b || !out) return SSM_EINVAL;
    out[0] = b->shape.packed;
    out[1] = BT;
    out[2] = b->shape.r1;
    out[3] = b->shape.r3;
    out[4] = (int)b->chunk_len;
    return SSM_OK;
}

void ssm_batch_destroy(ssm_batch *b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->graph_ready) {
        cudaGraphExecDestroy(b->gexec);
        cudaGraphDestroy(b->graph);
    }
    if (b->mem) cudaFree(b->mem);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"
