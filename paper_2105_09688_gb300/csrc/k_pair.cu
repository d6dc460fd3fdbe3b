// k_pair.cu -- single-context launchers of the O(N^2) pair sums (device code in
// pair_tile.cuh).  Grid = (target tiles) x (source chunks); chunk q of the
// partial sums is written to part[(q * NC + comp) * ps + t] (ps: the target count
// rounded up to 128 for a list of active targets, else Np) and the consuming
// O(N) kernel adds the chunks in a fixed order in double, so results are
// deterministic for a given launch shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pair_tile.cuh"

namespace ssm {

// The work of this block: its targets [t0, t0 + tile) of the ntgt targets, its
// sources [j0, j1), the offset of its target list in act (the ping-pong list of the
// pass) and of its partial sums in part (its chunk; the stride is ntgt rounded up to
// 128 for a list of active targets, else the caller's leading dimension Np).  For a pass over a list of active targets (act/cnt, or the pass index in
// dpass) with a pass plan (pplan, written by the update kernel of the previous pass,
// dyn_chunks) the launch's blocks are reassigned chunk-major over the tiles that hold
// targets, so the consecutive blocks of a chunk share sources; otherwise the planned
// shape: tile = blockIdx.x, chunk = blockIdx.y.  The kernels apply the offsets to
// their own parameters, so the tile code keeps the no-alias guarantees.
struct BlockWork {
    int64_t ntgt, t0, j0, j1, act_off, part_off, ps;
};
// False when the block has no work (block-uniform).
template <int TILE, int NC>
__device__ __forceinline__ bool block_work(const int *act, const int *cnt, const int *dpass, int64_t act_stride,
                                           int64_t N, int64_t Np, int64_t chunk_len, const DynChunks *pplan,
                                           BlockWork &w) {
    w.act_off = 0;
    if (dpass) { const int pass = *dpass; w.act_off = (pass & 1) * act_stride; cnt += pass; }
    int64_t ntgt = act ? (int64_t)(*cnt) : N;
    if (!SSM_IN_BOUNDS(ntgt >= 0 && ntgt <= Np)) ntgt = 0;
    int tile = blockIdx.x, chunk = blockIdx.y;
    int64_t len = chunk_len;
    if (act && pplan) {
        const DynChunks dc = *pplan;
        len = dc.len;
        if (dc.tiles != (int)gridDim.x) {
            const int b = blockIdx.y * gridDim.x + blockIdx.x;
            if (b >= dc.tiles * dc.chunks) return false;
            chunk = b / dc.tiles;
            tile = b - chunk * dc.tiles;
        }
    }
    w.ntgt = ntgt;
    w.t0 = (int64_t)tile * TILE;
    if (w.t0 >= ntgt) return false;
    w.j0 = (int64_t)chunk * len;
    w.j1 = (w.j0 + len < N) ? w.j0 + len : N;
    if (w.j0 >= w.j1) return false;
    w.ps = act ? partial_stride(ntgt) : Np;
    w.part_off = (int64_t)chunk * NC * w.ps;
    return true;
}

// act/cnt: optional compacted target list (targets t < *cnt are particles act[t]).
// dpass (optional): the pass index of step 1 in device memory, for launches inside a
// device-driven pass loop; then the list is act + (pass & 1) act_stride (the two
// ping-pong lists) and its length cnt[pass].
template <int KIND, typename T, int THREADS, int R>
__global__ void __launch_bounds__(THREADS)
k_pair(const double *__restrict__ src, const double *__restrict__ tgt, const int *__restrict__ act,
       const int *__restrict__ cnt, int64_t N, int64_t Np, int64_t chunk_len, double scale,
       double *__restrict__ part, const int *__restrict__ dpass, int64_t act_stride, const DynChunks *pplan) {
    BlockWork w;
    if (!block_work<THREADS * R, KindInfo<KIND>::NC>(act, cnt, dpass, act_stride, N, Np, chunk_len, pplan, w))
        return;   // block-uniform
    tile_scalar<KIND, T, THREADS, R>(src, tgt, act ? act + w.act_off : act, w.ntgt, Np, w.j0, w.j1, w.t0, scale,
                                     part + w.part_off, w.ps);
}

template <int KIND, int THREADS, int R>
__global__ void __launch_bounds__(THREADS)
k_pair2(const double *__restrict__ src, const double *__restrict__ tgt, const int *__restrict__ act,
        const int *__restrict__ cnt, int64_t N, int64_t Np, int64_t chunk_len, double scale,
        double *__restrict__ part, const int *__restrict__ dpass, int64_t act_stride, const DynChunks *pplan) {
    BlockWork w;
    if (!block_work<THREADS * R, KindInfo<KIND>::NC>(act, cnt, dpass, act_stride, N, Np, chunk_len, pplan, w))
        return;
    tile_packed<KIND, THREADS, R, false>(src, tgt, act ? act + w.act_off : act, w.ntgt, Np, w.j0, w.j1, w.t0, scale,
                                         part + w.part_off, w.ps);
}

// Centred expansion where a block's targets allow it (difference form otherwise).
template <int KIND, int THREADS, int R>
__global__ void __launch_bounds__(THREADS, packed_min_blocks(THREADS, R))
k_pair2x(const double *__restrict__ src, const double *__restrict__ tgt, const int *__restrict__ act,
         const int *__restrict__ cnt, int64_t N, int64_t Np, int64_t chunk_len, double scale,
         double *__restrict__ part, const int *__restrict__ dpass, int64_t act_stride, const DynChunks *pplan) {
    BlockWork w;
    if (!block_work<THREADS * R, KindInfo<KIND>::NC>(act, cnt, dpass, act_stride, N, Np, chunk_len, pplan, w))
        return;
    tile_packed<KIND, THREADS, R, true>(src, tgt, act ? act + w.act_off : act, w.ntgt, Np, w.j0, w.j1, w.t0, scale,
                                        part + w.part_off, w.ps);
}

template <int KIND, typename T, int THREADS, int R>
static cudaError_t launch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                          int64_t N, int64_t Np, double scale, double *part, cudaStream_t st, const int *dpass,
                          int64_t act_stride, const DynChunks *pplan) {
    const int64_t tiles = (N + THREADS * R - 1) / (THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)p.chunks);
    k_pair<KIND, T, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part, dpass,
                                                          act_stride, pplan);
    return cudaGetLastError();
}
template <int KIND, int THREADS, int R>
static cudaError_t launch2(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                           int64_t N, int64_t Np, double scale, double *part, cudaStream_t st, const int *dpass,
                           int64_t act_stride, const DynChunks *pplan) {
    const int64_t tiles = (N + THREADS * R - 1) / (THREADS * R);
    dim3 grid((unsigned)tiles, (unsigned)p.chunks);
    if (p.vec2 == 2)
        k_pair2x<KIND, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part,
                                                             dpass, act_stride, pplan);
    else
        k_pair2<KIND, THREADS, R><<<grid, THREADS, 0, st>>>(src, tgt, act, cnt, N, Np, p.chunk_len, scale, part,
                                                            dpass, act_stride, pplan);
    return cudaGetLastError();
}

// The (threads, targets per thread) shapes compiled for the scalar and the
// packed kernels.
#define SSM_PAIR_SHAPES(X) X(128, 2) X(128, 4) X(256, 2) X(256, 4) X(128, 8)
#define SSM_PAIR2_SHAPES(X) X(128, 4) X(128, 8) X(256, 4) X(256, 8)

template <int KIND, typename T>
static cudaError_t dispatch(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                            int64_t N, int64_t Np, double scale, double *part, cudaStream_t st, const int *dpass,
                            int64_t act_stride, const DynChunks *pplan) {
#define SSM_CASE(TH, RR) \
    if (p.threads == TH && p.rpt == RR) \
        return launch<KIND, T, TH, RR>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan);
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    return cudaErrorInvalidValue;
}
template <int KIND>
static cudaError_t dispatch2(const Plan &p, const double *src, const double *tgt, const int *act, const int *cnt,
                             int64_t N, int64_t Np, double scale, double *part, cudaStream_t st, const int *dpass,
                             int64_t act_stride, const DynChunks *pplan) {
#define SSM_CASE(TH, RR) \
    if (p.threads == TH && p.rpt == RR) \
        return launch2<KIND, TH, RR>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan);
    SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t pair_sums(int kind, bool fp32, const Plan &p, const double *src, const double *tgt, const int *act,
                      const int *cnt, int64_t N, int64_t Np, double scale, double *part, cudaStream_t st,
                      const int *dpass, int64_t act_stride, const DynChunks *pplan) {
    if (fp32 && p.vec2) {
        if (kind == PK_NEWTON3)
            return dispatch2<PK_NEWTON3>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan);
        if (kind == PK_DRIFT3)
            return dispatch2<PK_DRIFT3>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan);
        return cudaErrorInvalidValue;
    }
#define SSM_KIND(K) \
    case K: return fp32 ? dispatch<K, float>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan) \
                        : dispatch<K, double>(p, src, tgt, act, cnt, N, Np, scale, part, st, dpass, act_stride, pplan);
    switch (kind) {
        SSM_KIND(PK_DRIFT1)
        SSM_KIND(PK_DRIFT3)
        SSM_KIND(PK_NEWTON3)
        SSM_KIND(PK_NEWTON1)
    }
#undef SSM_KIND
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
template <int KIND, bool EXPAND>
static int occ_dispatch2(int threads, int rpt) {
    int nb = 0;
#define SSM_CASE(TH, RR) \
    if (threads == TH && rpt == RR) { \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, EXPAND ? (const void *)k_pair2x<KIND, TH, RR> \
                                                          : (const void *)k_pair2<KIND, TH, RR>, TH, 0) != cudaSuccess) \
            nb = 0; \
        return nb; }
    SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    return 0;
}

// Resident blocks per SM of a pair kernel shape (0 if unknown / no device).
int pair_blocks_per_sm(int kind, bool fp32, int vec2, int threads, int rpt) {
    if (fp32 && vec2) {
        if (kind == PK_NEWTON3)
            return vec2 == 2 ? occ_dispatch2<PK_NEWTON3, true>(threads, rpt) : occ_dispatch2<PK_NEWTON3, false>(threads, rpt);
        if (kind == PK_DRIFT3)
            return vec2 == 2 ? occ_dispatch2<PK_DRIFT3, true>(threads, rpt) : occ_dispatch2<PK_DRIFT3, false>(threads, rpt);
        return 0;
    }
#define SSM_KIND(K) case K: return fp32 ? occ_dispatch<K, float>(threads, rpt) : occ_dispatch<K, double>(threads, rpt);
    switch (kind) {
        SSM_KIND(PK_DRIFT1)
        SSM_KIND(PK_DRIFT3)
        SSM_KIND(PK_NEWTON3)
        SSM_KIND(PK_NEWTON1)
    }
#undef SSM_KIND
    return 0;
}

// Candidate launch shapes of a pair kind for the autotuner: {vec2, threads, rpt}
// (vec2: 0 scalar, 1 packed difference form, 2 packed centred expansion).
int pair_shape_candidates(int kind, bool fp32, int (*out)[3], int max_out) {
    int n = 0;
    auto add = [&](int v, int th, int r) { if (n < max_out) { out[n][0] = v; out[n][1] = th; out[n][2] = r; ++n; } };
#define SSM_CASE(TH, RR) add(0, TH, RR);
    SSM_PAIR_SHAPES(SSM_CASE)
#undef SSM_CASE
    if (fp32 && (kind == PK_NEWTON3 || kind == PK_DRIFT3)) {
#define SSM_CASE(TH, RR) add(1, TH, RR); add(2, TH, RR);
        SSM_PAIR2_SHAPES(SSM_CASE)
#undef SSM_CASE
    }
    return n;
}

SSM_BOUNDS_READER(bounds_hits_pair)

}  // namespace ssm
