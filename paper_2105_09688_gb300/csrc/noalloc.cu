// noalloc.cu -- ssm_drift_noalloc: the step-2 pair drift for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need this operation: code running inside a host callback or a
// real-time loop that must not block on the allocator, runtimes that hand out a
// fixed pre-reserved memory pool and forbid further device allocations, or
// embedders that budget every byte of device memory up front.  For them this
// entry point computes the same drift as ssm_get_stage(SSM_STAGE_B) from caller
// arrays, with its scratch (the per-chunk partial sums of the pair kernel) in
// the fixed, file-scope device array below instead of a context workspace.  It
// groups the pair sums in its own chunks, so it agrees with the context's drift
// to rounding, not bit for bit.
//
// Properties callers rely on:
//  - The scratch array is static device memory of SCRATCH_DOUBLES doubles
//    (8 MiB): every GPU that loads this library holds it until the process exits.
//  - The size is limited so that d * ld doubles fit: ld <= 349,525 for d = 3,
//    ld <= 1,048,576 for d = 1 (ld >= N is the array's leading dimension); larger
//    sizes return SSM_ENOMEM (scratch too small) without launching anything.
//  - The first call on a device looks up the device address of the scratch array
//    (cudaGetSymbolAddress, with that device current); make that first call
//    before any stream capture on that device.  The address is kept per device
//    together with the identity of the CUDA context it belongs to: after
//    cudaDeviceReset (a new primary context, the module loaded again) the next
//    call on that device looks it up again, so that call too must come before any
//    stream capture.
//  - No call allocates or frees device or host memory.
//  - Every call uses the same scratch array: calls whose work overlaps on the GPU
//    (different streams, or different host threads without ordering) race on it.
//    Calls on one stream are ordered and safe.  Every scratch element a call reads
//    was written earlier by the same call, so nothing needs clearing between calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ssm.h"
#include "ssm_device.cuh"

using namespace ssm;

namespace {

constexpr int64_t SCRATCH_DOUBLES = (int64_t)1 << 20;   // 8 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {};   // context identity the address belongs to

// The driver's context-identity query, fetched through the runtime (no link-time
// dependency on the driver library): cuCtxGetCurrent and cuCtxGetId, CUDA 12.0.
typedef int (*ctx_current_fn)(void **);
typedef int (*ctx_id_fn)(void *, unsigned long long *);
ctx_current_fn g_ctx_current = nullptr;
ctx_id_fn g_ctx_id = nullptr;
std::once_flag g_ctx_once;

// Identity of the current CUDA context (0 if the driver cannot tell).
unsigned long long current_context_id() {
    std::call_once(g_ctx_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = (ctx_current_fn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = (ctx_id_fn)f;
        cudaGetLastError();
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!g_ctx_current || !g_ctx_id || g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_scratch on the current device: looked up once per device
// and context (again after a device reset gave the device a new context).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// b[c*ld + i] = bscale * sum over chunks of the partials (chunk order fixed).
__global__ void k_combine_drift(const double *__restrict__ part, int chunks, int d, int64_t N, int64_t ld,
                                double bscale, double *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int q = 0; q < chunks; ++q) s += part[((int64_t)q * d + c) * ld + i];
            b[c * ld + i] = s * bscale;
        }
}

}  // namespace

extern "C" ssm_status ssm_drift_noalloc(int coef, int precision, int64_t N, const double *y, int64_t ld,
                                        double *b, void *stream) {
    if (!y || !b || N < 1 || ld < N) return SSM_EINVAL;
    if (coef != SSM_COEF_CUBIC1D_GAUSS && coef != SSM_COEF_COUPLED3D) return SSM_EINVAL;
    if (precision != SSM_FP64 && precision != SSM_FP32C) return SSM_EINVAL;
    const int d = coef == SSM_COEF_CUBIC1D_GAUSS ? 1 : 3;
    const int kind = d == 1 ? PK_DRIFT1 : PK_DRIFT3;
    const bool f32 = precision == SSM_FP32C;
    // one source chunk per pass as long as it fits; more chunks only if they fit too
    if ((int64_t)d * ld > SCRATCH_DOUBLES) return SSM_ENOMEM;
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return SSM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    Plan p;
    p.vec2 = 0;
    p.threads = 128;
    p.rpt = f32 ? (d == 1 ? 8 : 4) : 2;
    // Chunks: enough (tile, chunk) items to fill the device, bounded by the scratch.
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SSM_ECUDA;
    const int nb = pair_blocks_per_sm(kind, f32, 0, p.threads, p.rpt);
    const int64_t tiles = (N + p.threads * p.rpt - 1) / (p.threads * p.rpt);
    int64_t want = nb > 0 ? (4LL * sms * nb + tiles - 1) / tiles : 1;
    const int64_t fit = SCRATCH_DOUBLES / ((int64_t)d * ld);
    const int64_t maxc = (N + SUB - 1) / SUB;
    if (want > fit) want = fit;
    if (want > maxc) want = maxc;
    if (want < 1) want = 1;
    int64_t len = (N + want - 1) / want;
    len = (len + SUB - 1) / SUB * SUB;
    p.chunk_len = len;
    p.chunks = (int)((N + len - 1) / len);

    const double cexp = d == 1 ? 1.0 : 0.5, cb = d == 1 ? 0.5 : 1.0;
    const double scale = f32 ? sqrt(cexp * LOG2E) : 1.0;
    const double bscale = cb / ((double)N * scale);
    e = pair_sums(kind, f32, p, y, y, nullptr, nullptr, N, ld, scale, scratch, st);
    if (e != cudaSuccess) return SSM_ECUDA;
    const int64_t cap = (int64_t)sms * 8;   // grid-stride: at most 8 blocks an SM
    const int64_t blocks = (N + 255) / 256 < cap ? (N + 255) / 256 : cap;
    k_combine_drift<<<(unsigned)blocks, 256, 0, st>>>(scratch, p.chunks, d, N, ld, bscale, b);
    return cudaGetLastError() == cudaSuccess ? SSM_OK : SSM_ECUDA;
}
