// api.cu -- the C ABI declared in include/ssm.h: context life cycle, the launch
// sequence of one SSM step (§2.3, eq. SSTM:scheme 1 and SSTM:scheme 2), CUDA-graph
// replay of whole runs, state transfer and the component entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ssm.h"
#include "ssm_device.cuh"

namespace ssm {
cudaError_t launch_init_x0(ssm_ctx *c);
cudaError_t launch_moments(ssm_ctx *c);
cudaError_t launch_cardano(const double *x, double *y, int64_t n, double h, cudaStream_t st);
cudaError_t launch_mm_implicit(ssm_ctx *c);
cudaError_t launch_newton_begin(ssm_ctx *c);
cudaError_t launch_newton_update(ssm_ctx *c, int pass, int fp32, cudaGraphConditionalHandle hpass);
cudaError_t launch_step_stats(ssm_ctx *c);
cudaError_t launch_mi_begin(ssm_ctx *c);
cudaError_t launch_mi_pass(ssm_ctx *c, int pass, int fp32);
cudaError_t launch_euler(ssm_ctx *c, double bscale);
cudaError_t launch_set_step(ssm_ctx *c, long long n);
cudaError_t launch_aos_to_soa(const double *a, double *s, int d, int64_t N, int64_t Np, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *s, double *a, int d, int64_t N, int64_t Np, cudaStream_t st);
cudaError_t launch_stage_b(ssm_ctx *c, double bscale);
cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, int d, int64_t N, uint32_t step, uint32_t stream, double *out, cudaStream_t st);
cudaError_t launch_normals32(uint64_t seed, int d, int64_t N, uint32_t step, uint32_t stream, float *out,
                             cudaStream_t st);
cudaError_t ws_forward_start(ssm_ctx *c);
cudaError_t launch_carry_start(ssm_ctx *c);
}  // namespace ssm

namespace ssm {
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}
int bounds_hits_all() {
#ifdef SSM_CHECK_BOUNDS
    const int a = bounds_hits_pair(), b = bounds_hits_particle(), c = bounds_hits_batch();
    return a | b | c;
#else
    return 0;
#endif
}
}  // namespace ssm

using namespace ssm;

namespace {

constexpr int64_t N_MAX = (int64_t)1 << 26;

bool fp32_pairs(const ssm_ctx *c) { return c->prec != SSM_FP64; }

// Coordinate scale of the FP32 Gaussian kernels and the factor that turns the
// drift partial sums into b: b = coef * (1/N) * sum / scale.
void drift_scale(int coef, bool fp32, int64_t N, double *scale, double *bscale) {
    const double cexp = coef == SSM_COEF_CUBIC1D_GAUSS ? 1.0 : 0.5;   // exp(-cexp r^2)
    const double cb = coef == SSM_COEF_CUBIC1D_GAUSS ? 0.5 : 1.0;     // coefficient of the integral
    // FP32: exp(-c r^2) = 2^(-|s r|^2) with s = sqrt(c log2 e).  FP64: the d = 1
    // kernel evaluates exp(-r^2), so s = sqrt(c); the d = 3 kernel has c = 1/2 built in.
    const bool d1 = coef == SSM_COEF_CUBIC1D_GAUSS || coef == SSM_COEF_COUPLED1D;
    *scale = fp32 ? sqrt(cexp * LOG2E) : (d1 ? sqrt(cexp) : 1.0);
    *bscale = cb / ((double)N * *scale);
}

int64_t padded(int64_t N) { return (N + 127) / 128 * 128; }

// Most source chunks a pass may use: the partial-sum scratch holds
// chunks * NC * Np doubles, kept under 1 GiB and at most 32 chunks.
int chunks_cap(int64_t N, int nc) {
    int64_t cap = (N + SUB - 1) / SUB;
    if (cap > 32) cap = 32;
    const int64_t mem = ((int64_t)1 << 30) / ((int64_t)nc * padded(N) * 8);
    if (cap > mem) cap = mem;
    return cap < 1 ? 1 : (int)cap;
}

int kind_nc(int kind) {
    return kind == PK_NEWTON3 ? 4 : kind == PK_DRIFT3 ? 3 : kind == PK_NEWTON1 ? 2 : 1;
}
bool is_coupled(int coef) { return coef == SSM_COEF_COUPLED3D || coef == SSM_COEF_COUPLED1D; }
// Sets whose measure enters only through means: no pair sums, a per-particle step 1.
bool is_moment(int coef) {
    return coef == SSM_COEF_OU || coef == SSM_COEF_GL1 || coef == SSM_COEF_GL2 || coef == SSM_COEF_POLY ||
           coef == SSM_COEF_CS || coef == SSM_COEF_GLSTAB;
}
int newton_kind(int d) { return d == 1 ? PK_NEWTON1 : PK_NEWTON3; }
int drift_kind(int coef) { return (coef == SSM_COEF_CUBIC1D_GAUSS || coef == SSM_COEF_COUPLED1D) ? PK_DRIFT1 : PK_DRIFT3; }

// Resident-block slots of the device for a pair kernel shape (0 = no device).
int device_slots(int kind, bool fp32, int vec2, int threads, int rpt) {
    const int sms = device_sms();
    if (sms <= 0) return 0;
    const int nb = pair_blocks_per_sm(kind, fp32, vec2, threads, rpt);
    if (nb <= 0) { cudaGetLastError(); return 0; }
    return sms * nb;
}

// Launch shape of a pair kind: (threads x targets-per-thread) tiles over the
// targets times source chunks.  All work items cost the same, so the chunk count
// is chosen to make the number of items fill whole waves of the device's
// resident-block slots (smallest count reaching 97% wave efficiency with at least
// two waves, else the most efficient).
Plan make_plan_shape(int64_t N, int kind, int vec2, int threads, int rpt, int force_chunks, int slots) {
    Plan p;
    p.vec2 = vec2;
    p.threads = threads;
    p.rpt = rpt;
    const int64_t tiles = (N + p.threads * p.rpt - 1) / (p.threads * p.rpt);
    const int cap = chunks_cap(N, kind_nc(kind));
    int64_t chunks;
    if (force_chunks > 0) {
        chunks = force_chunks < cap ? force_chunks : cap;
    } else if (slots > 0) {
        int64_t best = 1;
        double best_eff = -1.0;
        for (int64_t c = 1; c <= cap; ++c) {
            const int64_t items = tiles * c;
            const int64_t waves = (items + slots - 1) / slots;
            const double eff = (double)items / (double)(waves * slots);
            if (eff >= 0.97 && items >= 2 * (int64_t)slots) { best = c; break; }
            if (eff > best_eff + 1e-9) { best_eff = eff; best = c; }
        }
        chunks = best;
    } else {
        chunks = (2432 + tiles - 1) / tiles;
        if (chunks > cap) chunks = cap;
    }
    if (chunks < 1) chunks = 1;
    // chunks are whole sub-tiles of the kernel (512 sources for the packed step-1 sums)
    const int64_t sub = (kind == PK_NEWTON3 && vec2) ? 512 : SUB;
    int64_t len = (N + chunks - 1) / chunks;
    len = (len + sub - 1) / sub * sub;
    p.chunk_len = len;
    p.chunks = (int)((N + len - 1) / len);
    return p;
}

// Default shape before any tuning: scalar kernels, 128 threads, 4 (FP32 d=3),
// 8 (FP32 d=1) or 2 (FP64) targets per thread; chunks from the device's slots.
Plan make_plan(int64_t N, bool fp32, int kind, int force_chunks) {
    const int th = 128, r = fp32 ? ((kind == PK_DRIFT1 || kind == PK_NEWTON1) ? 8 : 4) : 2;
    return make_plan_shape(N, kind, 0, th, r, force_chunks, device_slots(kind, fp32, 0, th, r));
}

struct Layout {
    size_t x, y, stage, part, mpart, mom, ymean, act0, act1, cnt, passes, err, ticket, dstep, counters, hist, wsw, sconv, mom_prev, rprev, mif, dpass, pplan, spred, wsprev, total;
    int64_t part_doubles;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// The partial-sum scratch is sized for the largest chunk count the planner may
// choose, so the layout is known without a device.
Layout make_layout(int d, int64_t N, int coef, int kmax) {
    Layout L;
    const int64_t Np = padded(N);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.x = take(sizeof(double) * d * Np);
    L.y = take(sizeof(double) * d * Np);
    L.stage = take(sizeof(double) * d * Np);
    size_t part = 0;
    if (is_coupled(coef)) {
        const int nn = d + 1, nd = d;   // step-1 and drift partial-sum components
        part = (size_t)chunks_cap(N, nn) * nn;
        if ((size_t)chunks_cap(N, nd) * nd > part) part = (size_t)chunks_cap(N, nd) * nd;
    } else if (coef == SSM_COEF_CUBIC1D_GAUSS) {
        part = (size_t)chunks_cap(N, 1);
    }
    L.part = take(sizeof(double) * part * Np);
    L.part_doubles = (int64_t)part * Np;
    L.mpart = take(sizeof(double) * RED_MAX_BLOCKS * 12);
    L.mom = take(sizeof(double) * 12);
    L.ymean = take(sizeof(double) * 4);
    const bool nt = is_coupled(coef);
    L.act0 = take(nt ? sizeof(int) * Np : 0);
    L.act1 = take(nt ? sizeof(int) * Np : 0);
    L.cnt = take(sizeof(int) * (kmax + 2));
    L.passes = take(nt ? sizeof(int) * Np : 0);
    L.err = take(sizeof(int));
    L.ticket = take(sizeof(unsigned));
    L.dstep = take(sizeof(long long));
    L.counters = take(sizeof(long long) * CNT_N);
    L.hist = take(sizeof(long long) * 16);
    L.wsw = take(nt ? 65536 * sizeof(float) : 0);
    L.sconv = take(nt ? sizeof(double) * 3 * Np : 0);
    L.mom_prev = take(sizeof(double) * 12);
    L.rprev = take(nt ? sizeof(float) * Np : 0);
    L.mif = take(nt ? sizeof(int) * MIF_WORDS(kmax) : 0);
    L.dpass = take(sizeof(int));
    L.pplan = take(sizeof(DynChunks));
    L.spred = take(nt ? sizeof(float) * 3 * Np : 0);
    L.wsprev = take(sizeof(int));
    L.total = o;
    return L;
}

void fill_defaults(ssm_opts *o) {
    memset(o, 0, sizeof *o);
    o->precision = SSM_FP64;
    o->newton_tol = 0.0;   // 0 = per-precision default
    o->newton_kmax = 12;
    o->fine_log2 = 0;
    o->x0_mean = 0.0;
    o->x0_std = 1.0;
    o->ws_passes = 4;
}

ssm_status check_args(int d, int64_t N, double h, double T, int coef, const ssm_opts &o) {
    if (N < 1 || N > N_MAX || !(h > 0.0) || !(T > 0.0) || !(h <= T)) return SSM_EINVAL;
    if (o.precision < SSM_FP64 || o.precision > SSM_FP32C_LEARNED) return SSM_EINVAL;
    if (o.newton_kmax < 1 || o.newton_kmax > 64) return SSM_EINVAL;
    double Lv;
    if (coef == SSM_COEF_CUBIC1D_GAUSS) {
        if (d != 1) return SSM_EINVAL;
        Lv = 1.0;
    } else if (coef == SSM_COEF_COUPLED3D || coef == SSM_COEF_COUPLED1D) {
        if (d != (coef == SSM_COEF_COUPLED3D ? 3 : 1)) return SSM_EINVAL;
        Lv = 1.0 / 16.0;
    } else if (coef == SSM_COEF_OU) {
        if (d < 1 || d > 3) return SSM_EINVAL;
        Lv = o.coef_params[0];
    } else if (coef == SSM_COEF_GL1 || coef == SSM_COEF_GL2) {
        if (d != 1) return SSM_EINVAL;
        Lv = 0.0;                       // -x^3 (+ a measure term constant in x): one-sided constant 0
    } else if (coef == SSM_COEF_POLY) {
        if (d != 1) return SSM_EINVAL;
        Lv = o.coef_params[0];          // gamma x - x mean(x^2): one-sided constant gamma - mean(x^2) <= gamma
    } else if (coef == SSM_COEF_CS) {
        if (d != 2) return SSM_EINVAL;
        Lv = 0.0;                       // (-V^3, 0)
    } else if (coef == SSM_COEF_GLSTAB) {
        // the stability study runs outside Theorem 2.3's step bound on purpose (§3.4.2,
        // h = 0.1 across gamma): only a unique step-1 root is required
        if (d != 1 || !(1.0 + h * (2.5 + o.coef_params[0]) > 0.0)) return SSM_EINVAL;
        Lv = -1.0;
    } else {
        return SSM_EINVAL;
    }
    if (o.precision == SSM_FP32C_LEARNED && coef != SSM_COEF_COUPLED3D) return SSM_EINVAL;
    if (o.measure_y != 0 && (o.measure_y != 1 || !is_coupled(coef) || o.precision == SSM_FP32C_LEARNED))
        return SSM_EINVAL;
    // Theorem 2.3: h <= 1/(1 + 2 L_v) when L_v > -1/2; also 1 - h L_v > 0 for Lemma 4.1.
    if (Lv > -0.5 && h > 1.0 / (1.0 + 2.0 * Lv)) return SSM_EINVAL;
    const double M = T / h;
    const double Mr = nearbyint(M);
    if (Mr < 1.0 || fabs(Mr * h - T) > 1e-12 * T) return SSM_EINVAL;
    if (o.fine_log2 < 0 || o.fine_log2 > 30) return SSM_EINVAL;
    if (o.fine_log2 > 0) {
        const double hf = T / (double)(1ll << o.fine_log2);
        const double r = h / hf;
        if (r < 1.0 || fabs(nearbyint(r) - r) > 1e-9) return SSM_EINVAL;
    }
    if (o.tile_chunks < 0 || o.fixed_pass_launches < 0 || o.fixed_pass_launches > 1 || o.ws_forward < 0 ||
        o.ws_forward > 1)
        return SSM_EINVAL;
    if (o.carry_start != 0 && (o.carry_start != 1 || !is_coupled(coef) || o.measure_y ||
                               o.precision == SSM_FP32C_LEARNED))
        return SSM_EINVAL;
    // ssm_opts.inject: only in the debug build, only the planted list entry of step 1
    // (coupled sets against mu^X) at an N whose padded arrays extend past particle N
#ifdef SSM_CHECK_BOUNDS
    if (o.inject != 0 && (o.inject != 1 || !is_coupled(coef) || o.measure_y || N % 128 == 0)) return SSM_EINVAL;
#else
    if (o.inject != 0) return SSM_EINVAL;
#endif
    return SSM_OK;
}

ssm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SSM_OK;
    if (e == cudaErrorMemoryAllocation) return SSM_ENOMEM;
    return SSM_ECUDA;
}

// Read the device error word and fold it into the sticky status.
ssm_status harvest(ssm_ctx *c) {
    if (c->status != SSM_OK) return (ssm_status)c->status;
    int e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) { c->status = SSM_ECUDA; return SSM_ECUDA; }
    if (e & ERR_NONFINITE) c->status = SSM_ENONFINITE;
    else if (e & ERR_NOCONV) c->status = SSM_ENOCONV;
    else if (e & ERR_TIMEOUT) c->status = SSM_ETIMEOUT;
    else if (bounds_hits_all()) c->status = SSM_EBOUNDS;
    return (ssm_status)c->status;
}

// The passes of step 1 (coupled sets, measure mu^X) as one conditional WHILE node of
// the graph being captured on c->st: its body -- the pair sums of the particles still
// active and their update -- repeats until the update kernel finds none left (or
// kmax passes were made), so only passes with work are launched.  The body is
// captured on the side stream c->st_body into the node's body graph.
cudaError_t enqueue_pass_loop(ssm_ctx *c, bool f32) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive || !c->st_body) return cudaErrorStreamCaptureUnsupported;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
    if (e != cudaSuccess) return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->st_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaStream_t main_st = c->st;
    c->st = c->st_body;
    cudaError_t eb = pair_sums(newton_kind(c->d), f32, c->plan_newton, c->x, c->y, c->act0, c->cnt, c->N, c->Np, 1.0,
                               c->part, c->st, c->dpass, (int64_t)(c->act1 - c->act0), c->pplan);
    if (eb == cudaSuccess) eb = launch_newton_update(c, 0, f32 ? 1 : 0, h);
    c->st = main_st;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c->st_body, &captured);
    if (eb != cudaSuccess) return eb;
    if (e != cudaSuccess) return e;
    return cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Enqueue one SSM step (no host synchronisation).  Captured into the context's step
// graph by ssm_run_steps (the coupled sets' pass loop is a graph node).
cudaError_t enqueue_step(ssm_ctx *c) {
    cudaError_t e = cudaSuccess;
    const bool f32 = fp32_pairs(c);
    double scale, bscale;
    drift_scale(c->coef, f32, c->N, &scale, &bscale);
    if (c->coef == SSM_COEF_CUBIC1D_GAUSS) {
        // step 1: closed-form root per particle
        if ((e = launch_cardano(c->x, c->y, c->N, c->h, c->st)) != cudaSuccess) return e;
        // step 2: b(Y_i, mu^Y) pair sums, then the fused update
        if ((e = pair_sums(PK_DRIFT1, f32, c->plan_drift, c->y, c->y, nullptr, nullptr, c->N, c->Np, scale, c->part,
                           c->st)) != cudaSuccess)
            return e;
        return launch_euler(c, bscale);
    }
    if (is_moment(c->coef)) {
        // OU and the polynomial drift take step 1 inside k_euler (fused_step1)
        if (!fused_step1(c->coef) && (e = launch_mm_implicit(c)) != cudaSuccess) return e;
        return launch_euler(c, 0.0);
    }
    // SSM_COEF_COUPLED3D / SSM_COEF_COUPLED1D
    if (c->opt.measure_y) {
        // step 1 against mu^Y: every pass evaluates all particles at the common iterate
        if ((e = launch_mi_begin(c)) != cudaSuccess) return e;
        for (int k = 0; k < c->kmax; ++k) {
            if ((e = pair_sums(newton_kind(c->d), f32, c->plan_newton, c->y, c->y, c->act0, c->cnt + k, c->N, c->Np,
                               1.0, c->part, c->st)) != cudaSuccess)
                return e;
            if ((e = launch_mi_pass(c, k, f32 ? 1 : 0)) != cudaSuccess) return e;
        }
    } else {
        if ((e = launch_newton_begin(c)) != cudaSuccess) return e;
        if (c->prec == SSM_FP32C_LEARNED && c->ws_loaded)
            if ((e = ws_forward_start(c)) != cudaSuccess) return e;
        if (c->opt.carry_start)
            if ((e = launch_carry_start(c)) != cudaSuccess) return e;
        if (c->opt.fixed_pass_launches) {
            for (int k = 0; k < c->kmax; ++k) {
                if ((e = pair_sums(newton_kind(c->d), f32, c->plan_newton, c->x, c->y, (k & 1) ? c->act1 : c->act0,
                                   c->cnt + k, c->N, c->Np, 1.0, c->part, c->st, nullptr, 0, c->pplan)) != cudaSuccess)
                    return e;
                if ((e = launch_newton_update(c, k, f32 ? 1 : 0, 0)) != cudaSuccess) return e;
            }
        } else if ((e = enqueue_pass_loop(c, f32)) != cudaSuccess) {
            return e;
        }
    }
    if ((e = launch_step_stats(c)) != cudaSuccess) return e;
    if ((e = pair_sums(drift_kind(c->coef), f32, c->plan_drift, c->y, c->y, nullptr, nullptr, c->N, c->Np, scale,
                       c->part, c->st)) != cudaSuccess)
        return e;
    return launch_euler(c, bscale);
}

}  // namespace

extern "C" {

void ssm_opts_default(ssm_opts *opts) {
    if (opts) fill_defaults(opts);
}

size_t ssm_workspace_bytes(int d, int64_t N, int coef, const ssm_opts *opts) {
    ssm_opts o;
    if (opts) o = *opts; else fill_defaults(&o);
    if (N < 1 || N > N_MAX || d < 1 || d > 3) return 0;
    return make_layout(d, N, coef, o.newton_kmax).total;
}

ssm_status ssm_create(int d, int64_t N, double h, double T, int coef, uint64_t seed, const ssm_opts *opts,
                      ssm_ctx **out) {
    if (!out) return SSM_EINVAL;
    *out = nullptr;
    ssm_opts o;
    if (opts) o = *opts; else fill_defaults(&o);
    if (o.newton_kmax == 0) o.newton_kmax = 12;
    if (o.ws_passes <= 0) o.ws_passes = 4;
    ssm_status s = check_args(d, N, h, T, coef, o);
    if (s != SSM_OK) return s;

    ssm_ctx *c = new (std::nothrow) ssm_ctx();
    if (!c) return SSM_ENOMEM;
    c->d = d; c->coef = coef; c->prec = o.precision; c->N = N; c->Np = padded(N);
    c->h = h; c->T = T; c->seed = seed; c->opt = o;
    c->M = (int64_t)nearbyint(T / h);
    c->n = 0;
    c->kmax = o.newton_kmax;
    c->tol = o.newton_tol > 0.0 ? o.newton_tol : default_tol(o.precision != SSM_FP64, h, N);
    const bool f32 = o.precision != SSM_FP64;
    c->plan_newton = make_plan(N, f32, newton_kind(d), o.tile_chunks);
    c->plan_drift = make_plan(N, f32, drift_kind(coef), o.tile_chunks);
    Layout L = make_layout(d, N, coef, c->kmax);

    cudaError_t e = cudaSuccess;
    if (o.stream) {
        c->st = (cudaStream_t)o.stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return cuda_status(e); }
        c->own_stream = true;
    }
    c->st_body = nullptr;
    if (is_coupled(coef) && !o.measure_y && !o.fixed_pass_launches) {
        e = cudaStreamCreateWithFlags(&c->st_body, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (c->own_stream) cudaStreamDestroy(c->st);
            delete c;
            return cuda_status(e);
        }
    }
    if (o.workspace) {
        if (o.workspace_bytes < L.total || ((uintptr_t)o.workspace & 255u)) {
            if (c->st_body) cudaStreamDestroy(c->st_body);
            if (c->own_stream) cudaStreamDestroy(c->st);
            delete c;
            return o.workspace_bytes < L.total ? SSM_ENOMEM : SSM_EINVAL;
        }
        c->ws = (char *)o.workspace;
        c->own_ws = false;
    } else {
        e = cudaMalloc((void **)&c->ws, L.total);
        if (e != cudaSuccess) {
            if (c->st_body) cudaStreamDestroy(c->st_body);
            if (c->own_stream) cudaStreamDestroy(c->st);
            delete c;
            return cuda_status(e);
        }
        c->own_ws = true;
    }
    c->ws_bytes = L.total;
    char *b = c->ws;
    c->x = (double *)(b + L.x); c->y = (double *)(b + L.y); c->stage = (double *)(b + L.stage);
    c->part = (double *)(b + L.part); c->mpart = (double *)(b + L.mpart); c->mom = (double *)(b + L.mom);
    c->ymean = (double *)(b + L.ymean);
    c->act0 = (int *)(b + L.act0); c->act1 = (int *)(b + L.act1); c->cnt = (int *)(b + L.cnt);
    c->passes = (int *)(b + L.passes); c->err = (int *)(b + L.err); c->ticket = (unsigned *)(b + L.ticket);
    c->dstep = (long long *)(b + L.dstep); c->counters = (long long *)(b + L.counters);
    c->hist = (long long *)(b + L.hist);
    c->ws_w = (float *)(b + L.wsw);
    c->sconv = (double *)(b + L.sconv);
    c->mom_prev = (double *)(b + L.mom_prev);
    c->rprev = (float *)(b + L.rprev);
    c->mif = (int *)(b + L.mif);
    c->ws_loaded = 0;
    c->sms = device_sms();
    c->dpass = (int *)(b + L.dpass);
    c->part_cap = L.part_doubles;
    c->pplan = (DynChunks *)(b + L.pplan);
    c->spred = (float *)(b + L.spred);
    c->ws_prev = (int *)(b + L.wsprev);

    // zero everything (padding lanes of the SoA arrays included), then draw X_0
    e = cudaMemsetAsync(c->ws, 0, L.total, c->st);
    if (e == cudaSuccess) e = launch_init_x0(c);
    if (e != cudaSuccess) {
        ssm_destroy(c);
        return cuda_status(e);
    }
    *out = c;
    return SSM_OK;
}

ssm_status ssm_step(ssm_ctx *c) {
    if (!c) return SSM_EINVAL;
    return ssm_run_steps(c, 1);
}

ssm_status ssm_run_steps(ssm_ctx *c, int64_t k) {
    if (!c || k < 0) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    if (c->n + k > c->M) return SSM_ESTATE;
    if (k == 0) return SSM_OK;
    cudaError_t e = cudaSuccess;
    if (!c->graph_ready) {
        cudaGraph_t g;
        e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = enqueue_step(c);
            e = cudaStreamEndCapture(c->st, &g);
            if (e1 != cudaSuccess) e = e1;
            if (e == cudaSuccess) {
                e = cudaGraphInstantiate(&c->gexec, g, 0);
                cudaGraphDestroy(g);
                if (e == cudaSuccess) c->graph_ready = true;
            }
        }
        if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    }
    for (int64_t s = 0; s < k; ++s) {
        e = cudaGraphLaunch(c->gexec, c->st);
        if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    }
    c->n += k;
    return SSM_OK;
}

ssm_status ssm_run(ssm_ctx *c) {
    if (!c) return SSM_EINVAL;
    return ssm_run_steps(c, c->M - c->n);
}

ssm_status ssm_sync(ssm_ctx *c) {
    if (!c) return SSM_EINVAL;
    return harvest(c);
}

ssm_status ssm_moments(ssm_ctx *c, double *out) {
    if (!c || !out) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    cudaError_t e = cudaMemcpyAsync(out, c->mom, sizeof(double) * 4 * c->d, cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    return harvest(c);
}

ssm_status ssm_get_state(ssm_ctx *c, double *x, int64_t *n) {
    if (!c) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    if (x) {
        cudaError_t e = launch_soa_to_aos(c->x, c->stage, c->d, c->N, c->Np, c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x, c->stage, sizeof(double) * c->d * c->N, cudaMemcpyDeviceToHost, c->st);
        if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    }
    if (n) *n = c->n;
    return harvest(c);
}

ssm_status ssm_set_state(ssm_ctx *c, const double *x, int64_t n) {
    if (!c || !x || n < 0 || n > c->M) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    cudaError_t e = cudaMemcpyAsync(c->stage, x, sizeof(double) * c->d * c->N, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = launch_aos_to_soa(c->stage, c->x, c->d, c->N, c->Np, c->st);
    // the learned start's carried error refers to the previous step of this run: kept
    // when the state comes back at the step where it stands (a host round trip of
    // the current state), dropped otherwise (the start only steers the passes; the
    // roots are certified to the same tolerance either way)
    if (e == cudaSuccess && n != c->n) e = cudaMemsetAsync(c->ws_prev, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = launch_set_step(c, n);
    if (e == cudaSuccess) e = launch_moments(c);
    // the caller's array may be reused once this returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    c->n = n;
    return SSM_OK;
}

ssm_status ssm_get_stage(ssm_ctx *c, int which, double *out) {
    if (!c || !out || (which != SSM_STAGE_Y && which != SSM_STAGE_B)) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    cudaError_t e;
    if (which == SSM_STAGE_Y) {
        e = launch_soa_to_aos(c->y, c->stage, c->d, c->N, c->Np, c->st);
    } else {
        double scale, bscale;
        drift_scale(c->coef, fp32_pairs(c), c->N, &scale, &bscale);
        e = launch_stage_b(c, bscale);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, c->stage, sizeof(double) * c->d * c->N, cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    return harvest(c);
}

ssm_status ssm_stats(ssm_ctx *c, ssm_stats_t *out) {
    if (!c || !out) return SSM_EINVAL;
    long long cn[CNT_N], hs[16];
    cudaError_t e = cudaMemcpyAsync(cn, c->counters, sizeof cn, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, c->hist, sizeof hs, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    memset(out, 0, sizeof *out);
    out->steps = cn[CNT_STEPS];
    out->newton_passes = cn[CNT_NEWTON_PASSES];
    out->newton_rows = cn[CNT_NEWTON_ROWS];
    out->drift_rows = cn[CNT_DRIFT_ROWS];
    out->fallbacks = cn[CNT_FALLBACKS];
    out->max_passes = cn[CNT_MAX_PASSES];
    out->floor_accepts = cn[CNT_FLOOR];
    for (int k = 0; k < 16; ++k) out->hist[k] = hs[k];
    return harvest(c);
}

void ssm_destroy(ssm_ctx *c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->graph_ready) cudaGraphExecDestroy(c->gexec);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->st_body) cudaStreamDestroy(c->st_body);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

int ssm_build_flags(void) {
#ifdef SSM_CHECK_BOUNDS
    return SSM_BUILD_CHECK_BOUNDS;
#else
    return 0;
#endif
}

const char *ssm_status_str(int s) {
    switch (s) {
    case SSM_OK: return "SSM_OK";
    case SSM_EINVAL: return "SSM_EINVAL: invalid argument";
    case SSM_ENOMEM: return "SSM_ENOMEM: out of device memory or workspace too small";
    case SSM_ECUDA: return "SSM_ECUDA: CUDA runtime error";
    case SSM_ENOCONV: return "SSM_ENOCONV: implicit step did not reach its tolerance";
    case SSM_ENONFINITE: return "SSM_ENONFINITE: non-finite particle state";
    case SSM_ETIMEOUT: return "SSM_ETIMEOUT: bounded device wait gave up";
    case SSM_ESTATE: return "SSM_ESTATE: call not valid in the current state";
    case SSM_EBOUNDS: return "SSM_EBOUNDS: an index checked by the debug build fell outside its array";
    }
    return "unknown ssm_status";
}

// ---- component entry points ------------------------------------------------

ssm_status ssm_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out) {
    if (!ctr || !out || n < 0 || n > N_MAX) return SSM_EINVAL;
    if (n == 0) return SSM_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc((void **)&dc, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dout, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(seed, dc, n, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return cuda_status(e);
}

ssm_status ssm_normals(uint64_t seed, int d, int64_t N, int64_t step, int stream, double *out) {
    if (!out || d < 1 || d > 3 || N < 0 || N > N_MAX || step < 0 || step > 0xffffffffll || stream < 0) return SSM_EINVAL;
    if (N == 0) return SSM_OK;
    double *dz = nullptr;
    cudaError_t e = cudaMalloc((void **)&dz, sizeof(double) * d * N);
    if (e == cudaSuccess) e = launch_normals(seed, d, N, (uint32_t)step, (uint32_t)stream, dz, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dz, sizeof(double) * d * N, cudaMemcpyDeviceToHost);
    cudaFree(dz);
    return cuda_status(e);
}

ssm_status ssm_stability_beta(double Lv, double Lvt, double Lb, double Lbt, double Ls, double Lst, double h,
                              double *beta) {
    if (!beta) return SSM_EINVAL;
    const double in[7] = { Lv, Lvt, Lb, Lbt, Ls, Lst, h };
    for (double v : in)
        if (!isfinite(v)) return SSM_EINVAL;
    if (Lvt < 0.0 || Lb < 0.0 || Lbt < 0.0 || Ls < 0.0 || Lst < 0.0 || !(h > 0.0)) return SSM_EINVAL;
    const double A = 2.0 * sqrt(Lb) + 2.0 * sqrt(Lbt) + Ls + Lst, B = Lb + Lbt;
    const double den = 1.0 - h * (2.0 * Lv + 1.0);
    if (den == 0.0) return SSM_EINVAL;
    *beta = ((2.0 * Lv + A + 1.0 + Lvt) + h * (Lvt * A + B) + h * h * B * Lvt) / den;
    return SSM_OK;
}

ssm_status ssm_convert_check(const double *in, int64_t n, float *out32, double *out64) {
    if (n < 0 || (n > 0 && (!in || !out32 || !out64))) return SSM_EINVAL;
    for (int64_t k = 0; k < n; ++k) {
        out32[k] = f64_to_f32(in[k]);
        out64[k] = f32_to_f64(out32[k]);
    }
    return SSM_OK;
}

ssm_status ssm_normals_fp32(uint64_t seed, int d, int64_t N, int64_t step, int stream, float *out) {
    if (!out || d < 1 || d > 3 || N < 0 || N > N_MAX || step < 0 || step > 0xffffffffll || stream < 0) return SSM_EINVAL;
    if (N == 0) return SSM_OK;
    float *dz = nullptr;
    cudaError_t e = cudaMalloc((void **)&dz, sizeof(float) * d * N);
    if (e == cudaSuccess) e = launch_normals32(seed, d, N, (uint32_t)step, (uint32_t)stream, dz, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dz, sizeof(float) * d * N, cudaMemcpyDeviceToHost);
    cudaFree(dz);
    return cuda_status(e);
}

ssm_status ssm_pair_pass(ssm_ctx *c, int which, int64_t *pairs) {
    if (!c || which < 0 || which > 2) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    if (is_moment(c->coef) || (which == 0 && !is_coupled(c->coef))) return SSM_EINVAL;
    if (which == 2 && !(c->prec == SSM_FP32C_LEARNED && c->ws_loaded)) return SSM_EINVAL;
    const bool f32 = fp32_pairs(c);
    cudaError_t e;
    if (which == 2) {
        e = ws_forward_start(c);
        // the start alone leaves predictions that no step converged: no correction next step
        if (e == cudaSuccess) e = cudaMemsetAsync(c->ws_prev, 0, sizeof(int), c->st);
        if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
        if (pairs) *pairs = 0;
        return SSM_OK;
    }
    if (which == 0) {
        e = pair_sums(newton_kind(c->d), f32, c->plan_newton, c->x, c->y, nullptr, nullptr, c->N, c->Np, 1.0,
                      c->part, c->st);
    } else {
        double scale, bscale;
        drift_scale(c->coef, f32, c->N, &scale, &bscale);
        e = pair_sums(drift_kind(c->coef), f32, c->plan_drift, c->y, c->y,
                      nullptr, nullptr, c->N, c->Np, scale, c->part, c->st);
    }
    if (e != cudaSuccess) { c->status = cuda_status(e); return (ssm_status)c->status; }
    if (pairs) *pairs = c->N * c->N;
    return SSM_OK;
}

// Time every compiled launch shape of each pair kind this context uses on its
// current state (CUDA events on the context's stream) and keep the fastest.
ssm_status ssm_autotune(ssm_ctx *c, double *best_ms) {
    if (!c) return SSM_EINVAL;
    if (c->status != SSM_OK) return (ssm_status)c->status;
    if (is_moment(c->coef)) return SSM_OK;
    const bool f32 = fp32_pairs(c);
    double scale, bscale;
    drift_scale(c->coef, f32, c->N, &scale, &bscale);
    const int kd = drift_kind(c->coef), kn = newton_kind(c->d);
    const int kinds[2] = { kn, kd };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SSM_ECUDA;
    cudaError_t err = cudaSuccess;
    for (int q = 0; q < 2 && err == cudaSuccess; ++q) {
        const int kind = kinds[q];
        if (q == 0 && !is_coupled(c->coef)) continue;
        const double *src = q == 0 ? c->x : c->y;
        const double sc = q == 0 ? 1.0 : scale;
        int cand[32][3];
        const int nc = pair_shape_candidates(kind, f32, cand, 32);
        Plan best = q == 0 ? c->plan_newton : c->plan_drift;
        float best_t = 1e30f;
        // one warm pass, then two timed passes of plan p; keeps the fastest
        auto try_plan = [&](const Plan &p) {
            err = pair_sums(kind, f32, p, src, c->y, nullptr, nullptr, c->N, c->Np, sc, c->part, c->st);
            if (err == cudaSuccess) err = cudaEventRecord(e0, c->st);
            for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep)
                err = pair_sums(kind, f32, p, src, c->y, nullptr, nullptr, c->N, c->Np, sc, c->part, c->st);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c->st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < best_t) { best_t = ms; best = p; }
        };
        for (int k = 0; k < nc && err == cudaSuccess; ++k) {
            const int slots = device_slots(kind, f32, cand[k][0], cand[k][1], cand[k][2]);
            if (slots <= 0) continue;
            try_plan(make_plan_shape(c->N, kind, cand[k][0], cand[k][1], cand[k][2], c->opt.tile_chunks, slots));
        }
        // Then the chunk count of the fastest shape: 1.5, 2 and 2.5 times the planned
        // count (finer work items balance the last wave better; measured at N = 2^18,
        // 128 x 8 drift: 17.9 ms with 7 chunks, 17.6 ms with 16).  Every chunk adds a
        // set of partial sums that is written to memory and read back by the
        // consumer, so a larger count is kept only when it is faster by more than
        // 0.5%.
        if (c->opt.tile_chunks <= 0) {
            const Plan base = best;
            const int cap = chunks_cap(c->N, kind_nc(kind));
            for (int m = 3; m <= 5 && err == cudaSuccess; ++m) {
                int ch = base.chunks * m / 2;
                if (ch > cap) ch = cap;
                if (ch <= base.chunks) continue;
                const Plan p = make_plan_shape(c->N, kind, base.vec2, base.threads, base.rpt, ch, 0);
                if (p.chunks == base.chunks) continue;
                const Plan keep = best;
                const float keep_t = best_t;
                try_plan(p);
                if (best.chunks == p.chunks && !(best_t < 0.995f * keep_t)) { best = keep; best_t = keep_t; }
            }
        }
        if (q == 0) c->plan_newton = best; else c->plan_drift = best;
        if (best_ms) best_ms[q] = best_t / 2.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) { c->status = cuda_status(err); return (ssm_status)c->status; }
    if (c->graph_ready) { cudaGraphExecDestroy(c->gexec); c->graph_ready = false; }
    return SSM_OK;
}

ssm_status ssm_get_plan(ssm_ctx *c, int which, int *out) {
    if (!c || !out || (which != 0 && which != 1)) return SSM_EINVAL;
    const Plan &p = which == 0 ? c->plan_newton : c->plan_drift;
    out[0] = p.vec2; out[1] = p.threads; out[2] = p.rpt; out[3] = p.chunks; out[4] = (int)p.chunk_len;
    return SSM_OK;
}

// A compiled shape {form, threads, targets per thread} with `chunks` source chunks
// (0: planned from the device's slots, or ssm_opts.tile_chunks).
static ssm_status set_plan_shape(ssm_ctx *c, int which, const int *in, int chunks) {
    if (!c || !in || (which != 0 && which != 1)) return SSM_EINVAL;
    if (is_moment(c->coef) || (which == 0 && !is_coupled(c->coef))) return SSM_EINVAL;
    const bool f32 = fp32_pairs(c);
    const int kind = which == 0 ? newton_kind(c->d) : drift_kind(c->coef);
    if (chunks < 0 || chunks > chunks_cap(c->N, kind_nc(kind))) return SSM_EINVAL;
    int cand[32][3];
    const int nc = pair_shape_candidates(kind, f32, cand, 32);
    bool ok = false;
    for (int k = 0; k < nc; ++k)
        if (cand[k][0] == in[0] && cand[k][1] == in[1] && cand[k][2] == in[2]) ok = true;
    if (!ok) return SSM_EINVAL;
    const int slots = device_slots(kind, f32, in[0], in[1], in[2]);
    Plan p = make_plan_shape(c->N, kind, in[0], in[1], in[2], chunks > 0 ? chunks : c->opt.tile_chunks, slots);
    if (which == 0) c->plan_newton = p; else c->plan_drift = p;
    if (c->graph_ready) { cudaGraphExecDestroy(c->gexec); c->graph_ready = false; }
    return SSM_OK;
}

ssm_status ssm_set_plan(ssm_ctx *c, int which, const int *in) { return set_plan_shape(c, which, in, 0); }

ssm_status ssm_set_plan_chunks(ssm_ctx *c, int which, const int *in) {
    if (!in) return SSM_EINVAL;
    if (in[3] < 1) return SSM_EINVAL;
    return set_plan_shape(c, which, in, in[3]);
}

ssm_status ssm_cardano(const double *x, int64_t n, double h, double *y) {
    if (!x || !y || n < 0 || n > N_MAX || !(h > 0.0) || !(h < 1.0 / 3.0 + 1e-15)) return SSM_EINVAL;
    if (n == 0) return SSM_OK;
    double *dx = nullptr, *dy = nullptr;
    cudaError_t e = cudaMalloc((void **)&dx, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dy, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_cardano(dx, dy, n, h, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dy);
    return cuda_status(e);
}

}  // extern "C"
