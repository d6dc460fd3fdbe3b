// k_particle.cu -- the O(N) kernels of the split-step method: initial state,
// the per-particle parts of step 1 (Cardano closed form, the Newton-type update
// that consumes the pair sums, the linear OU solve), and step 2 fused with the
// Brownian increments and the FP64 moment reduction.
//
// References are to Chen & dos Reis, arXiv:2105.09688: §2.3 (eq. SSTM:scheme 1
// and SSTM:scheme 2), Lemma 4.1 (unique root of the implicit map), §3.4.1
// (the OU example).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include "particle_ops.cuh"
#include "ssm_device.cuh"

namespace ssm {

// ---------------------------------------------------------------------------
// Block reduction of NV doubles per thread into out[NV] (thread 0 writes).
// ---------------------------------------------------------------------------
template <int NV, int THREADS>
__device__ __forceinline__ void block_sum(double *v, double *out) {
    __shared__ double sh[THREADS / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) s += sh[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// True in exactly one block: the last to finish (its view of the other blocks'
// partials is complete).  Resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) *ticket = 0u;
    return is_last;
}

// Moments (1/N) sum_i x^k, k = 1..4, for D components: per-block partials in
// mpart[block][4*D], reduced in block order by the last block into mom[4*D].
template <int D>
__device__ __forceinline__ void moments_epilogue(double (&m)[4 * D], int64_t N, double *mpart, unsigned *ticket,
                                                 double *mom, int *err) {
    __shared__ double bsum[4 * D];
    block_sum<4 * D, EUL_THREADS>(m, bsum);
    __syncthreads();
    if (threadIdx.x < 4 * D) mpart[(int64_t)blockIdx.x * 4 * D + threadIdx.x] = bsum[threadIdx.x];
    if (last_block(ticket)) {
        if (threadIdx.x < 4 * D) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&mpart[(int64_t)b * 4 * D + threadIdx.x]);
            const double v = s / (double)N;
            mom[threadIdx.x] = v;
            if (!isfinite(v)) atomicOr(err, ERR_NONFINITE);
        }
    }
}

// X_0^i = mean + std Z^i, Z from Philox stream 0 at step 0 (and its moments).
template <int D>
__global__ void __launch_bounds__(EUL_THREADS)
k_init_x0(double *x, int64_t N, int64_t Np, uint64_t seed, double mean, double sd, double *mpart,
          unsigned *ticket, double *mom, int *err) {
    double m[4 * D];
#pragma unroll
    for (int k = 0; k < 4 * D; ++k) m[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double z[3];
        normals<D>(seed, (uint32_t)i, 0u, 0u, z);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double v = mean + sd * z[c];
            x[c * Np + i] = v;
            add_powers<D>(m, c, v);
        }
    }
    moments_epilogue<D>(m, N, mpart, ticket, mom, err);
}

template <int D>
__global__ void __launch_bounds__(EUL_THREADS)
k_moments(const double *x, int64_t N, int64_t Np, double *mpart, unsigned *ticket, double *mom, int *err) {
    double m[4 * D];
#pragma unroll
    for (int k = 0; k < 4 * D; ++k) m[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < D; ++c) add_powers<D>(m, c, x[c * Np + i]);
    moments_epilogue<D>(m, N, mpart, ticket, mom, err);
}

// ---------------------------------------------------------------------------
// Step 1 for a cubic drift: the real root of h y^3 + a y - x = 0, a > 0
// (a = 1 - h for v = x - x^3, SSM_COEF_CUBIC1D_GAUSS; a = 1 for v = -x^3, the GL
// and Cucker-Smale sets).  Depressed cubic y^3 + p y + q = 0, p = a/h > 0,
// q = -x/h: one real root.  With y = u + w, u w = -p/3 and u^3 + w^3 = -q, the
// root equals -q / (u^2 + p/3 + w^2), a quotient of positive sums that keeps full
// relative accuracy for small |x|.  One Newton correction follows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cardano_root_a(double x, double h, double a) {
    if (x == 0.0) return 0.0;
    const double p = a / h, q = -x / h;
    const double p3 = p / 3.0;
    const double disc = 0.25 * q * q + p3 * p3 * p3;
    double u = cbrt(0.5 * fabs(q) + sqrt(disc));
    if (q > 0.0) u = -u;
    const double w = -p3 / u;
    const double y = -q / (u * u + p3 + w * w);
    const double f = h * y * y * y + a * y - x;
    const double fp = 3.0 * h * y * y + a;
    return y - f / fp;
}
__device__ __forceinline__ double cardano_root(double x, double h) { return cardano_root_a(x, h, 1.0 - h); }

// The root of h y^3 + a y = x + c for the FP32C forms (c: GL2's measure term, else
// 0).  The Cardano form in FP32 gives y0 (relative error ~1e-7; its cube root and
// square root on the special-function unit); one Newton
// correction y0 - f(y0) / f'(y0) follows, with the residual f = h y0^3 + a y0 - x - c
// evaluated in double-float arithmetic on the FP32 pipe (error-free products by FMA
// and Knuth's two-sum; x split into two floats on the integer pipes, h, a and c
// split once per thread) to ~2^-47 of its terms, and the derivative in FP32.  That
// leaves ~1e-13 relative (quadratic convergence plus the derivative's rounding
// times the first error; for |x| < 2^-74 the low half of x is dropped, < 2^-98
// absolute).  One FP64 operation per root: the final add.
struct Cubic32 {
    float hf, af, p3, ih;           // h, a, a / (3 h), 1 / h in FP32
    float h_hi, h_lo, a_hi, a_lo;   // h and a as unevaluated pairs of floats
    float c_hi, c_lo;               // c likewise
};
__device__ __forceinline__ void split_pair(double v, float &hi, float &lo) {
    hi = f64_to_f32(v);
    lo = f64_to_f32(v - f32_to_f64(hi));
}
__device__ __forceinline__ Cubic32 make_cubic32(double h, double a, double c) {   // once per thread
    Cubic32 k;
    k.hf = (float)h;
    k.af = (float)a;
    k.p3 = (float)(a / (3.0 * h));
    k.ih = (float)(1.0 / h);
    split_pair(h, k.h_hi, k.h_lo);
    split_pair(a, k.a_hi, k.a_lo);
    split_pair(c, k.c_hi, k.c_lo);
    return k;
}
template <bool A1, bool SHIFT>   // A1: a = 1; SHIFT: c != 0
__device__ __forceinline__ double cardano32_a(double x, const Cubic32 &k) {
    float xh, xl;
    split_f64(x, xh, xl);
    const float xs = SHIFT ? xh + k.c_hi : xh;
    const float q = -xs * k.ih;
    const float disc = fmaf(0.25f * q, q, k.p3 * k.p3 * k.p3);
    // u = cbrt(cv), cv = |q|/2 + sqrt(disc) >= p3^(3/2) > 0 (a normal float):
    // 2^(log2(cv)/3) on the special-function unit (~3e-7 relative), then one Newton step
    // for the cube root, u <- (2u + cv/u^2)/3, to FP32 rounding; the square root's ~2^-22
    // only moves cv, which the correction of the cubic's root below absorbs
    const float cv = fmaf(0.5f, fabsf(q), sqrt_approx(disc));
    float u = ex2_approx(lg2_approx(cv) * (1.0f / 3.0f));
    u = (2.0f * u + cv * (rcp_approx(u * u))) * (1.0f / 3.0f);
    if (q > 0.0f) u = -u;
    const float w = __fdividef(-k.p3, u);
    const float y0 = __fdividef(-q, fmaf(u, u, k.p3) + w * w);
    // h y0^3 = r + rl
    const float p = y0 * y0, ep = fmaf(y0, y0, -p);
    const float cb = p * y0, ecb = fmaf(p, y0, -cb);
    const float cl = fmaf(ep, y0, ecb);
    const float r = k.h_hi * cb, er = fmaf(k.h_hi, cb, -r);
    const float rl = fmaf(k.h_hi, cl, fmaf(k.h_lo, cb, er));
    // a y0 = s + sl
    float s = y0, sl = 0.0f;
    if (!A1) {
        s = k.a_hi * y0;
        sl = fmaf(k.a_lo, y0, fmaf(k.a_hi, y0, -s));
    }
    // f = (s - x_hi - c_hi) + r + (small terms)
    float t, te, v, ve;
    two_sum(s, -xh, t, te);
    float ce = 0.0f;
    if (SHIFT) {
        float t2;
        two_sum(t, -k.c_hi, t2, ce);
        t = t2;
    }
    two_sum(t, r, v, ve);
    const float f = v + ((ve + te + ce) + (rl + sl - xl - (SHIFT ? k.c_lo : 0.0f)));
    const float fp = fmaf(3.0f * k.hf * y0, y0, k.af);
    // the FP64 result with the hardware conversions: this kernel's integer pipe is the
    // busier one (the bit-level conversions and splits), its FP64 pipe the idler
    return (double)y0 - (double)__fdividef(f, fp);
}

__global__ void k_cardano(const double *__restrict__ x, double *__restrict__ y, int64_t n, double h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = cardano_root(x[i], h);
}

// Step 1 of the sets whose measure enters through means (OU, GL1, GL2, POLY, CS),
// all per particle against the frozen mu^X, whose moments mom (of X_n) are known:
//   OU:   Y = X / (1 - h rho) (Remark 4.3), as a product with the reciprocal
//         (an FP64 division costs many FP64-pipe instructions, and that pipe runs
//         at 1/64 of the FP32 rate here);
//   GL1:  Y + h Y^3 = X;  GL2: Y + h Y^3 = X + h c mean(X);
//   POLY: Y = X / (1 - h gamma + h mean(X^2));  CS: V_Y + h V_Y^3 = V, X_Y = X;
//   GLSTAB: (h/4) Y^3 + (1 + h (5/2 + gamma)) Y = X;
// and the mean of Y that step 2 needs -- summed in compensated FP32 per thread in
// the FP32C form (whose cubic roots are cardano32_a), in FP64 otherwise; blocks
// combine in FP64.
template <int D, bool F32>
__global__ void __launch_bounds__(EUL_THREADS)
k_mm_implicit(int coef, const double *__restrict__ x, double *__restrict__ y, int64_t N, int64_t Np, double h,
              double p0, double p1, const double *__restrict__ xmom, double *mpart, unsigned *ticket,
              double *ymean) {
    double m[D];
    float mh[D], ml[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { m[c] = 0.0; mh[c] = 0.0f; ml[c] = 0.0f; }
    double lin = 1.0, shift = 0.0;   // OU and POLY: the factor; GL2: the measure term
    if (coef == SSM_COEF_OU) lin = 1.0 / (1.0 - h * p0);
    if (coef == SSM_COEF_POLY) lin = 1.0 / (1.0 - h * p0 + h * xmom[D]);
    if (coef == SSM_COEF_GL2) shift = h * p1 * xmom[0];
    const bool cubic = coef == SSM_COEF_GL1 || coef == SSM_COEF_GL2 || coef == SSM_COEF_CS || coef == SSM_COEF_GLSTAB;
    // the cubic h3 y^3 + a1 y = x + shift
    const double h3 = coef == SSM_COEF_GLSTAB ? 0.25 * h : h;
    const double a1 = coef == SSM_COEF_GLSTAB ? 1.0 + h * (2.5 + p0) : 1.0;
    const Cubic32 k32 = make_cubic32(h3, a1, shift);
    auto add = [&](int c, double v) {
        if (F32) two_sum_acc(mh[c], ml[c], f64_to_f32(v));
        else m[c] += v;
    };
    // The loop is compiled once per (LIN: the linear sets, SHIFT: GL2's measure term,
    // A1: a1 = 1), so no FP64 operation that a set does not need is issued, not even
    // predicated off (the FP64 pipe bounds this kernel in the FP32C form).  Two
    // particles per iteration, both loaded before either is used (memory-level
    // parallelism for this streaming kernel).
    auto sweep = [&](auto lin_t, auto shift_t, auto a1_t) {
        constexpr bool LIN = decltype(lin_t)::value, SHIFT = decltype(shift_t)::value, A1 = decltype(a1_t)::value;
        auto root = [&](int c, double xv) -> double {
            if (LIN) return xv * lin;
            if (c > 0) return xv;   // X part of Cucker-Smale's (V, X): v = 0
            if (F32) return cardano32_a<A1, SHIFT>(xv, k32);
            return cardano_root_a(SHIFT ? xv + shift : xv, h3, a1);
        };
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += 2 * stride) {
            const bool two = i + stride < N;
            double xa[D], xb[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                xa[c] = x[c * Np + i];
                xb[c] = two ? x[c * Np + i + stride] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double va = root(c, xa[c]);
                y[c * Np + i] = va;
                add(c, va);
                if (two) {
                    const double vb = root(c, xb[c]);
                    y[c * Np + i + stride] = vb;
                    add(c, vb);
                }
            }
        }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (!cubic) sweep(T_{}, F_{}, T_{});                      // OU, POLY
    else if (coef == SSM_COEF_GL2) sweep(F_{}, T_{}, T_{});
    else if (coef == SSM_COEF_GLSTAB) sweep(F_{}, F_{}, F_{});
    else sweep(F_{}, F_{}, T_{});                             // GL1, CS
    if (F32)
#pragma unroll
        for (int c = 0; c < D; ++c) m[c] = (double)mh[c] + (double)ml[c];
    __shared__ double bsum[D];
    block_sum<D, EUL_THREADS>(m, bsum);
    __syncthreads();
    if (threadIdx.x < D) mpart[(int64_t)blockIdx.x * D + threadIdx.x] = bsum[threadIdx.x];
    if (last_block(ticket) && threadIdx.x < D) {
        double sm = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) sm += __ldcg(&mpart[(int64_t)b * D + threadIdx.x]);
        ymean[threadIdx.x] = sm / (double)N;
    }
}

// ---------------------------------------------------------------------------
// Step 1 of the coupled sets (d = 3 and d = 1).  The implicit equation
//   F(Y) = Y - X - h ( -Y|Y|^2 + 0.5 S(Y) ) = 0,  S(Y) = (1/N) sum_j (X_j - Y) w_j,
//   w_j = 1 / (1 + |X_j - Y|^2)
// is solved for all particles at once in passes.  Each pass evaluates S and
// Sw = (1/N) sum_j w_j at the current Y of every unconverged particle (the
// O(N^2) pair kernel), then k_newton_update forms the FP64 residual and either
// retires the particle or moves it (newton_update_particle).  The outer
// iteration contracts by about 0.5 h |(2 w^2 d d^T)| per pass.
// ---------------------------------------------------------------------------
// Plain start Y = X (a learned start, when enabled, overwrites Y afterwards);
// resets the active list, pass counters and histogram, and keeps the moments of
// X_n that the learned start and the training-data collection use.
template <int D>
__global__ void k_newton_begin(const double *__restrict__ x, double *__restrict__ y, int *__restrict__ act,
                               int *__restrict__ cnt, int kmax, int *__restrict__ passes, long long *hist,
                               const double *__restrict__ mom, double *__restrict__ mom_prev, int64_t N, int64_t Np,
                               int *__restrict__ dpass, int inject, DynChunks *pplan, DynChunks full) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
#pragma unroll
        for (int c = 0; c < D; ++c) y[c * Np + i] = x[c * Np + i];
        act[i] = (int)i;
        passes[i] = 0;
    }
    if (i == 0) {
        cnt[0] = (int)N;
        for (int k = 1; k <= kmax; ++k) cnt[k] = 0;
        for (int k = 0; k < 16; ++k) hist[k] = 0;
        for (int k = 0; k < 4 * D; ++k) mom_prev[k] = mom[k];
        *dpass = 0;
        *pplan = full;   // the first pass covers every particle: the planned shape
#ifdef SSM_CHECK_BOUNDS
        // ssm_opts.inject = 1 (debug builds, N not a multiple of 128): list entry 0
        // names particle N, past the particles but inside the padded arrays, for
        // the bounds checks to catch
        if (inject == 1) act[0] = (int)N;
#endif
    }
}

// One pass's update of every active particle.  The pass index and the active lists:
// pass = *dpass inside the device-driven pass loop of the step graph (LOOP; the last
// block then advances *dpass and sets the loop's condition hpass: another pass while
// particles remain and pass + 1 < kmax), else pass_arg; the particles of the pass are
// act[pass & 1][0 .. cnt[pass]) and the survivors go to the other list and
// cnt[pass + 1].  The instance without LOOP holds no device-side graph call, so
// profilers that skip such kernels still see it in the fixed pass sequence.
template <int D, bool LOOP>
__global__ void __launch_bounds__(256)
k_newton_update(const double *__restrict__ x, double *__restrict__ y, int *__restrict__ act0,
                int *__restrict__ act1, int *__restrict__ cnt, const double *__restrict__ part, DynChunks *pplan,
                Plan plan, int sub, int64_t part_cap, int64_t N, int64_t Np, double h, double tol, int fp32_targets,
                int pass_arg, int kmax,
                int *__restrict__ passes, long long *hist, int *err, double *__restrict__ sconv, int restart_pass,
                long long *counters, float *__restrict__ rprev, int *__restrict__ dpass, unsigned *ticket,
                cudaGraphConditionalHandle hpass) {
    constexpr int NC = D + 1;
    const int pass = LOOP ? *dpass : pass_arg;
    const int *__restrict__ act_in = (pass & 1) ? act1 : act0;
    int *__restrict__ act_out = (pass & 1) ? act0 : act1;
    const int *cnt_in = cnt + pass;
    int *cnt_out = cnt + pass + 1;
    __shared__ int bh[16];
    __shared__ int nrestart, nfloor;
    if (threadIdx.x < 16) bh[threadIdx.x] = 0;
    if (threadIdx.x == 0) { nrestart = 0; nfloor = 0; }
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n_in = *cnt_in;
    if (t == 0 && !SSM_IN_BOUNDS(n_in >= 0 && n_in <= N)) n_in = 0;
    if (!(n_in >= 0 && n_in <= N)) n_in = 0;
    const DynChunks dc = *pplan;   // the chunking the pair kernel used for this pass
    bool keep = false;
    int i = 0;
    if (t < n_in && SSM_IN_BOUNDS(act_in[t] >= 0 && act_in[t] < N)) {
        i = act_in[t];
        double S[D], Sw = 0.0, Y[D], X[D];
#pragma unroll
        for (int c = 0; c < D; ++c) S[c] = 0.0;
        for (int k = 0; k < dc.chunks; ++k) {
            const double *pk = part + (int64_t)k * NC * dc.stride + t;
#pragma unroll
            for (int c = 0; c < D; ++c) S[c] += pk[c * dc.stride];
            Sw += pk[D * dc.stride];
        }
        const double invN = 1.0 / (double)N;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            S[c] *= invN;
            Y[c] = y[c * Np + i];
            X[c] = x[c * Np + i];
        }
        Sw *= invN;
        const int r = newton_update_particle<D>(S, Sw, Y, X, h, tol, fp32_targets != 0, pass, kmax, restart_pass,
                                                &rprev[i]);
        if (r == UPD_CONVERGED || r == UPD_FLOOR) {
            passes[i] = pass + 1;
            atomicAdd(&bh[pass + 1 < 15 ? pass + 1 : 15], 1);
            if (r == UPD_FLOOR) atomicAdd(&nfloor, 1);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                y[c * Np + i] = Y[c];
                sconv[c * Np + i] = S[c];
            }
        } else if (r == UPD_NOCONV || r == UPD_NONFINITE) {
            passes[i] = pass + 1;
            atomicOr(err, r == UPD_NOCONV ? ERR_NOCONV : ERR_NONFINITE);
        } else {
            // UPD_RESTART (a learned start that missed the tolerance after
            // restart_pass passes goes back to the plain start Y = X) or UPD_CONTINUE
#pragma unroll
            for (int c = 0; c < D; ++c) y[c * Np + i] = Y[c];
            if (r == UPD_RESTART) atomicAdd(&nrestart, 1);
            keep = true;
        }
    }
    // warp-aggregated append of the particles that stay active
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m) {
        const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(cnt_out, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (keep) act_out[base + __popc(m & ((1u << lane) - 1u))] = i;
    }
    __syncthreads();
    if (threadIdx.x < 16 && bh[threadIdx.x]) atomicAdd((unsigned long long *)&hist[threadIdx.x], (unsigned long long)bh[threadIdx.x]);
    if (threadIdx.x == 0 && nrestart)
        atomicAdd((unsigned long long *)&counters[CNT_FALLBACKS], (unsigned long long)nrestart);
    if (threadIdx.x == 0 && nfloor)
        atomicAdd((unsigned long long *)&counters[CNT_FLOOR], (unsigned long long)nfloor);
    // the last block (every block has read this pass's plan and appended its survivors)
    // writes the chunking of the next pass and, in the device-driven loop, its index
    // and whether it runs
    if (last_block(ticket) && threadIdx.x == 0) {
        const int next = __ldcg(cnt_out);
        const int tile = plan.threads * plan.rpt;
        *pplan = dyn_chunks(next, N, Np, tile, (int)((N + tile - 1) / tile), plan.chunks, plan.chunk_len, sub, NC,
                            part_cap);
        if constexpr (LOOP) {
            *dpass = pass + 1;
            cudaGraphSetConditional(hpass, (next > 0 && pass + 1 < kmax) ? 1u : 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// Step 1 against mu^Y (ssm_opts.measure_y): the joint system G(Y) = 0 in R^{dN},
// G_i = Y_i - X_i - h v(Y_i, mu^Y), of the earlier implicit scheme that §1 sets the
// SSM against.  Nonlinear block-Jacobi passes: pass k evaluates S_i and Sw_i at the
// common iterate Y^k for every particle (the pair kernel with sources = targets =
// Y^k), which is the exact joint residual G_i(Y^k).  When every particle is within
// tol the step ends at Y^k; otherwise every particle moves to the root of its local
// model with the others held at Y^k (the local solve of the SSM's step 1), into a
// proposal array that k_mi_commit copies over Y.  The coupling through the other
// particles is O(h/2) per pass, so a few passes reach tol from Y = X -- Krylov
// acceleration of the outer iteration would not pay at these contraction rates.
// The pass that would only verify the last move is saved by a bound: with the
// local bound b_i of the SSM's step 1 at the proposal (mean value theorem on the
// particle's own pair terms) and every pair term f(d) = d / (1 + |d|^2) being
// 1-Lipschitz, moving the other particles by D_j changes S_i by at most
// (1/N) sum_j |D_j| <= max_j |D_j|, so |G_i(Y^{k+1})| <= b_i + (h/2) max_j |D_j|.
// flags[k] is set when some particle of pass k was not within tol; flags[kmax+1+2k]
// and flags[kmax+2+2k] hold max_i b_i and max_j |D_j| (non-negative floats as bits).
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_mi_begin(const double *__restrict__ x, double *__restrict__ y, int *__restrict__ act,
                           int *__restrict__ cnt, int *__restrict__ flags, int kmax, int64_t N, int64_t Np) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
#pragma unroll
        for (int c = 0; c < D; ++c) y[c * Np + i] = x[c * Np + i];
        act[i] = (int)i;
    }
    if (i == 0) {
        cnt[0] = (int)N;
        for (int k = 1; k <= kmax; ++k) cnt[k] = 0;
        for (int k = 0; k < MIF_WORDS(kmax); ++k) flags[k] = 0;
    }
}

template <int D>
__global__ void __launch_bounds__(256)
k_mi_update(const double *__restrict__ x, const double *__restrict__ y, double *__restrict__ prop,
            const int *__restrict__ cnt, const double *__restrict__ part, int chunks, int64_t N, int64_t Np, double h,
            double tol, int fp32, int pass, int kmax, int *__restrict__ flags, float *__restrict__ rprev, int *err) {
    constexpr int NC = D + 1;
    if (cnt[pass] == 0) return;   // converged at an earlier pass (grid-uniform)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool conv = true, floor_acc = false;
    float lb = 0.0f, mv = 0.0f;
    if (i < N) {
        double S[D], Sw = 0.0, Y[D], X[D];
#pragma unroll
        for (int c = 0; c < D; ++c) S[c] = 0.0;
        for (int k = 0; k < chunks; ++k) {
            const double *pk = part + (int64_t)k * NC * Np + i;
#pragma unroll
            for (int c = 0; c < D; ++c) S[c] += pk[c * Np];
            Sw += pk[D * Np];
        }
        const double invN = 1.0 / (double)N;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            S[c] *= invN;
            Y[c] = y[c * Np + i];
            X[c] = x[c * Np + i];
        }
        Sw *= invN;
        if (fp32)   // numerators were taken at fl(Y_i): (y_j - Y_i) = (y_j - fl(Y_i)) - (Y_i - fl(Y_i))
#pragma unroll
            for (int c = 0; c < D; ++c) S[c] -= (Y[c] - (double)(float)Y[c]) * Sw;
        double yy = 0.0, rinf = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) yy += Y[c] * Y[c];
        bool bad = !(yy < 1e300);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double r = Y[c] - X[c] - h * (-Y[c] * yy + 0.5 * S[c]);
            if (!(r == r)) bad = true;
            rinf = fmax(rinf, fabs(r));
        }
        if (bad) atomicOr(err, ERR_NONFINITE);
        // FP32 sums: accepted at their evaluation floor as in the SSM's step 1
        conv = bad || rinf <= tol || (fp32 && pass > 0 && rinf <= 64.0 * tol && rinf > 0.1 * (double)rprev[i]);
        floor_acc = conv && !bad && !(rinf <= tol);
        rprev[i] = (float)rinf;
        double u[D];
        local_root<D>(S, Sw, Y, X, h, u);
        double uu = 0.0, du2 = 0.0, ginf = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) uu += u[c] * u[c];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            prop[c * Np + i] = u[c];
            const double du = u[c] - Y[c];
            ginf = fmax(ginf, fabs(u[c] - X[c] + h * u[c] * uu - 0.5 * h * S[c] + 0.5 * h * Sw * du));
            du2 += du * du;
        }
        const double dn = sqrt(du2);
        lb = (float)(0.5 * h * (0.5 + 0.65 * dn) * dn + ginf) * 1.0001f;   // rounded up past FP32
        mv = (float)dn * 1.0001f;
    }
    if (__any_sync(0xffffffffu, !conv) && (threadIdx.x & 31) == 0) atomicOr(&flags[pass], 1);
    const unsigned fm = __ballot_sync(0xffffffffu, floor_acc);
    if (fm && (threadIdx.x & 31) == 0) atomicAdd(&flags[MIF_FLOOR(kmax) + pass], __popc(fm));
    for (int o = 16; o > 0; o >>= 1) {
        lb = fmaxf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
        mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, o));
    }
    if ((threadIdx.x & 31) == 0) {   // non-negative floats order like their bit patterns
        atomicMax(&flags[kmax + 1 + 2 * pass], __float_as_int(lb));
        atomicMax(&flags[kmax + 2 + 2 * pass], __float_as_int(mv));
    }
}

template <int D>
__global__ void k_mi_commit(double *__restrict__ y, const double *__restrict__ prop, int *__restrict__ cnt,
                            const int *__restrict__ flags, int pass, int kmax, int64_t N, int64_t Np, double h,
                            double tol, int *err) {
    if (cnt[pass] == 0 || flags[pass] == 0) return;   // done: Y^pass is the solution
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N)
#pragma unroll
        for (int c = 0; c < D; ++c) y[c * Np + i] = prop[c * Np + i];
    if (i == 0) {
        const double lbmax = (double)__int_as_float(flags[kmax + 1 + 2 * pass]);
        const double mvmax = (double)__int_as_float(flags[kmax + 2 + 2 * pass]);
        const bool certified = lbmax + 0.5 * h * mvmax <= tol;   // done at the proposal
        if (!certified) {
            if (pass + 1 < kmax) cnt[pass + 1] = (int)N;
            else atomicOr(err, ERR_NOCONV);
        }
    }
}

// Work counters of one implicit step (one thread).  mi_flags (step 1 against mu^Y,
// else null): the particles accepted at the FP32 floor in the step's last pass.
__global__ void k_step_stats(const int *cnt, int kmax, long long N, long long *counters, const int *mi_flags,
                             int *ws_prev) {
    if (ws_prev) *ws_prev = 1;   // learned or carried start: this step's converged sums (and predictions) match
    long long rows = 0, npass = 0;
    for (int k = 0; k < kmax; ++k) {
        rows += cnt[k];
        if (cnt[k] > 0) npass = k + 1;
    }
    if (mi_flags && npass > 0) counters[CNT_FLOOR] += mi_flags[MIF_FLOOR(kmax) + npass - 1];
    counters[CNT_NEWTON_ROWS] += rows;
    counters[CNT_NEWTON_PASSES] += npass;
    if (npass > counters[CNT_MAX_PASSES]) counters[CNT_MAX_PASSES] = npass;
}

// ---------------------------------------------------------------------------
// Step 2 (eq. SSTM:scheme 2) fused with the Brownian increment and the moments
// of the new state:  X'_i = Y_i + h b(Y_i, mu^Y) + sigma(Y_i) dW_n^i.
// b comes from the pair partials (bscale folds in 1/N, the coefficient and the
// FP32 coordinate scale) or, for OU, from lambda * mean(Y).  dW is drawn on the
// step's own grid (fine_r = 1) or summed over fine_r increments of the finer
// grid, so that runs at different h share one Brownian path.
// ---------------------------------------------------------------------------
// FP32C form (F32): dW from the FP32 transform, the increment h b + sigma dW in FP32
// added to the FP64 state with one FP64 add, and the moments from FP32 powers summed
// in FP32 over 32 particles and in FP64 beyond (per thread, then across threads and
// blocks).  FP64 form:
// all FP64.  Compiled for eul_min_blocks<D> resident blocks per SM (3 at d = 2 and
// 3, whose FP32C forms need more than 64 registers a thread; 4 at d = 1) and
// launched on that many blocks per SM, one wave.
// FAM, the coefficient family, fixed at compile time so that each instance carries
// only its own branch: EUL_PAIR (b from the pair partial sums, sigma per particle),
// EUL_OU (b = lambda mean(Y), sigma = eta, the same for every particle), EUL_GEN
// (the other moment sets: b and sigma from Y and its means, moment_b / moment_sigma).
// S1: step 1 in the same kernel, for the sets whose step 1 is linear in the particle
// (OU: Y = X / (1 - h rho); polynomial drift: Y = X / (1 - h gamma + h mean(X^2))).
// Then Y = lin X needs only the moments of X_n, which the previous step (or the
// initial state) left in mom, and so does mean(Y) = lin mean(X); the kernel reads X,
// writes the stage Y and the new X, one pass over the state instead of two kernels
// (k_mm_implicit, then this one) and no grid-wide reduction between them.  mean(Y)
// differs from the sum over the Y_i by rounding only.
enum : int { EUL_PAIR = 0, EUL_OU = 1, EUL_GEN = 2 };
template <int D> constexpr int eul_min_blocks = D >= 2 ? EUL_MIN_BLOCKS : RED_PER_SM;
// CF: the coefficient set fixed at compile time (the EUL_GEN instances, so that the
// per-particle b and sigma carry no switch over the sets), or -1 to take `coef`.
template <int D, bool F32, int FAM, bool S1 = false, int CF = -1>
__global__ void __launch_bounds__(EUL_THREADS, eul_min_blocks<D>)
k_euler(double *__restrict__ x, double *__restrict__ y, const double *__restrict__ part, int chunks,
        double bscale, int coef_arg, double p0, double p1, double p2, double *__restrict__ ymean, int64_t N,
        int64_t Np, double h, double sqrt_h, int fine_r, double sqrt_hf, uint64_t seed, long long *dstep,
        double *mpart, unsigned *ticket, double *mom, int *err, long long *counters) {
    const int coef = CF >= 0 ? CF : coef_arg;
    const long long n = *dstep;
    constexpr bool GEN = FAM == EUL_GEN, OU = FAM == EUL_OU, MM = FAM != EUL_PAIR;
    static_assert(!S1 || MM, "step 1 is fused only for the linear moment sets");
    // S1: the factor of step 1 and mean(Y) from the moments of X_n (every block reads
    // mom here, before its ticket; the last block overwrites it with the moments of
    // X_{n+1} only after every block has taken one)
    double lin = 1.0, ymd[D];
#pragma unroll
    for (int c = 0; c < D; ++c) ymd[c] = 0.0;
    if (S1) {
        lin = coef == SSM_COEF_POLY ? 1.0 / (1.0 - h * p0 + h * mom[D]) : 1.0 / (1.0 - h * p0);
#pragma unroll
        for (int c = 0; c < D; ++c) ymd[c] = lin * mom[c];
        if (blockIdx.x == 0 && threadIdx.x < D) ymean[threadIdx.x] = ymd[threadIdx.x];
    } else if (MM) {
#pragma unroll
        for (int c = 0; c < D; ++c) ymd[c] = ymean[c];
    }
    // Y of particle i: step 1 here (S1, also stored as the stage Y) or as step 1 left it
    auto load_y = [&](int64_t i, double (&yv)[D]) {
        if (S1) {
            double xv[D];
#pragma unroll
            for (int c = 0; c < D; ++c) xv[c] = x[c * Np + i];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                yv[c] = xv[c] * lin;
                y[c * Np + i] = yv[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) yv[c] = y[c * Np + i];
        }
    };
    // b of particle i from the pair partial sums (pair sets)
    auto pair_drift = [&](int64_t i, int c) -> double {
        double sm = 0.0;
        for (int k = 0; k < chunks; ++k) sm += part[((int64_t)k * D + c) * Np + i];
        return sm * bscale;
    };
    double m[4 * D];
#pragma unroll
    for (int k = 0; k < 4 * D; ++k) m[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (F32) {
        float ymf[D], hb_ou[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            ymf[c] = MM ? (float)ymd[c] : 0.0f;
            hb_ou[c] = OU ? (float)(h * p1 * ymd[c]) : 0.0f;
        }
        const float hf = (float)h, p0f = (float)p0, p1f = (float)p1, p2f = (float)p2;
        const float sqh = (float)sqrt_h, sqhf = (float)sqrt_hf;
        // X' = Y + inc for particle i; returns the FP32 powers 1..4 of X' (4 D values).
        // The loads are issued before the Philox and Box-Muller arithmetic they overlap.
        auto advance = [&](int64_t i, float (&p)[4 * D]) {
            double yv[D];
            float yf[D], hb[D];
            load_y(i, yv);
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (!GEN) hb[c] = OU ? hb_ou[c] : hf * f64_to_f32(pair_drift(i, c));
#pragma unroll
            for (int c = 0; c < D; ++c)   // the d = 1 sets with step 1 in its own kernel: FP64 pipe to spare
                yf[c] = (D == 1 && GEN && !S1) ? (float)yv[c] : f64_to_f32_fast(yv[c]);
            if (GEN)
#pragma unroll
                for (int c = 0; c < D; ++c) hb[c] = hf * moment_b<float>(coef, c, yf, ymf, p0f, p1f);
            float dw[D];
            brownian32<D>(seed, i, n, sqh, fine_r, sqhf, dw);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float sg = GEN ? moment_sigma<float>(coef, c, yf, ymf, p0f, p1f, p2f) : OU ? p2f : sigma_of32(coef, yf[c], p2f);
                const float inc = fmaf(sg, dw[c], hb[c]);
                // at d <= 2 the FP64 pipe has room for the hardware conversion, which
                // frees the integer pipe; at d = 3 (three adds a particle) it does not
                x[c * Np + i] = yv[c] + (D <= 2 ? (double)inc : f32_to_f64(inc));
                const float v = yf[c] + inc, v2 = v * v;
                p[0 * D + c] = v;
                p[1 * D + c] = v2;
                p[2 * D + c] = v2 * v;
                p[3 * D + c] = v2 * v2;
            }
        };
        // the powers are summed in FP32 over 32 particles at a time (error < 32 eps of
        // their absolute sum) and those sums added in FP64 into this thread's slots in
        // shared memory (fewer registers and instructions than a compensated sum per
        // particle)
        __shared__ double msum[4 * D][EUL_THREADS];
        float ms[4 * D];
#pragma unroll
        for (int k = 0; k < 4 * D; ++k) { ms[k] = 0.0f; msum[k][threadIdx.x] = 0.0; }
        int nb = 0;
#pragma unroll 1
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
            float p[4 * D];
            advance(i, p);
#pragma unroll
            for (int k = 0; k < 4 * D; ++k) ms[k] += p[k];
            if (++nb == 32) {
#pragma unroll
                for (int k = 0; k < 4 * D; ++k) { msum[k][threadIdx.x] += (double)ms[k]; ms[k] = 0.0f; }
                nb = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 4 * D; ++k) m[k] = msum[k][threadIdx.x] + (double)ms[k];
    } else {
        double ym[D];
#pragma unroll
        for (int c = 0; c < D; ++c) ym[c] = ymd[c];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
            double yv[D];
            load_y(i, yv);
            double dw[D];
            brownian<D>(seed, i, n, sqrt_h, fine_r, sqrt_hf, dw);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const double b = GEN ? moment_b<double>(coef, c, yv, ym, p0, p1) : OU ? p1 * ym[c] : pair_drift(i, c);
                const double sg = GEN ? moment_sigma<double>(coef, c, yv, ym, p0, p1, p2) : sigma_of(coef, yv[c], p2);
                const double xn = yv[c] + h * b + sg * dw[c];
                x[c * Np + i] = xn;
                add_powers<D>(m, c, xn);
            }
        }
    }
    moments_epilogue<D>(m, N, mpart, ticket, mom, err);
}

// The step index advances in a separate one-thread kernel after k_euler, so no
// block of k_euler can observe the new value.
__global__ void k_advance(long long *dstep, long long *counters, long long N) {
    *dstep += 1;
    counters[CNT_STEPS] += 1;
    counters[CNT_DRIFT_ROWS] += N;
}

__global__ void k_set_step(long long *dstep, long long n) { *dstep = n; }

// Host particle-major <-> device SoA.
__global__ void k_aos_to_soa(const double *__restrict__ a, double *__restrict__ s, int d, int64_t N, int64_t Np) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N * d; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / d;
        const int c = (int)(k - i * d);
        s[c * Np + i] = a[k];
    }
}
__global__ void k_soa_to_aos(const double *__restrict__ s, double *__restrict__ a, int d, int64_t N, int64_t Np) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N * d; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / d;
        const int c = (int)(k - i * d);
        a[k] = s[c * Np + i];
    }
}
// b of the last step, particle-major, from the drift partials.
__global__ void k_stage_b(const double *__restrict__ part, int chunks, double bscale, int coef, double p0, double p1,
                          const double *__restrict__ ymean, const double *__restrict__ y, double *__restrict__ a,
                          int d, int64_t N, int64_t Np) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N * d; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / d;
        const int c = (int)(k - i * d);
        if (is_moment_set(coef)) {
            double yv[3] = {0.0, 0.0, 0.0}, ym[3] = {0.0, 0.0, 0.0};
            for (int e = 0; e < d; ++e) { yv[e] = y[e * Np + i]; ym[e] = ymean[e]; }
            a[k] = moment_b<double>(coef, c, yv, ym, p0, p1);
        } else {
            double s = 0.0;
            for (int q = 0; q < chunks; ++q) s += part[((int64_t)q * d + c) * Np + i];
            a[k] = s * bscale;
        }
    }
}

// Component kernels behind ssm_philox / ssm_normals / ssm_cardano.
__global__ void k_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox10(U4{ ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2], ctr[4 * k + 3] }, (uint32_t)seed,
                              (uint32_t)(seed >> 32));
        out[4 * k] = w.a;
        out[4 * k + 1] = w.b;
        out[4 * k + 2] = w.c;
        out[4 * k + 3] = w.d;
    }
}
template <int D>
__global__ void k_normals(uint64_t seed, int64_t N, uint32_t step, uint32_t stream, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double z[3];
        normals<D>(seed, (uint32_t)i, step, stream, z);
#pragma unroll
        for (int c = 0; c < D; ++c) out[i * D + c] = z[c];
    }
}

template <int D>
__global__ void k_normals32(uint64_t seed, int64_t N, uint32_t step, uint32_t stream, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float z[3];
        normals32<D>(seed, (uint32_t)i, step, stream, z);
#pragma unroll
        for (int c = 0; c < D; ++c) out[i * D + c] = z[c];
    }
}

// ---------------------------------------------------------------------------
// Host launchers (enqueue only).
// ---------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }
static inline unsigned gs_blocks(int64_t n, int th) {   // grid-stride launch size: at most 8 blocks an SM
    const int64_t b = (n + th - 1) / th;
    int sms = device_sms();
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_init_x0(ssm_ctx *c) {
    if (c->d == 1)
        k_init_x0<1><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->seed, c->opt.x0_mean, c->opt.x0_std,
                                                           c->mpart, c->ticket, c->mom, c->err);
    else if (c->d == 2)
        k_init_x0<2><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->seed, c->opt.x0_mean, c->opt.x0_std,
                                                           c->mpart, c->ticket, c->mom, c->err);
    else
        k_init_x0<3><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->seed, c->opt.x0_mean, c->opt.x0_std,
                                                           c->mpart, c->ticket, c->mom, c->err);
    return cudaGetLastError();
}

// X_0 and its moments for arrays outside a context (used by the batched form).
cudaError_t launch_init_x0_raw(int d, double *x, int64_t N, int64_t Np, uint64_t seed, double mean, double sd,
                               double *mpart, unsigned *ticket, double *mom, int *err, cudaStream_t st) {
    if (d == 1) k_init_x0<1><<<RED_BLOCKS, EUL_THREADS, 0, st>>>(x, N, Np, seed, mean, sd, mpart, ticket, mom, err);
    else k_init_x0<3><<<RED_BLOCKS, EUL_THREADS, 0, st>>>(x, N, Np, seed, mean, sd, mpart, ticket, mom, err);
    return cudaGetLastError();
}

cudaError_t launch_moments(ssm_ctx *c) {
    if (c->d == 1) k_moments<1><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->mpart, c->ticket, c->mom, c->err);
    else if (c->d == 2) k_moments<2><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->mpart, c->ticket, c->mom, c->err);
    else k_moments<3><<<RED_BLOCKS, EUL_THREADS, 0, c->st>>>(c->x, c->N, c->Np, c->mpart, c->ticket, c->mom, c->err);
    return cudaGetLastError();
}

cudaError_t launch_cardano(const double *x, double *y, int64_t n, double h, cudaStream_t st) {
    k_cardano<<<gs_blocks(n, 256), 256, 0, st>>>(x, y, n, h);
    return cudaGetLastError();
}

cudaError_t launch_mm_implicit(ssm_ctx *c) {
    const bool f32 = c->prec != SSM_FP64;
    const double p0 = c->opt.coef_params[0], p1 = c->opt.coef_params[1];
#define SSM_MM(D) \
    if (f32) k_mm_implicit<D, true><<<red_grid(c->sms, RED_PER_SM), EUL_THREADS, 0, c->st>>>(c->coef, c->x, c->y, c->N, c->Np, c->h, p0, \
                                                                          p1, c->mom, c->mpart, c->ticket, c->ymean); \
    else k_mm_implicit<D, false><<<red_grid(c->sms, RED_PER_SM), EUL_THREADS, 0, c->st>>>(c->coef, c->x, c->y, c->N, c->Np, c->h, p0, \
                                                                       p1, c->mom, c->mpart, c->ticket, c->ymean);
    if (c->d == 1) { SSM_MM(1) }
    else if (c->d == 2) { SSM_MM(2) }
    else { SSM_MM(3) }
#undef SSM_MM
    return cudaGetLastError();
}

#define D_KIND(d) ((d) == 1 ? PK_NEWTON1 : PK_NEWTON3)
cudaError_t launch_newton_begin(ssm_ctx *c) {
    const int tile = c->plan_newton.threads * c->plan_newton.rpt;
    const DynChunks full = dyn_chunks(c->N, c->N, c->Np, tile, (int)((c->N + tile - 1) / tile), c->plan_newton.chunks,
                                      c->plan_newton.chunk_len, pair_sub(D_KIND(c->d), c->plan_newton.vec2), c->d + 1,
                                      c->part_cap);
    if (c->d == 1)
        k_newton_begin<1><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->act0, c->cnt, c->kmax, c->passes, c->hist,
                                                              c->mom, c->mom_prev, c->N, c->Np, c->dpass,
                                                              c->opt.inject, c->pplan, full);
    else
        k_newton_begin<3><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->act0, c->cnt, c->kmax, c->passes, c->hist,
                                                              c->mom, c->mom_prev, c->N, c->Np, c->dpass,
                                                              c->opt.inject, c->pplan, full);
    return cudaGetLastError();
}

// Update of pass `pass` (hpass == 0), or of the pass *c->dpass inside the step
// graph's device-driven loop whose condition is hpass.
cudaError_t launch_newton_update(ssm_ctx *c, int pass, int fp32, cudaGraphConditionalHandle hpass) {
    const int rp = (c->prec == SSM_FP32C_LEARNED && c->ws_loaded) ? c->opt.ws_passes : -1;
    const int sub = pair_sub(D_KIND(c->d), c->plan_newton.vec2);
#define SSM_UPD1(D, L) k_newton_update<D, L><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->act0, c->act1, \
        c->cnt, c->part, c->pplan, c->plan_newton, sub, c->part_cap, c->N, c->Np, c->h, c->tol, fp32, pass, c->kmax, \
        c->passes, c->hist, c->err, c->sconv, rp, c->counters, c->rprev, c->dpass, c->ticket, hpass)
#define SSM_UPD(D) { if (hpass) SSM_UPD1(D, true); else SSM_UPD1(D, false); }
    if (c->d == 1) SSM_UPD(1)
    else SSM_UPD(3)
#undef SSM_UPD
#undef SSM_UPD1
    return cudaGetLastError();
}

cudaError_t launch_mi_begin(ssm_ctx *c) {
    if (c->d == 1)
        k_mi_begin<1><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->act0, c->cnt, c->mif, c->kmax, c->N, c->Np);
    else
        k_mi_begin<3><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->act0, c->cnt, c->mif, c->kmax, c->N, c->Np);
    return cudaGetLastError();
}

cudaError_t launch_mi_pass(ssm_ctx *c, int pass, int fp32) {
#define SSM_MI(D) \
    k_mi_update<D><<<nblk(c->N, 256), 256, 0, c->st>>>(c->x, c->y, c->stage, c->cnt, c->part, c->plan_newton.chunks, \
                                                       c->N, c->Np, c->h, c->tol, fp32, pass, c->kmax, c->mif, c->rprev, \
                                                       c->err); \
    k_mi_commit<D><<<nblk(c->N, 256), 256, 0, c->st>>>(c->y, c->stage, c->cnt, c->mif, pass, c->kmax, c->N, c->Np, \
                                                       c->h, c->tol, c->err);
    if (c->d == 1) { SSM_MI(1) }
    else { SSM_MI(3) }
#undef SSM_MI
    return cudaGetLastError();
}

cudaError_t launch_step_stats(ssm_ctx *c) {
    // the learned start and the carried start read the converged sums of a completed step
    const bool learned = (c->prec == SSM_FP32C_LEARNED && c->ws_loaded && !c->opt.measure_y) || c->opt.carry_start;
    k_step_stats<<<1, 1, 0, c->st>>>(c->cnt, c->kmax, c->N, c->counters, c->opt.measure_y ? c->mif : nullptr,
                                     learned ? c->ws_prev : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_euler(ssm_ctx *c, double bscale) {
    const int fine_r = c->opt.fine_log2 > 0 ? (int)llround(c->h / (c->T / (double)(1ll << c->opt.fine_log2))) : 1;
    const double sqrt_hf = c->opt.fine_log2 > 0 ? sqrt(c->T / (double)(1ll << c->opt.fine_log2)) : 0.0;
    const int chunks = c->plan_drift.chunks;
    const double p0 = c->opt.coef_params[0], p1 = c->opt.coef_params[1], p2 = c->opt.coef_params[2];
    const bool f32 = c->prec != SSM_FP64;
    // families by dimension: d = 1 pair sets, OU, GL/POLY/GLSTAB; d = 2 OU, CS; d = 3 pair sets, OU
    const int fam = c->coef == SSM_COEF_OU ? EUL_OU : is_moment_set(c->coef) ? EUL_GEN : EUL_PAIR;
    // OU and the polynomial drift: step 1 fused into this kernel (the caller launches
    // no k_mm_implicit for them)
    const bool s1 = fused_step1(c->coef);
#define SSM_EUL(D, F, G, S, CF) k_euler<D, F, G, S, CF><<<red_grid(c->sms, eul_min_blocks<D>), EUL_THREADS, 0, c->st>>>(c->x, c->y, \
        c->part, chunks, bscale, c->coef, p0, p1, p2, c->ymean, c->N, c->Np, c->h, sqrt(c->h), fine_r, sqrt_hf, c->seed, \
        c->dstep, c->mpart, c->ticket, c->mom, c->err, c->counters)
#define SSM_EUL_G(D, G, S, CF) { if (f32) SSM_EUL(D, true, G, S, CF); else SSM_EUL(D, false, G, S, CF); }
    if (c->d == 1) {
        if (fam == EUL_GEN) {
            if (c->coef == SSM_COEF_POLY) SSM_EUL_G(1, EUL_GEN, true, SSM_COEF_POLY)
            else if (c->coef == SSM_COEF_GL1) SSM_EUL_G(1, EUL_GEN, false, SSM_COEF_GL1)
            else if (c->coef == SSM_COEF_GL2) SSM_EUL_G(1, EUL_GEN, false, SSM_COEF_GL2)
            else SSM_EUL_G(1, EUL_GEN, false, -1)   // GLSTAB
        } else if (fam == EUL_OU) SSM_EUL_G(1, EUL_OU, true, -1)
        else SSM_EUL_G(1, EUL_PAIR, false, -1)
    } else if (c->d == 2) {
        if (fam == EUL_GEN) SSM_EUL_G(2, EUL_GEN, false, SSM_COEF_CS) else SSM_EUL_G(2, EUL_OU, true, -1)
    } else {
        if (fam == EUL_OU) SSM_EUL_G(3, EUL_OU, true, -1) else SSM_EUL_G(3, EUL_PAIR, false, -1)
    }
#undef SSM_EUL_G
#undef SSM_EUL
    k_advance<<<1, 1, 0, c->st>>>(c->dstep, c->counters, c->N);
    return cudaGetLastError();
}

cudaError_t launch_set_step(ssm_ctx *c, long long n) {
    k_set_step<<<1, 1, 0, c->st>>>(c->dstep, n);
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double *a, double *s, int d, int64_t N, int64_t Np, cudaStream_t st) {
    k_aos_to_soa<<<gs_blocks(N * d, 256), 256, 0, st>>>(a, s, d, N, Np);
    return cudaGetLastError();
}
cudaError_t launch_soa_to_aos(const double *s, double *a, int d, int64_t N, int64_t Np, cudaStream_t st) {
    k_soa_to_aos<<<gs_blocks(N * d, 256), 256, 0, st>>>(s, a, d, N, Np);
    return cudaGetLastError();
}
cudaError_t launch_stage_b(ssm_ctx *c, double bscale) {
    k_stage_b<<<gs_blocks(c->N * c->d, 256), 256, 0, c->st>>>(c->part, c->plan_drift.chunks, bscale, c->coef,
                                                             c->opt.coef_params[0], c->opt.coef_params[1], c->ymean,
                                                             c->y, c->stage, c->d, c->N, c->Np);
    return cudaGetLastError();
}
cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out, cudaStream_t st) {
    k_philox<<<gs_blocks(n, 256), 256, 0, st>>>(seed, ctr, n, out);
    return cudaGetLastError();
}
cudaError_t launch_normals(uint64_t seed, int d, int64_t N, uint32_t step, uint32_t stream, double *out, cudaStream_t st) {
    if (d == 1) k_normals<1><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    else if (d == 2) k_normals<2><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    else k_normals<3><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    return cudaGetLastError();
}

cudaError_t launch_normals32(uint64_t seed, int d, int64_t N, uint32_t step, uint32_t stream, float *out,
                             cudaStream_t st) {
    if (d == 1) k_normals32<1><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    else if (d == 2) k_normals32<2><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    else k_normals32<3><<<gs_blocks(N, 256), 256, 0, st>>>(seed, N, step, stream, out);
    return cudaGetLastError();
}

SSM_BOUNDS_READER(bounds_hits_particle)

}  // namespace ssm
