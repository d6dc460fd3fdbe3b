// particle_ops.cuh -- per-particle device code of the SSM step shared by the
// single-context kernels (k_particle.cu) and the batched kernels (batch.cu).
// References: Chen & dos Reis, arXiv:2105.09688, §2.3 (eq. SSTM:scheme 1 and 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssm_device.cuh"

namespace ssm {

// Outcome of one update of step 1 for a particle.
// UPD_FLOOR: accepted at the FP32 evaluation floor of the residual (above tol, see
// below); Y and S stay as for UPD_CONVERGED.
enum : int { UPD_CONVERGED = 0, UPD_CONTINUE = 1, UPD_RESTART = 2, UPD_NOCONV = 3, UPD_NONFINITE = 4,
             UPD_FLOOR = 5 };

// Step 1 of the coupled set, v(y, mu) = -y|y|^2 + 0.5 S(y), for one particle after
// a pair pass: S[D] = (1/N) sum_j (X_j - fl(Y)) w_j and Sw = (1/N) sum_j w_j were
// evaluated at the current Y (fl = FP32 rounding when fp32_targets, exact
// otherwise).  Forms the FP64 residual r = Y - X - h v(Y); if max|r| <= tol the
// particle is done (Y and S stay).  Otherwise Y moves to the root of
// the local model u = X + h(-u|u|^2 + 0.5(S - Sw (u - Y))): the cubic part exact,
// the pair part linearised with the diagonal -Sw I of its Jacobian.  The local
// Jacobian a I + 2h u u^T (a = 1 + h|u|^2 + 0.5 h Sw) is inverted by
// Sherman-Morrison; Newton on the local model converges to rounding in a few steps.
// If a bound on the residual at that root is within tol, the particle is done
// there (UPD_CONVERGED with Y moved): the pass that would only have verified it
// is saved.
//
// FP32 pair sums can only certify the residual down to their evaluation floor
// (rounding of the pair terms and of the FP32 target), which at large h or small
// N may lie above tol.  A pass normally cuts the residual by ~10^3; when it no
// longer cuts it tenfold and the residual is within 64 tol, the iteration has
// reached that floor and the particle is accepted (rprev holds the previous
// pass's residual of this particle); the outcome is then UPD_FLOOR, which the
// kernels count (ssm_stats_t.floor_accepts).
// Root u of the local model u = X + h(-u|u|^2 + 0.5(S - Sw (u - Y))) by Newton with
// the Sherman-Morrison inverse of a I + 2h u u^T (a = 1 + h|u|^2 + 0.5 h Sw).
template <int D>
__device__ __forceinline__ void local_root(const double *S, double Sw, const double *Y, const double *X, double h,
                                           double *u) {
#pragma unroll
    for (int c = 0; c < D; ++c) u[c] = Y[c];
    for (int it = 0; it < 30; ++it) {
        double uu = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) uu += u[c] * u[c];
        double g[D], ug = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            g[c] = u[c] - X[c] + h * u[c] * uu - 0.5 * h * S[c] + 0.5 * h * Sw * (u[c] - Y[c]);
            ug += u[c] * g[c];
        }
        // Sherman-Morrison with both reciprocals from one division: 1/a = b/(ab),
        // 1/b = a/(ab), b = a + 2h|u|^2 (an FP64 division is a long sequence on
        // the FP64 pipe, the slow pipe of this part)
        const double a = 1.0 + h * uu + 0.5 * h * Sw;
        const double b = a + 2.0 * h * uu;
        const double r = 1.0 / (a * b);
        const double ia = b * r, f = 2.0 * h * ug * (a * r);
        double smax = 0.0, umax = 1.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double s = (g[c] - f * u[c]) * ia;
            u[c] -= s;
            smax = fmax(smax, fabs(s));
            umax = fmax(umax, fabs(u[c]));
        }
        if (smax <= 1e-16 * umax) break;
    }
}

template <int D>
__device__ __forceinline__ int newton_update_particle(double *S, double Sw, double *Y, const double *X, double h,
                                                      double tol, bool fp32_targets, int pass, int kmax,
                                                      int restart_pass, float *rprev) {
    if (fp32_targets)   // numerators were taken at fl(Y): (x_j - Y) = (x_j - fl(Y)) - (Y - fl(Y))
#pragma unroll
        for (int c = 0; c < D; ++c) S[c] -= (Y[c] - (double)(float)Y[c]) * Sw;
    double yy = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) yy += Y[c] * Y[c];
    double rinf = 0.0;
    bool bad = !(yy < 1e300);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double r = Y[c] - X[c] - h * (-Y[c] * yy + 0.5 * S[c]);
        if (!(r == r)) bad = true;
        rinf = fmax(rinf, fabs(r));
    }
    if (bad) return UPD_NONFINITE;
    if (rinf <= tol) return UPD_CONVERGED;
    if (fp32_targets && pass > 0 && rinf <= 64.0 * tol && rinf > 0.1 * (double)*rprev) return UPD_FLOOR;
    *rprev = (float)rinf;
    double u[D];
    local_root<D>(S, Sw, Y, X, h, u);
    // Residual bound at u without another pair pass.  G(u) = 0 is the local model;
    // r(u) - G(u) = -h/2 (S(u) - S(Y) + Sw (u - Y)), and by the mean value theorem
    // |S(u) - S(Y) + Sw (u - Y)| <= (max_z ||2 M2(z)|| + |grad Sw| |u - Y|) |u - Y|
    // over z on the segment from Y to u, with M2 = (1/N) sum_j w_j^2 d_j d_j^T and
    // |grad Sw| <= 2 max_r r/(1+r^2)^2 < 0.65.  M2 is positive semidefinite, so
    // ||2 M2|| <= 2 tr M2 = (2/N) sum_j w_j^2 |d_j|^2 = (2/N) sum_j w_j (1 - w_j)
    // (w |d|^2 = 1 - w), and (1/N) sum_j w_j^2 >= Sw^2 (Cauchy-Schwarz), so
    // ||2 M2|| <= 2 Sw (1 - Sw) <= 1/2: small where the sum is dominated by near
    // (Sw -> 1) or by far (Sw -> 0) sources.  Along the segment Sw moves by at most
    // 0.65 |u - Y| and s (1 - s) has slope at most 1, hence m2 below (1e-6 covers the
    // rounding of the FP32 pair sum and its FP32 target).  When the bound is within
    // tol the particle is done at u (S is moved to u to first order for the record).
    double uu = 0.0, du2 = 0.0, ginf = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) uu += u[c] * u[c];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double du = u[c] - Y[c];
        const double g = u[c] - X[c] + h * u[c] * uu - 0.5 * h * S[c] + 0.5 * h * Sw * du;
        ginf = fmax(ginf, fabs(g));
        du2 += du * du;
    }
    const double dn = sqrt(du2);
    const double m2 = fmin(0.5, 2.0 * Sw * (1.0 - Sw) + 1.3 * dn + 1e-6);
    const double bound = 0.5 * h * (m2 + 0.65 * dn) * dn + ginf;
    if (bound <= tol) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            S[c] -= Sw * (u[c] - Y[c]);
            Y[c] = u[c];
        }
        return UPD_CONVERGED;
    }
    if (pass + 1 >= kmax) return UPD_NOCONV;
    if (pass + 1 == restart_pass) {
#pragma unroll
        for (int c = 0; c < D; ++c) Y[c] = X[c];
        return UPD_RESTART;
    }
#pragma unroll
    for (int c = 0; c < D; ++c) Y[c] = u[c];
    return UPD_CONTINUE;
}

// A start of step 1 from a pair sum S (predicted, or carried from the previous step):
// Y^0 = X + delta with delta the root of
// delta = h(-(X + delta)|X + delta|^2 + 0.5 S), by Newton in FP32 on delta (the
// Jacobian a I + 2h u u^T, u = X + delta, inverted by Sherman-Morrison with one
// reciprocal for 1/a and 1/(a + 2h|u|^2)); FP32 on the small increment is far more
// accurate than the start needs (the prediction itself is good to ~1e-6), and the FP64
// state keeps X exact.  A non-finite result leaves the plain start Y = X.
template <int D>
__device__ __forceinline__ void cubic_start(const double (&X)[D], const float (&S)[D], double h, double *yi,
                                            int64_t Np) {
    const float hf = (float)h;
    float xf[D], s2[D], dl[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { xf[c] = f64_to_f32_fast(X[c]); s2[c] = 0.5f * hf * S[c]; dl[c] = 0.0f; }
    for (int it = 0; it < 10; ++it) {
        float u[D], g[D], uu = 0.0f, ug = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) { u[c] = xf[c] + dl[c]; uu += u[c] * u[c]; }
#pragma unroll
        for (int c = 0; c < D; ++c) { g[c] = dl[c] + hf * u[c] * uu - s2[c]; ug += u[c] * g[c]; }
        const float a = 1.0f + hf * uu, b = a + 2.0f * hf * uu;
        const float r = 1.0f / (a * b);
        const float ia = b * r, f = 2.0f * hf * ug * (a * r);
        float smax = 0.0f, dmax = 0.0f;
        bool fin = true;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float st = (g[c] - f * u[c]) * ia;
            dl[c] -= st;
            smax = fmaxf(smax, fabsf(st));
            dmax = fmaxf(dmax, fabsf(dl[c]));
            fin = fin && isfinite(dl[c]);
        }
        if (!fin) return;   // a non-finite result leaves the plain start
        if (smax <= 1e-7f * dmax) break;
    }
#pragma unroll
    for (int c = 0; c < D; ++c) yi[c * Np] = X[c] + f32_to_f64(dl[c]);
}

// Brownian increment dW_n^i on the step's own grid (fine_r <= 1) or as the sum of
// fine_r increments of the finer grid (runs at different h share one path).
template <int D>
__device__ __forceinline__ void brownian(uint64_t seed, int64_t i, long long n, double sqrt_h, int fine_r,
                                         double sqrt_hf, double *dw) {
    if (fine_r <= 1) {
        double z[3];
        normals<D>(seed, (uint32_t)i, (uint32_t)n, 1u, z);
#pragma unroll
        for (int c = 0; c < D; ++c) dw[c] = sqrt_h * z[c];
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) dw[c] = 0.0;
        for (int r = 0; r < fine_r; ++r) {
            double z[3];
            normals<D>(seed, (uint32_t)i, (uint32_t)(n * fine_r + r), 1u, z);
#pragma unroll
            for (int c = 0; c < D; ++c) dw[c] += sqrt_hf * z[c];
        }
    }
}

// The same increments in FP32 (FP32C forms).
template <int D>
__device__ __forceinline__ void brownian32(uint64_t seed, int64_t i, long long n, float sqrt_h, int fine_r,
                                           float sqrt_hf, float *dw) {
    if (fine_r <= 1) {
        float z[3];
        normals32<D>(seed, (uint32_t)i, (uint32_t)n, 1u, z);
#pragma unroll
        for (int c = 0; c < D; ++c) dw[c] = sqrt_h * z[c];
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) dw[c] = 0.0f;
        for (int r = 0; r < fine_r; ++r) {
            float z[3];
            normals32<D>(seed, (uint32_t)i, (uint32_t)(n * fine_r + r), 1u, z);
#pragma unroll
            for (int c = 0; c < D; ++c) dw[c] = fmaf(sqrt_hf, z[c], dw[c]);
        }
    }
}

// Step-2 coefficients of the sets whose measure enters through means (OU and the
// examples of §3.2-3.4), component c at Y = y[0..d-1], with m = mean(Y) per
// component and p = the set's parameters:
//   OU   (§3.4.1): b = lambda m,                 sigma = eta         (p = rho, lambda, eta)
//   GL1  (§3.2 v1): b = s^2/2 y + c m,           sigma = s y          (p = s, c)
//   GL2  (§3.2 v2): b = s^2/2 y,                 sigma = s y
//   POLY (§3.3):    b = m,                        sigma = y           (p = gamma)
//   CS   (§3.4, y = (V, X)): b = (1 + lambda (m_V - V), V), sigma = diag(s (m_V - V), 0)
//                                                                     (p = lambda, s)
//   GLSTAB (§3.4.2): b = m + gamma y,            sigma = y            (p = gamma)
// (CS with the sign of the paper's particle system, which flocks to the mean.)
__host__ __device__ inline bool is_moment_set(int coef) {
    return coef == SSM_COEF_OU || coef == SSM_COEF_GL1 || coef == SSM_COEF_GL2 || coef == SSM_COEF_POLY ||
           coef == SSM_COEF_CS || coef == SSM_COEF_GLSTAB;
}
template <typename T>
__device__ __forceinline__ T moment_b(int coef, int c, const T *y, const T *m, T p0, T p1) {
    switch (coef) {
    case SSM_COEF_GL1: return p0 * p0 / T(2) * y[0] + p1 * m[0];
    case SSM_COEF_GL2: return p0 * p0 / T(2) * y[0];
    case SSM_COEF_POLY: return m[0];
    case SSM_COEF_CS: return c == 0 ? T(1) + p0 * (m[0] - y[0]) : y[0];
    case SSM_COEF_GLSTAB: return m[0] + p0 * y[0];
    default: return p1 * m[c];   // OU
    }
}
template <typename T>
__device__ __forceinline__ T moment_sigma(int coef, int c, const T *y, const T *m, T p0, T p1, T p2) {
    switch (coef) {
    case SSM_COEF_GL1:
    case SSM_COEF_GL2: return p0 * y[0];
    case SSM_COEF_POLY:
    case SSM_COEF_GLSTAB: return y[0];
    case SSM_COEF_CS: return c == 0 ? p1 * (m[0] - y[0]) : T(0);
    default: return p2;   // OU
    }
}

// Diffusion coefficient of each coefficient set, evaluated at Y (step 2).
__device__ __forceinline__ double sigma_of(int coef, double y, double eta) {
    if (coef == SSM_COEF_CUBIC1D_GAUSS) return 0.4 * y + 0.1;
    if (coef == SSM_COEF_COUPLED3D || coef == SSM_COEF_COUPLED1D) return 0.3 * y + 0.2;
    return eta;
}

__device__ __forceinline__ float sigma_of32(int coef, float y, float eta) {
    if (coef == SSM_COEF_CUBIC1D_GAUSS) return fmaf(0.4f, y, 0.1f);
    if (coef == SSM_COEF_COUPLED3D || coef == SSM_COEF_COUPLED1D) return fmaf(0.3f, y, 0.2f);
    return eta;
}

// Powers 1..4 of v accumulated in compensated FP32 (hi + lo per moment).
template <int D>
__device__ __forceinline__ void add_powers32(float (&hi)[4 * D], float (&lo)[4 * D], int c, float v) {
    const float v2 = v * v;
    two_sum_acc(hi[0 * D + c], lo[0 * D + c], v);
    two_sum_acc(hi[1 * D + c], lo[1 * D + c], v2);
    two_sum_acc(hi[2 * D + c], lo[2 * D + c], v2 * v);
    two_sum_acc(hi[3 * D + c], lo[3 * D + c], v2 * v2);
}

template <int D>
__device__ __forceinline__ void add_powers(double (&m)[4 * D], int c, double v) {
    const double v2 = v * v;
    m[0 * D + c] += v;
    m[1 * D + c] += v2;
    m[2 * D + c] += v2 * v;
    m[3 * D + c] += v2 * v2;
}

}  // namespace ssm
