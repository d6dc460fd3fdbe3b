/*
 * ssm_oracle.c -- plain FP64 CPU oracle of the split-step method (SSM) for
 * McKean-Vlasov SDEs of Chen & dos Reis, "A flexible split-step scheme for
 * solving McKean-Vlasov stochastic differential equations" (arXiv:2105.09688).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (all in IEEE double, no fused multiply-add, sums over
 * particles in index order):
 *
 *   Interacting particle system, §1 Eq. (MV-SDE Propagation): N particles in
 *   R^d, empirical measure mu^N = (1/N) sum_{j=1..N} delta_{X^j} (self term
 *   included, weight 1/N).
 *
 *   SSM, §2.3 (eq. SSTM:scheme 1 and SSTM:scheme 2), uniform grid t_n = n h:
 *     step 1 (implicit):  Y_i = X_i + h v(t_n, Y_i, mu^X_n)      (mu^X frozen)
 *     step 2 (explicit):  X'_i = Y_i + h b(t_n, Y_i, mu^Y_n)
 *                                    + sigma(t_n, Y_i, mu^Y_n) dW_i
 *   with dW_i ~ N(0, h I_d) drawn from Philox4x32-10 (below).
 *
 * Coefficient sets (the paper leaves the workloads' coefficients to the user;
 * these are the ones the hot path is built for):
 *   ORC_COEF_CUBIC1D_GAUSS, d = 1:
 *     v(x) = x - x^3,  b(y, mu) = 0.5 * int (z - y) exp(-(y - z)^2) mu(dz),
 *     sigma(y) = 0.4 y + 0.1.
 *   ORC_COEF_COUPLED3D, d = 3:
 *     v(y, mu) = -y|y|^2 + 0.5 * int (z - y) / (1 + |y - z|^2) mu(dz),
 *     b(y, mu) = int (z - y) exp(-|y - z|^2 / 2) mu(dz),
 *     sigma(y) = diag(0.3 y_k + 0.2).
 *   ORC_COEF_COUPLED1D: the same three formulas at d = 1.
 *   ORC_COEF_OU, any d (componentwise), §3.4.1 Eq. (stablity:OU):
 *     v(x) = rho x,  b(mu) = lambda * int z mu(dz),  sigma = eta.
 *   The moment-interaction examples of §3 (each measure enters through a mean):
 *   ORC_COEF_GL1, d = 1, §3.2 Eq. (MV-GL-SDE-veresion1), p = (sigma', c):
 *     v(x) = -x^3,  b(y, mu) = sigma'^2/2 y + c int z mu(dz),  sigma(y) = sigma' y.
 *   ORC_COEF_GL2, d = 1, §3.2 Eq. (MV-GL-SDE-veresion2), p = (sigma', c):
 *     v(x, mu) = -x^3 + c int z mu(dz),  b(y) = sigma'^2/2 y,  sigma(y) = sigma' y.
 *   ORC_COEF_POLY, d = 1, §3.3 Eq. (poly1), p = (gamma):
 *     v(x, mu) = gamma x - x int z^2 mu(dz),  b(mu) = int z mu(dz),  sigma(y) = y.
 *   ORC_COEF_CS, d = 2, x = (V, X), §3.4 (Cucker-Smale), p = (lambda, sigma'):
 *     v = (-V^3, 0),  b(y, mu) = (1 + lambda int (z - V) mu^V(dz), V),
 *     sigma(y, mu) = diag(sigma' int (z - V) mu^V(dz), 0).
 *     The drift and diffusion integrals are taken with the sign of the paper's
 *     particle system, (lambda/N) sum_j (V_j - V_i): the flocking towards the mean
 *     that the section describes.
 *   ORC_COEF_GLSTAB, d = 1, §3.4.2 Eq. (satblity:MV-GL-SDE), p = (gamma): the
 *     stability example with a linear term gamma x moved from v to b,
 *     v(x) = -(5/2 + gamma) x - x^3/4,  b(y, mu) = int z mu(dz) + gamma y,  sigma(y) = y.
 *
 * The implicit step is solved as follows.
 *   CUBIC1D_GAUSS: h y^3 + (1 - h) y - x = 0 has exactly one real root for
 *     0 < h < 1 (Lemma 4.1 with L_v = 1).  Cardano's formula in a
 *     cancellation-free form, then one Newton correction.
 *   COUPLED3D / COUPLED1D: Newton's method on F(y) = y - x - h v(y, mu^X) with
 *     the exact d x d Jacobian, Gaussian elimination with partial pivoting, step
 *     halving when the residual grows, start y = x.
 *   OU: y = x / (1 - h rho) (Remark 4.3 gives this closed form for v = a x).
 *   GL1, GL2, the V part of CS: y + h y^3 = x (+ h c mean(X) for GL2), one real
 *     root for every h > 0, by the same Cardano form and Newton correction.
 *   POLY: the equation is linear in y: y = x / (1 - h gamma + h mean(X^2)).
 *   GLSTAB: (h/4) y^3 + (1 + h (5/2 + gamma)) y = x, the same Cardano form (one real
 *     root while 1 + h (5/2 + gamma) > 0).
 *   measure_y = 1 (coupled sets): step 1 with mu^Y in place of mu^X, the joint
 *     system G(Y) = 0 in R^{dN}, G_i = Y_i - X_i - h v(Y_i, mu^Y) -- the earlier
 *     implicit scheme that §1 contrasts with the SSM.  Newton's method on the whole
 *     system with its exact dN x dN Jacobian (dense Gaussian elimination with
 *     partial pivoting), step halving when the residual grows, start Y = X;
 *     N d <= 1536.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed mod 2^32, seed >> 32),
 * counter = (particle i, step index, stream, call k).  Each FP64 uniform is
 * u = (k53 + 1) 2^-53 in (0, 1], with k53 the top 53 bits of (w_a << 32 | w_b).
 * Normals by Box-Muller: r = sqrt(-2 ln u1), z0 = r cos(2 pi u2),
 * z1 = r sin(2 pi u2).  d = 1 uses z0 of call 0; d = 3 uses z0, z1 of call 0
 * and z0 of call 1.  Stream 0 draws X_0, stream 1 draws the Brownian
 * increments.  With fine_log2 = L > 0 the Brownian path lives on the grid
 * T 2^-L and a coarse increment is the sum of its fine increments, so runs at
 * different h share one path (§3: every method uses the same Brownian paths).
 */
#include "ssm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    /* Multipliers and Weyl key increments of the Philox-4x32 family (SC'11, Table 2). */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double uniform53(uint32_t a, uint32_t b)
{
    uint64_t w = ((uint64_t)a << 32) | (uint64_t)b;
    uint64_t k = w >> 11;                       /* 53 bits */
    return (double)(k + 1) * (1.0 / 9007199254740992.0); /* 2^-53, u in (0, 1] */
}

/* Two standard normals from one Philox call at counter (i, step, stream, k). */
static void box_muller_pair(uint64_t seed, uint32_t i, uint32_t step, uint32_t stream,
                            uint32_t k, double *z0, double *z1)
{
    uint32_t ctr[4] = { i, step, stream, k };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double u1 = uniform53(w[0], w[1]);
    double u2 = uniform53(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    double a = 2.0 * ORC_PI * u2;
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

void orc_normals(uint64_t seed, int d, int64_t i, int64_t step, int stream, double *z)
{
    double a, b;
    box_muller_pair(seed, (uint32_t)i, (uint32_t)step, (uint32_t)stream, 0u, &a, &b);
    z[0] = a;
    if (d == 1) return;
    z[1] = b;
    box_muller_pair(seed, (uint32_t)i, (uint32_t)step, (uint32_t)stream, 1u, &a, &b);
    z[2] = a;
}

/* Brownian increment dW_n^i (d components) on the step's own grid or as a sum of
 * fine increments of the grid T 2^-fine_log2. */
void orc_brownian(const orc_problem *P, int64_t i, int64_t n, double *dw)
{
    const int d = P->d;
    double z[3];
    for (int c = 0; c < d; ++c) dw[c] = 0.0;
    if (P->fine_log2 <= 0) {
        orc_normals(P->seed, d, i, n, 1, z);
        double sh = sqrt(P->h);
        for (int c = 0; c < d; ++c) dw[c] = sh * z[c];
        return;
    }
    /* r fine steps of length hf per coarse step; requires h = r * hf exactly. */
    double hf = P->T / (double)((int64_t)1 << P->fine_log2);
    int64_t r = (int64_t)llround(P->h / hf);
    double shf = sqrt(hf);
    for (int64_t m = 0; m < r; ++m) {
        orc_normals(P->seed, d, i, n * r + m, 1, z);
        for (int c = 0; c < d; ++c) dw[c] += shf * z[c];
    }
}

/* ------------------------------------------------------------------------ */
/* Coefficients                                                              */
/* ------------------------------------------------------------------------ */

/* (1/N) sum_j y_{j,c}^k over all particles: a plain moment of the empirical measure. */
static double mean_power(const orc_problem *P, const double *y, int c, int k)
{
    double s = 0.0;
    for (int64_t j = 0; j < P->N; ++j) {
        double v = y[(int64_t)P->d * j + c], p = v;
        for (int e = 1; e < k; ++e) p *= v;
        s += p;
    }
    return s / (double)P->N;
}

/* b(y_i, mu^Y); y is the particle-major array of all particles (the support of
 * the empirical measure). */
static void drift_b(const orc_problem *P, const double *y, const double *yi, double *b)
{
    const int d = P->d;
    const int64_t N = P->N;
    if (P->coef == ORC_COEF_GL1) {
        b[0] = P->p[0] * P->p[0] / 2.0 * yi[0] + P->p[1] * mean_power(P, y, 0, 1);
        return;
    }
    if (P->coef == ORC_COEF_GL2) {
        b[0] = P->p[0] * P->p[0] / 2.0 * yi[0];
        return;
    }
    if (P->coef == ORC_COEF_POLY) {
        b[0] = mean_power(P, y, 0, 1);
        return;
    }
    if (P->coef == ORC_COEF_GLSTAB) {
        b[0] = mean_power(P, y, 0, 1) + P->p[0] * yi[0];
        return;
    }
    if (P->coef == ORC_COEF_CS) {
        b[0] = 1.0 + P->p[0] * (mean_power(P, y, 0, 1) - yi[0]);
        b[1] = yi[0];
        return;
    }
    if (P->coef == ORC_COEF_CUBIC1D_GAUSS) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double dz = y[j] - yi[0];
            s += dz * exp(-(dz * dz));
        }
        b[0] = 0.5 * (s / (double)N);
    } else if (P->coef == ORC_COEF_COUPLED3D || P->coef == ORC_COEF_COUPLED1D) {
        double s[3] = { 0.0, 0.0, 0.0 };
        for (int64_t j = 0; j < N; ++j) {
            double dd[3], r2 = 0.0;
            for (int c = 0; c < d; ++c) { dd[c] = y[(int64_t)d * j + c] - yi[c]; r2 += dd[c] * dd[c]; }
            double e = exp(-r2 / 2.0);
            for (int c = 0; c < d; ++c) s[c] += dd[c] * e;
        }
        for (int c = 0; c < d; ++c) b[c] = s[c] / (double)N;
    } else { /* OU: lambda * mean */
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int64_t j = 0; j < N; ++j) s += y[d * j + c];
            b[c] = P->p[1] * (s / (double)N);
        }
    }
}

static void diffusion_times_dw(const orc_problem *P, const double *y, const double *yi, const double *dw,
                               double *out)
{
    const int d = P->d;
    if (P->coef == ORC_COEF_GL1 || P->coef == ORC_COEF_GL2) {
        out[0] = P->p[0] * yi[0] * dw[0];
    } else if (P->coef == ORC_COEF_POLY || P->coef == ORC_COEF_GLSTAB) {
        out[0] = yi[0] * dw[0];
    } else if (P->coef == ORC_COEF_CS) {
        out[0] = P->p[1] * (mean_power(P, y, 0, 1) - yi[0]) * dw[0];
        out[1] = 0.0;
    } else if (P->coef == ORC_COEF_CUBIC1D_GAUSS) {
        out[0] = (0.4 * yi[0] + 0.1) * dw[0];
    } else if (P->coef == ORC_COEF_COUPLED3D || P->coef == ORC_COEF_COUPLED1D) {
        for (int c = 0; c < d; ++c) out[c] = (0.3 * yi[c] + 0.2) * dw[c];
    } else {
        for (int c = 0; c < d; ++c) out[c] = P->p[2] * dw[c];
    }
}

/* Pair part of v for the coupled sets (d = 3 or 1) at the point y against mu^X:
 *   S(y)  = (1/N) sum_j (x_j - y) w_j,  w_j = 1 / (1 + |x_j - y|^2)
 *   JS(y) = dS/dy = (1/N) sum_j ( -w_j I + 2 w_j^2 (x_j - y)(x_j - y)^T ).
 * JS is d x d, row-major. */
static void pair_sum_coupled(const orc_problem *P, const double *x, const double *y,
                             double S[3], double JS[9])
{
    const int64_t N = P->N;
    const int d = P->d;
    double s[3] = { 0, 0, 0 };
    double j9[9] = { 0, 0, 0, 0, 0, 0, 0, 0, 0 };
    for (int64_t j = 0; j < N; ++j) {
        double dd[3] = { 0, 0, 0 }, q = 1.0;
        for (int a = 0; a < d; ++a) dd[a] = x[(int64_t)d * j + a] - y[a];
        for (int a = 0; a < d; ++a) q += dd[a] * dd[a];
        double w = 1.0 / q;
        for (int a = 0; a < d; ++a) {
            s[a] += dd[a] * w;
            for (int c = 0; c < d; ++c)
                j9[d * a + c] += (a == c ? -w : 0.0) + 2.0 * w * w * dd[a] * dd[c];
        }
    }
    for (int a = 0; a < d; ++a) S[a] = s[a] / (double)N;
    if (JS)
        for (int k = 0; k < d * d; ++k) JS[k] = j9[k] / (double)N;
}

/* Residual F(y) = y - x_i - h v(y, mu^X) for the coupled sets, and optionally its
 * Jacobian (d x d, row-major). */
static void coupled_residual(const orc_problem *P, const double *x, const double *xi,
                             const double *y, double F[3], double J[9])
{
    const int d = P->d;
    double S[3], JS[9];
    pair_sum_coupled(P, x, y, S, J ? JS : NULL);
    double r2 = 0.0;
    for (int a = 0; a < d; ++a) r2 += y[a] * y[a];
    for (int a = 0; a < d; ++a) {
        double v = -y[a] * r2 + 0.5 * S[a];
        F[a] = y[a] - xi[a] - P->h * v;
    }
    if (J) {
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c) {
                /* dv_a/dy_c = -(r2 delta_ac + 2 y_a y_c) + 0.5 JS_ac */
                double dv = -((a == c ? r2 : 0.0) + 2.0 * y[a] * y[c]) + 0.5 * JS[d * a + c];
                J[d * a + c] = (a == c ? 1.0 : 0.0) - P->h * dv;
            }
    }
}

/* Solve the d x d system A s = r (d <= 3) by Gaussian elimination with partial pivoting. */
static int solve_small(int d, const double *A_in, const double *r_in, double *s)
{
    double A[3][4];
    for (int a = 0; a < d; ++a) {
        for (int c = 0; c < d; ++c) A[a][c] = A_in[d * a + c];
        A[a][d] = r_in[a];
    }
    for (int col = 0; col < d; ++col) {
        int piv = col;
        for (int row = col + 1; row < d; ++row)
            if (fabs(A[row][col]) > fabs(A[piv][col])) piv = row;
        if (A[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c <= d; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
        for (int row = col + 1; row < d; ++row) {
            double f = A[row][col] / A[col][col];
            for (int c = col; c <= d; ++c) A[row][c] -= f * A[col][c];
        }
    }
    for (int row = d - 1; row >= 0; --row) {
        double acc = A[row][d];
        for (int c = row + 1; c < d; ++c) acc -= A[row][c] * s[c];
        s[row] = acc / A[row][row];
    }
    return 0;
}

static double norminf(int d, const double *v) {
    double m = 0.0;
    for (int c = 0; c < d; ++c)
        if (fabs(v[c]) > m) m = fabs(v[c]);
    return m;
}

/* Cardano root of h y^3 + (1 - h) y - x = 0 (v = y - y^3 in step 1), then one
 * Newton correction.  Depressed cubic y^3 + p y + q = 0 with p = (1-h)/h > 0,
 * q = -x/h; one real root since the discriminant (q/2)^2 + (p/3)^3 > 0.  With
 * y = u + w, u w = -p/3, u^3 + w^3 = -q, the root is written as
 * -q / (u^2 - u w + w^2) = -q / (u^2 + p/3 + w^2): a sum of positive terms, so it
 * loses no digits when q is small. */
static double cardano_root(double x, double h, double a)
{
    /* h y^3 + a y - x = 0 with a > 0, h > 0 */
    if (x == 0.0) return 0.0;
    double p = a / h;
    double q = -x / h;
    double disc = (q / 2.0) * (q / 2.0) + (p / 3.0) * (p / 3.0) * (p / 3.0);
    double sq = sqrt(disc);
    double u = cbrt(fabs(q) / 2.0 + sq);
    if (q > 0.0) u = -u;
    double w = -p / (3.0 * u);
    double y = -q / (u * u + p / 3.0 + w * w);
    double f = h * y * y * y + a * y - x;
    double fp = 3.0 * h * y * y + a;
    return y - f / fp;
}

double orc_cardano_cubic(double x, double h) { return cardano_root(x, h, 1.0 - h); }

/* Root of y + h y^3 = x: step 1 for v = -x^3 (the GL and Cucker-Smale sets). */
double orc_cardano_gl(double x, double h) { return cardano_root(x, h, 1.0); }

/* The implicit map F_h of Lemma 4.1: the root c of c = xi + h v(c, mu^X) for an
 * arbitrary point xi, with mu^X the empirical measure of the array x.  Returns
 * Newton iterations (0 for closed forms), or -1 when Newton did not converge in
 * 50 iterations. */
int orc_implicit_point(const orc_problem *P, const double *x, const double *xi, double *y_out)
{
    const int d = P->d;
    if (P->coef == ORC_COEF_CUBIC1D_GAUSS) {
        y_out[0] = orc_cardano_cubic(xi[0], P->h);
        return 0;
    }
    if (P->coef == ORC_COEF_OU) {
        for (int c = 0; c < d; ++c) y_out[c] = xi[c] / (1.0 - P->h * P->p[0]);
        return 0;
    }
    if (P->coef == ORC_COEF_GL1) {
        y_out[0] = orc_cardano_gl(xi[0], P->h);
        return 0;
    }
    if (P->coef == ORC_COEF_GL2) {
        y_out[0] = orc_cardano_gl(xi[0] + P->h * P->p[1] * mean_power(P, x, 0, 1), P->h);
        return 0;
    }
    if (P->coef == ORC_COEF_POLY) {
        y_out[0] = xi[0] / (1.0 - P->h * P->p[0] + P->h * mean_power(P, x, 0, 2));
        return 0;
    }
    if (P->coef == ORC_COEF_CS) {
        y_out[0] = orc_cardano_gl(xi[0], P->h);
        y_out[1] = xi[1];
        return 0;
    }
    if (P->coef == ORC_COEF_GLSTAB) {
        y_out[0] = cardano_root(xi[0], P->h / 4.0, 1.0 + P->h * (2.5 + P->p[0]));
        return 0;
    }
    /* coupled sets: damped Newton from y = x_i. */
    double y[3] = { 0, 0, 0 };
    for (int a = 0; a < d; ++a) y[a] = xi[a];
    double F[3], J[9], s[3];
    coupled_residual(P, x, xi, y, F, J);
    for (int it = 1; it <= 50; ++it) {
        if (solve_small(d, J, F, s) != 0) return -1;
        double fn = norminf(d, F);
        double lam = 1.0, yt[3] = { 0, 0, 0 }, Ft[3], Jt[9];
        for (int half = 0; half < 40; ++half) {
            for (int a = 0; a < d; ++a) yt[a] = y[a] - lam * s[a];
            coupled_residual(P, x, xi, yt, Ft, Jt);
            if (norminf(d, Ft) <= fn || half == 39) break;
            lam *= 0.5;
        }
        double step = lam * norminf(d, s);
        for (int a = 0; a < d; ++a) { y[a] = yt[a]; F[a] = Ft[a]; }
        memcpy(J, Jt, sizeof J);
        double scale = norminf(d, y) > 1.0 ? norminf(d, y) : 1.0;
        if (step <= 1e-14 * scale) {
            for (int a = 0; a < d; ++a) y_out[a] = y[a];
            return it;
        }
    }
    for (int a = 0; a < d; ++a) y_out[a] = y[a];
    return -1;
}

/* Implicit step for particle i (step 1): y_out[d] = F_h(X_i; mu^X). */
int orc_implicit_one(const orc_problem *P, const double *x, int64_t i, double *y_out)
{
    return orc_implicit_point(P, x, x + (int64_t)P->d * i, y_out);
}

/* Explicit step for particle i (step 2): x_out[d] = X_{n+1}^i given all Y. */
void orc_explicit_one(const orc_problem *P, const double *y, int64_t i, int64_t n, double *x_out)
{
    const int d = P->d;
    const double *yi = y + (int64_t)d * i;
    double b[3], dw[3], sdw[3];
    drift_b(P, y, yi, b);
    orc_brownian(P, i, n, dw);
    diffusion_times_dw(P, y, yi, dw, sdw);
    for (int c = 0; c < d; ++c) x_out[c] = yi[c] + P->h * b[c] + sdw[c];
}

/* Drift b(y_i, mu^Y) for particle i (exposed for component tests). */
void orc_drift_one(const orc_problem *P, const double *y, int64_t i, double *b_out)
{
    drift_b(P, y, y + (int64_t)P->d * i, b_out);
}

/* Pair sum S and its Jacobian JS for COUPLED3D at an arbitrary point y. */
void orc_pair_sum_coupled(const orc_problem *P, const double *x, const double *y,
                          double *S, double *JS)
{
    pair_sum_coupled(P, x, y, S, JS);
}

/* Joint residual G (dN) of step 1 against mu^Y and, optionally, its dense
 * Jacobian J (dN x dN, row-major):
 *   G_i = Y_i - X_i - h (-Y_i |Y_i|^2 + 0.5 S_i),  S_i = (1/N) sum_j (Y_j - Y_i) w_ij,
 *   w_ij = 1 / (1 + |Y_j - Y_i|^2);
 *   dS_i/dY_j = (1/N) (w I - 2 w^2 d d^T)  (j != i),  d = Y_j - Y_i,
 *   dS_i/dY_i = -sum_{j != i} dS_i/dY_j  (the self term is identically zero). */
static void joint_residual(const orc_problem *P, const double *x, const double *y, double *G, double *J)
{
    const int d = P->d;
    const int64_t N = P->N, n = N * d;
    if (J) memset(J, 0, sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < N; ++i) {
        const double *yi = y + d * i;
        double S[3] = { 0, 0, 0 };
        for (int64_t j = 0; j < N; ++j) {
            double dd[3] = { 0, 0, 0 }, q = 1.0;
            for (int a = 0; a < d; ++a) { dd[a] = y[d * j + a] - yi[a]; q += dd[a] * dd[a]; }
            double w = 1.0 / q;
            for (int a = 0; a < d; ++a) S[a] += dd[a] * w;
            if (J && j != i)
                for (int a = 0; a < d; ++a)
                    for (int c = 0; c < d; ++c) {
                        double g = ((a == c ? w : 0.0) - 2.0 * w * w * dd[a] * dd[c]) / (double)N;
                        /* dG_i/dY_j = -h 0.5 dS_i/dY_j, and dS_i/dY_i gets -g */
                        J[(d * i + a) * n + d * j + c] += -P->h * 0.5 * g;
                        J[(d * i + a) * n + d * i + c] -= -P->h * 0.5 * g;
                    }
        }
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) r2 += yi[a] * yi[a];
        for (int a = 0; a < d; ++a) {
            double v = -yi[a] * r2 + 0.5 * S[a] / (double)N;
            G[d * i + a] = yi[a] - x[d * i + a] - P->h * v;
        }
        if (J)
            for (int a = 0; a < d; ++a)
                for (int c = 0; c < d; ++c) {
                    double dv = -((a == c ? r2 : 0.0) + 2.0 * yi[a] * yi[c]);
                    J[(d * i + a) * n + d * i + c] += (a == c ? 1.0 : 0.0) - P->h * dv;
                }
    }
}

/* Dense Gaussian elimination with partial pivoting: A s = r, A n x n (destroyed). */
static int solve_dense(int64_t n, double *A, double *r, double *s)
{
    for (int64_t col = 0; col < n; ++col) {
        int64_t piv = col;
        for (int64_t row = col + 1; row < n; ++row)
            if (fabs(A[row * n + col]) > fabs(A[piv * n + col])) piv = row;
        if (A[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int64_t c = 0; c < n; ++c) { double t = A[col * n + c]; A[col * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int64_t row = col + 1; row < n; ++row) {
            double f = A[row * n + col] / A[col * n + col];
            if (f == 0.0) continue;
            for (int64_t c = col; c < n; ++c) A[row * n + c] -= f * A[col * n + c];
            r[row] -= f * r[col];
        }
    }
    for (int64_t row = n - 1; row >= 0; --row) {
        double acc = r[row];
        for (int64_t c = row + 1; c < n; ++c) acc -= A[row * n + c] * s[c];
        s[row] = acc / A[row * n + row];
    }
    return 0;
}

/* G_i of the joint system at the full state y (any N; for checks at large N). */
void orc_joint_residual_one(const orc_problem *P, const double *x, const double *y, int64_t i, double *g)
{
    const int d = P->d;
    const double *yi = y + (int64_t)d * i;
    double S[3] = { 0, 0, 0 }, r2 = 0.0;
    for (int64_t j = 0; j < P->N; ++j) {
        double dd[3] = { 0, 0, 0 }, q = 1.0;
        for (int a = 0; a < d; ++a) { dd[a] = y[(int64_t)d * j + a] - yi[a]; q += dd[a] * dd[a]; }
        for (int a = 0; a < d; ++a) S[a] += dd[a] / q;
    }
    for (int a = 0; a < d; ++a) r2 += yi[a] * yi[a];
    for (int a = 0; a < d; ++a)
        g[a] = yi[a] - x[(int64_t)d * i + a] - P->h * (-yi[a] * r2 + 0.5 * S[a] / (double)P->N);
}

/* Step 1 against mu^Y: Newton on G(Y) = 0 from Y = X.  Returns the iterations, or
 * -1 when it did not converge in 50 (or N d is beyond the dense limit). */
static int joint_implicit_step(const orc_problem *P, const double *x, double *y)
{
    const int64_t n = P->N * (int64_t)P->d;
    if (n > 1536) return -1;
    double *G = (double *)malloc(sizeof(double) * (size_t)n), *Gt = (double *)malloc(sizeof(double) * (size_t)n);
    double *J = (double *)malloc(sizeof(double) * (size_t)(n * n)), *s = (double *)malloc(sizeof(double) * (size_t)n);
    double *yt = (double *)malloc(sizeof(double) * (size_t)n);
    int result = -1;
    memcpy(y, x, sizeof(double) * (size_t)n);
    joint_residual(P, x, y, G, J);
    for (int it = 1; it <= 50; ++it) {
        double fn = 0.0, ymax = 0.0;
        for (int64_t k = 0; k < n; ++k) fn = fabs(G[k]) > fn ? fabs(G[k]) : fn;
        memcpy(Gt, G, sizeof(double) * (size_t)n);
        if (solve_dense(n, J, Gt, s) != 0) break;
        double lam = 1.0, gn = 0.0;
        for (int half = 0; half < 40; ++half) {
            for (int64_t k = 0; k < n; ++k) yt[k] = y[k] - lam * s[k];
            joint_residual(P, x, yt, Gt, NULL);
            gn = 0.0;
            for (int64_t k = 0; k < n; ++k) gn = fabs(Gt[k]) > gn ? fabs(Gt[k]) : gn;
            if (gn <= fn || half == 39) break;
            lam *= 0.5;
        }
        double step = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            step = fabs(lam * s[k]) > step ? fabs(lam * s[k]) : step;
            y[k] = yt[k];
            ymax = fabs(y[k]) > ymax ? fabs(y[k]) : ymax;
        }
        joint_residual(P, x, y, G, J);
        if (step <= 1e-14 * (ymax > 1.0 ? ymax : 1.0)) { result = it; break; }
    }
    free(G); free(Gt); free(J); free(s); free(yt);
    return result;
}

int orc_implicit_step(const orc_problem *P, const double *x, double *y, int *iters)
{
    if (P->measure_y && (P->coef == ORC_COEF_COUPLED3D || P->coef == ORC_COEF_COUPLED1D)) {
        int it = joint_implicit_step(P, x, y);
        if (iters)
            for (int64_t i = 0; i < P->N; ++i) iters[i] = it;
        return it < 0 ? (int)P->N : 0;
    }
    const int64_t N = P->N;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int64_t i = 0; i < N; ++i) {
        int it = orc_implicit_one(P, x, i, y + (int64_t)P->d * i);
        if (iters) iters[i] = it;
        if (it < 0) bad += 1;
    }
    return bad;
}

void orc_explicit_step(const orc_problem *P, const double *y, int64_t n, double *xnext)
{
    const int64_t N = P->N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i)
        orc_explicit_one(P, y, i, n, xnext + (int64_t)P->d * i);
}

/* One SSM step restricted to the target particles idx[0..n-1], used to time a
 * bounded sample of a step: Y_i = F_h(X_i; mu^X) against all N particles,
 * written into y (an N*d array the caller fills with the measure step 2 uses
 * for the particles outside the sample), then X'_i into xout[d*k]. */
void orc_sample_step(const orc_problem *P, const double *x, double *y, const int64_t *idx, int64_t n,
                     int64_t step, double *xout)
{
    const int d = P->d;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; ++k)
        orc_implicit_one(P, x, idx[k], y + (int64_t)d * idx[k]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; ++k)
        orc_explicit_one(P, y, idx[k], step, xout + (int64_t)d * k);
}

/* X_0^i = x0_mean + x0_std * Z^i, Z from stream 0 at step index 0. */
void orc_init_x0(const orc_problem *P, double *x)
{
    const int d = P->d;
    for (int64_t i = 0; i < P->N; ++i) {
        double z[3];
        orc_normals(P->seed, d, i, 0, 0, z);
        for (int c = 0; c < d; ++c) x[(int64_t)d * i + c] = P->x0_mean + P->x0_std * z[c];
    }
}

/* Raw empirical moments m[k][c] = (1/N) sum_i x_{i,c}^(k+1), k = 0..3. */
void orc_moments(const orc_problem *P, const double *x, double *m)
{
    const int d = P->d;
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int64_t i = 0; i < P->N; ++i) {
                double v = x[(int64_t)d * i + c], p = v;
                for (int e = 0; e < k; ++e) p *= v;
                s += p;
            }
            m[k * d + c] = s / (double)P->N;
        }
}

/* Advance x (particle-major, N*d) from step n0 through nsteps SSM steps.  If
 * mom != NULL it receives the moments of X_{n0+s+1} for s = 0..nsteps-1
 * ([nsteps][4][d]).  Returns the number of failed implicit solves. */
int orc_run(const orc_problem *P, double *x, int64_t n0, int64_t nsteps, double *mom,
            int64_t *newton_iters_total)
{
    const int64_t nd = P->N * (int64_t)P->d;
    double *y = (double *)malloc(sizeof(double) * (size_t)nd);
    int *it = (int *)malloc(sizeof(int) * (size_t)P->N);
    int bad = 0;
    int64_t total = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        bad += orc_implicit_step(P, x, y, it);
        for (int64_t i = 0; i < P->N; ++i) total += it[i] > 0 ? it[i] : 0;
        orc_explicit_step(P, y, n0 + s, x);
        if (mom) orc_moments(P, x, mom + s * 4 * P->d);
    }
    if (newton_iters_total) *newton_iters_total = total;
    free(y);
    free(it);
    return bad;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}
