"""Pins of the oracle's moment-interaction sets (§3.2 Ginzburg-Landau versions 1
and 2, §3.3 polynomial drift, §3.4 Cucker-Smale) against facts the paper and the
mathematics fix: a high-precision root, the closed-form solution of the
noise-free equation, the step-1 equations as residuals with the measure's mean
computed here, exact recursions of the particle mean, the noise-free flocking
fixed point, and the strong rate 1/2 of Theorem 2.3 on the paper's GL example.
CPU only (no GPU marker).
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import inputs

GL = (1.5, 0.5)          # sigma', c of §3.2
CS = (2.0, 4.0)          # lambda, sigma' of §3.4


def test_gl_root_matches_high_precision_root():
    """Root of y + h y^3 = x (step 1 for v = -x^3) within 2 ulp of a 40-digit root."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for h in (1e-3, 2.0 ** -4, 0.1, 0.9):
        for x in list(inputs.uniform_points(30, -8.0, 8.0, seed=12)) + [0.0, 1e-300, -3e-9, 40.0]:
            y = O.cardano_gl(x, h)
            f = lambda t: mp.mpf(h) * t ** 3 + t - mp.mpf(x)
            lo, hi = mp.mpf(-50), mp.mpf(50)
            for _ in range(1100):
                mid = (lo + hi) / 2
                if f(mid) > 0:
                    hi = mid
                else:
                    lo = mid
            exact = float((lo + hi) / 2)
            assert abs(y - exact) <= 2 * np.spacing(abs(exact)) + 1e-320, (x, h, y, exact)


def test_noise_free_gl_is_backward_euler_of_the_ode():
    """With sigma' = 0 and c = 0 the GL sets reduce to dx/dt = -x^3, whose solution
    from x0 = 1 is 1/sqrt(1 + 2t).  Step 1 is then backward Euler and step 2 the
    identity, so the error at T = 1 halves with h (first order)."""
    exact = 1.0 / math.sqrt(3.0)
    errs = []
    for k in (5, 6, 7, 8):
        h = 2.0 ** -k
        for coef in (O.COEF_GL1, O.COEF_GL2):
            P = O.problem(d=1, coef=coef, N=3, h=h, seed=1, p=(0.0, 0.0), x0_mean=1.0, x0_std=0.0)
            x = O.run(P, O.init_x0(P), 0, 1 << k)
            assert np.all(x == x[0])
            if coef == O.COEF_GL1:
                errs.append(abs(x[0, 0] - exact))
            else:
                assert abs(x[0, 0] - exact) == pytest.approx(errs[-1], rel=1e-12)
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    assert errs[-1] < 2e-3


def test_step1_equations_hold_with_the_mean_of_x():
    """GL2: y + h y^3 = x + h c mean(X); POLY: y = x + h (gamma y - y mean(X^2)).
    The means are taken here from the X array (the frozen measure of step 1)."""
    x = inputs.gaussian_cloud(9, 1, seed=21)
    h = 2.0 ** -3
    P = O.problem(d=1, coef=O.COEF_GL2, N=9, h=h, p=GL)
    y, it, bad = O.implicit_step(P, x)
    assert bad == 0
    r = y + h * y ** 3 - x - h * GL[1] * np.mean(x)
    assert np.max(np.abs(r)) < 1e-14
    ry = y + h * y ** 3 - x - h * GL[1] * np.mean(y)       # the measure at Y would not satisfy it
    assert np.max(np.abs(ry)) > 1e-6
    gamma = -1.0
    P = O.problem(d=1, coef=O.COEF_POLY, N=9, h=h, p=(gamma,))
    y, it, bad = O.implicit_step(P, x)
    r = y - x - h * (gamma * y - y * np.mean(x ** 2))
    assert np.max(np.abs(r)) < 1e-15


@pytest.mark.parametrize("coef", [O.COEF_GL1, O.COEF_GL2, O.COEF_POLY, O.COEF_CS])
def test_particle_mean_follows_exact_recursion(coef):
    """Step 2 is linear in the measure, so the particle mean of X' is fixed by Y and
    the draws: GL1 mean(Y)(1 + h (s^2/2 + c)) + s mean(Y dW); GL2 the same with c
    absent; POLY mean(Y)(1 + h) + mean(Y dW); CS (V) mean(Y_V) + h + s' mean((mean
    Y_V - Y_V) dW_0) and X' = X + h Y_V exactly.  A measure taken at X, a missing
    self term, a 1/(N-1) weight or the wrong sign of the flocking term break it."""
    d = 2 if coef == O.COEF_CS else 1
    p = {O.COEF_GL1: GL, O.COEF_GL2: GL, O.COEF_POLY: (-1.0,), O.COEF_CS: CS}[coef]
    N, h = 40, 2.0 ** -5
    P = O.problem(d=d, coef=coef, N=N, h=h, seed=8, p=p, x0_mean=1.0, x0_std=0.7)
    x = O.init_x0(P)
    for n in range(6):
        y, it, bad = O.implicit_step(P, x)
        assert bad == 0
        x1 = O.explicit_step(P, y, n)
        dw = np.stack([O.brownian(P, i, n) for i in range(N)])
        if coef in (O.COEF_GL1, O.COEF_GL2):
            s, c = p
            kappa = s * s / 2 + (c if coef == O.COEF_GL1 else 0.0)
            pred = np.mean(y) * (1 + h * kappa) + s * np.mean(y[:, 0] * dw[:, 0])
            assert abs(np.mean(x1) - pred) < 1e-13
        elif coef == O.COEF_POLY:
            pred = np.mean(y) * (1 + h) + np.mean(y[:, 0] * dw[:, 0])
            assert abs(np.mean(x1) - pred) < 1e-13
        else:
            lam, s = p
            mv = np.mean(y[:, 0])
            pred = mv + h + s * np.mean((mv - y[:, 0]) * dw[:, 0])
            assert abs(np.mean(x1[:, 0]) - pred) < 1e-13
            assert np.max(np.abs(x1[:, 1] - (x[:, 1] + h * y[:, 0]))) < 1e-15
            b = np.stack([O.drift_one(P, y, i) for i in range(N)])
            assert np.all(b[:, 1] == y[:, 0])
            assert abs(np.sum(b[:, 0] - 1.0)) < 1e-12
        x = x1


def test_noise_free_cucker_smale_reaches_the_flocking_fixed_point():
    """With sigma' = 0 the V part of the scheme maps V to Y + h (1 + lambda (mean Y - Y))
    with Y + h Y^3 = V: its fixed point is Y = 1, V = 1 + h for every particle (the
    flock moves at speed 1, the limit the paper quotes)."""
    lam, h = 2.0, 0.05
    P = O.problem(d=2, coef=O.COEF_CS, N=16, h=h, seed=3, p=(lam, 0.0), x0_mean=1.0, x0_std=math.sqrt(2.0),
                  T=10.0)
    x = O.run(P, O.init_x0(P), 0, 200)
    assert np.max(np.abs(x[:, 0] - (1.0 + h))) < 1e-10
    y, _, _ = O.implicit_step(P, x)
    assert np.max(np.abs(y[:, 0] - 1.0)) < 1e-10


def test_gl_strong_error_decays_at_rate_one_half():
    """The paper's GL example (sigma' = 1.5, c = 0.5, x0 = 1): rMSE at T against an
    h = 2^-11 run on the same Brownian paths decreases with a fitted slope >= 0.4
    (Theorem 2.3 gives 1/2)."""
    N, L = 128, 11
    for coef in (O.COEF_GL1, O.COEF_GL2):
        ref_P = O.problem(d=1, coef=coef, N=N, h=2.0 ** -L, seed=41, p=GL, x0_mean=1.0, x0_std=0.0, fine_log2=L)
        x0 = O.init_x0(ref_P)
        ref = O.run(ref_P, x0, 0, 1 << L)
        hs, errs = [], []
        for k in range(3, 8):
            P = O.problem(d=1, coef=coef, N=N, h=2.0 ** -k, seed=41, p=GL, x0_mean=1.0, x0_std=0.0, fine_log2=L)
            xk = O.run(P, x0, 0, 1 << k)
            hs.append(2.0 ** -k)
            errs.append(math.sqrt(np.mean((xk - ref) ** 2)))
        slope = np.polyfit(np.log2(hs), np.log2(errs), 1)[0]
        assert errs[-1] < errs[0], errs
        assert slope >= 0.4, (coef, slope, errs)
