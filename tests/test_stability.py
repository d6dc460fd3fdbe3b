"""The mean-square stability constant beta (the stability theorem of §2, eq.
(SSTM:beta formula)) against what the paper derives from it: the OU step-size
threshold of §3.4.1, the sign of beta across gamma in the Ginzburg-Landau example
of §3.4.2 at h = 0.1, and the theorem's sufficient condition for beta < 0 at small
h.  Host arithmetic only (no GPU marker).  Also the oracle's GL stability set:
its step-1 root at 40 digits and the exact recursion of the particle mean.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs


@pytest.fixture(scope="module")
def S():
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


def test_ou_threshold(S):
    """§3.4.1: beta < 0 exactly when h < -(2 rho + 2 lambda + 1) / lambda^2."""
    from paper_2105_09688_gb300 import stability as st
    for rho, lam in [(-2.0, 0.5), (-3.0, 1.0), (-1.5, 0.25)]:
        hstar = -(2 * rho + 2 * lam + 1) / lam ** 2
        L = st.ou_constants(rho, lam)
        assert st.beta(hstar * 0.999, **L) < 0 < st.beta(hstar * 1.001, **L)
        assert abs(st.beta(hstar, **L)) < 1e-12


def test_ginzburg_landau_example_signs(S):
    """§3.4.2 at h = 0.1: gamma = 0 contracts (beta < 0); for gamma >= 5 the paper
    finds 1 + beta h above 1 (beta > 0); at gamma = -12 the step lies outside the
    theorem's choice of h, and 1 + beta h is not even positive."""
    from paper_2105_09688_gb300 import stability as st
    h = 0.1
    assert st.beta(h, **st.glstab_constants(0.0)) < 0
    for g in (5.0, 8.0, 12.0):
        assert st.beta(h, **st.glstab_constants(g)) > 0
    L = st.glstab_constants(-12.0)
    assert 1.0 - h * (2 * L["Lv"] + 1) < 0
    assert 1.0 + st.beta(h, **L) * h < 0


def test_sufficient_condition_for_contraction(S):
    """L_v < -(1 + L_vt + A)/2 gives beta < 0 for small h; above it beta > 0."""
    from paper_2105_09688_gb300 import stability as st
    rng = np.random.default_rng(9)
    for _ in range(200):
        Lvt, Lb, Lbt, Ls, Lst = rng.uniform(0, 2, 5)
        A = 2 * np.sqrt(Lb) + 2 * np.sqrt(Lbt) + Ls + Lst
        edge = -(1 + Lvt + A) / 2
        assert st.beta(1e-9, edge - 0.1, Lvt, Lb, Lbt, Ls, Lst) < 0
        assert st.beta(1e-9, edge + 0.1, Lvt, Lb, Lbt, Ls, Lst) > 0


def test_beta_rejects_bad_constants(S):
    with pytest.raises(S.SSMError):
        S.ssm_stability_beta(-1.0, -0.1, 0, 0, 0, 0, 0.1)
    with pytest.raises(S.SSMError):
        S.ssm_stability_beta(-1.0, 0, 0, 0, 0, 0, 0.0)
    with pytest.raises(S.SSMError):
        S.ssm_stability_beta(0.5, 0, 0, 0, 0, 0, 0.5)      # 1 - h (2 L_v + 1) = 0


def test_glstab_root_matches_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for gamma, h in [(0.0, 0.1), (12.0, 0.1), (-12.0, 0.1), (-2.0, 0.01)]:
        x = inputs.uniform_points(12, -20.0, 20.0, seed=14)
        P = O.problem(d=1, coef=O.COEF_GLSTAB, N=x.size, h=h, p=(gamma,))
        y, _, bad = O.implicit_step(P, x.reshape(-1, 1))
        a = 1 + mp.mpf(h) * (mp.mpf(5) / 2 + mp.mpf(gamma))
        for xv, yv in zip(x, y[:, 0]):
            f = lambda t: mp.mpf(h) / 4 * t ** 3 + a * t - mp.mpf(float(xv))
            lo, hi = mp.mpf(-100), mp.mpf(100)
            for _ in range(1100):
                mid = (lo + hi) / 2
                if f(mid) > 0:
                    hi = mid
                else:
                    lo = mid
            exact = float((lo + hi) / 2)
            assert abs(yv - exact) <= 2 * np.spacing(abs(exact)) + 1e-320


def test_glstab_particle_mean_recursion():
    """mean(X') = mean(Y) (1 + h (1 + gamma)) + mean(Y dW) exactly (b = mean + gamma y,
    sigma = y)."""
    N, h = 50, 0.05
    for gamma in (0.0, 5.0, -3.0):
        P = O.problem(d=1, coef=O.COEF_GLSTAB, N=N, h=h, seed=5, p=(gamma,), x0_mean=1.0, x0_std=0.8)
        x = O.init_x0(P)
        for n in range(4):
            y, _, bad = O.implicit_step(P, x)
            x1 = O.explicit_step(P, y, n)
            dw = np.array([O.brownian(P, i, n)[0] for i in range(N)])
            pred = np.mean(y) * (1 + h * (1 + gamma)) + np.mean(y[:, 0] * dw)
            assert abs(np.mean(x1) - pred) < 1e-13
            x = x1


def test_oracle_contraction_within_the_theorems_bound(S):
    """The stability theorem of §2 on the oracle itself: two GLSTAB runs (gamma = 0,
    h = 0.01, where 1 - h (2 L_v + 1) > 0 and beta < 0) from X_0 = 1 and Z_0 = 5 driven
    by the same Brownian paths (same seed) satisfy
    (1/N) sum_i |X_n^i - Z_n^i|^2 <= (1 + beta h)^n |1 - 5|^2 at every step n.  The
    theorem's beta is conservative (observed factor 0.960 a step against 0.990), so
    this catches a split whose drift expands, not a small error in its constants."""
    N, h, T = 400, 0.01, 2.0
    k = dict(Lv=-2.5, Lvt=0.0, Lb=0.0, Lbt=1.0, Ls=1.0, Lst=0.0)   # §3.4.2 at gamma = 0
    beta = S.ssm_stability_beta(k["Lv"], k["Lvt"], k["Lb"], k["Lbt"], k["Ls"], k["Lst"], h)
    assert beta < 0
    PX = O.problem(d=1, coef=O.COEF_GLSTAB, N=N, h=h, T=T, seed=86, p=(0.0,), x0_mean=1.0, x0_std=0.0)
    PZ = O.problem(d=1, coef=O.COEF_GLSTAB, N=N, h=h, T=T, seed=86, p=(0.0,), x0_mean=5.0, x0_std=0.0)
    x, z = O.init_x0(PX), O.init_x0(PZ)
    for n in range(1, int(round(T / h)) + 1):
        x, z = O.run(PX, x, n - 1, 1), O.run(PZ, z, n - 1, 1)
        assert np.mean((x - z) ** 2) <= (1 + beta * h) ** n * 16.0 * (1 + 1e-12), n
