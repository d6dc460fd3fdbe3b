"""The Ginzburg-Landau stability example (§3.4.2) on the GPU: against the oracle,
the mean-square contraction bound of the stability theorem of §2 on two runs driven
by the same noise, and the decay of E|X_t|^2 the paper shows for gamma = 0."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.mark.parametrize("gamma", [0.0, 12.0, -2.0])
def test_fp64_matches_oracle(S, gamma):
    N, h = 1000, 0.01
    s = S.SSM(d=1, N=N, h=h, T=1.0, coef=S.SSM_COEF_GLSTAB, seed=81, coef_params=(gamma,), x0_mean=1.0, x0_std=0.0)
    s.run()
    x, n = s.get_state()
    s.close()
    P = O.problem(d=1, coef=O.COEF_GLSTAB, N=N, h=h, seed=81, p=(gamma,), x0_mean=1.0, x0_std=0.0)
    assert n == 100 and relerr(x, O.run(P, O.init_x0(P), 0, 100)) < 1e-10


def test_fp32c_matches_oracle(S):
    N, h = 1000, 0.01
    s = S.SSM(d=1, N=N, h=h, T=1.0, coef=S.SSM_COEF_GLSTAB, seed=82, precision=S.SSM_FP32C, coef_params=(0.0,),
              x0_mean=1.0, x0_std=0.0)
    s.run()
    x, _ = s.get_state()
    m = s.moments()
    s.close()
    P = O.problem(d=1, coef=O.COEF_GLSTAB, N=N, h=h, seed=82, p=(0.0,), x0_mean=1.0, x0_std=0.0)
    xo = O.run(P, O.init_x0(P), 0, 100)
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert abs(m[0, 0] - mo[0, 0]) < 1e-5 and abs((m[1, 0] - m[0, 0] ** 2) - (mo[1, 0] - mo[0, 0] ** 2)) < 1e-5


def test_contraction_within_the_theorems_bound(S):
    """X_0 = 1 and Z_0 = 5 on the same Brownian paths, gamma = 0, h = 0.01, T = 3:
    the particle average of |X_n - Z_n|^2 stays below (1 + beta h)^n |1 - 5|^2."""
    from paper_2105_09688_gb300 import stability as st
    h, T = 0.01, 3.0
    b = st.beta(h, **st.glstab_constants(0.0))
    assert b < 0
    t, d2 = st.contraction_curve(0.0, h, T, 1.0, 5.0, N=1000, seed=83)
    n = np.arange(t.size)
    bound = (1 + b * h) ** n * 16.0
    assert np.all(d2 <= bound * (1 + 1e-12))
    assert d2[-1] < 1e-3 * d2[0]


@pytest.mark.parametrize("h", [1e-2, 1e-3])
def test_second_moment_decays(S, h):
    """§3.4.2 Fig. (a): E|X_t|^2 from X_0 = 1 decreases towards 0 (gamma = 0, T = 3)."""
    from paper_2105_09688_gb300 import stability as st
    t, m2 = st.second_moment_curve(0.0, h, 3.0, N=1000, x0=1.0, seed=84)
    assert m2[0] == pytest.approx(1.0)
    assert m2[-1] < 0.05
    assert np.all(m2[1:] < m2[0])


def test_gamma_sweep_at_the_papers_step(S):
    """§3.4.2 at h = 0.1: where the theorem applies (1 - h (2 L_v + 1) > 0) and gives
    beta < 0 (gamma = 0 here) the observed mean-square contraction factor per step is
    within 1 + beta h; the factor grows with gamma (the gamma-split moves the linear
    damping from the implicit v to the explicit b: per step the difference of two runs
    scales by about (1 + h gamma) / (1 + h (5/2 + gamma)), increasing in gamma)."""
    from paper_2105_09688_gb300 import stability as st
    rows = st.gamma_sweep(gammas=(-8.0, -4.0, 0.0, 4.0, 8.0), T=2.0, N=500, seed=85)
    checked = 0
    for r in rows:
        if r["theorem_applies"] and r["beta"] < 0:
            assert r["observed_factor"] <= r["theorem_factor"] * (1 + 1e-9), r
            checked += 1
    assert checked >= 1
    f = [r["observed_factor"] for r in rows]
    assert all(f[k] <= f[k + 1] for k in range(len(f) - 1)), rows
