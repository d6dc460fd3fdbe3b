"""The paper's moment-interaction examples on the GPU against the oracle: GL
versions 1 and 2 (§3.2), polynomial drift (§3.3) and Cucker-Smale (§3.4), at the
paper's sizes (N = 1000, the paper's parameters, h = 1e-2) over the whole horizon,
one step's stages element by element, and the grid-stride launch at N = 2^22 on
sampled particles.

Tolerances: FP64 form 1e-10 relative per particle; FP32C form 1e-4 absolute per
particle at T and 1e-5 on mean and variance.  At N = 2^22 the FP32C step is checked
per step: the FP32 normals move x by < |sigma| sqrt(h) 5e-6, the FP32 increment
by < 2^-24 |h b + sigma dW|, the FP32-started cubic root by ~1e-13 relative, so
|dx| < 1e-5 max(1, |x|) for these sets (|sigma| <= 4 |mean - V| for Cucker-Smale).
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

# name: (d, GPU set, oracle set, params, T, x0 mean, x0 std, seed)
SETS = {
    "gl1": (1, "SSM_COEF_GL1", O.COEF_GL1, (1.5, 0.5), 1.0, 1.0, 0.0, 51),
    "gl2": (1, "SSM_COEF_GL2", O.COEF_GL2, (1.5, 0.5), 1.0, 1.0, 0.0, 52),
    "poly": (1, "SSM_COEF_POLY", O.COEF_POLY, (-1.0,), 2.0, 1.0, 0.0, 53),
    "cs": (2, "SSM_COEF_CS", O.COEF_CS, (2.0, 4.0), 2.0, 1.0, math.sqrt(2.0), 54),
}
H = 1e-2


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


def _ctx(S, name, N, prec, seed=None):
    d, gcoef, _, p, T, m0, s0, sd = SETS[name]
    return S.SSM(d=d, N=N, h=H, T=T, coef=getattr(S, gcoef), seed=sd if seed is None else seed, precision=prec,
                 coef_params=p, x0_mean=m0, x0_std=s0)


def _problem(name, N, seed=None):
    d, _, ocoef, p, T, m0, s0, sd = SETS[name]
    return O.problem(d=d, coef=ocoef, N=N, h=H, T=T, seed=sd if seed is None else seed, p=p, x0_mean=m0, x0_std=s0)


@pytest.mark.parametrize("name", list(SETS))
def test_fp64_full_horizon(S, name):
    N = 1000
    s = _ctx(S, name, N, S.SSM_FP64)
    s.run()
    x, n = s.get_state()
    m = s.moments()
    s.close()
    P = _problem(name, N)
    M = int(round(SETS[name][4] / H))
    xo = O.run(P, O.init_x0(P), 0, M)
    assert n == M
    assert relerr(x, xo) < 1e-10
    assert relerr(m, O.moments(P, xo)) < 1e-10


@pytest.mark.parametrize("name", list(SETS))
def test_fp32c_full_horizon(S, name):
    N = 1000
    s = _ctx(S, name, N, S.SSM_FP32C)
    s.run()
    x, n = s.get_state()
    m = s.moments()
    s.close()
    P = _problem(name, N)
    xo = O.run(P, O.init_x0(P), 0, int(round(SETS[name][4] / H)))
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert np.max(np.abs(m[0] - mo[0])) < 1e-5
    assert np.max(np.abs((m[1] - m[0] ** 2) - (mo[1] - mo[0] ** 2))) < 1e-5


@pytest.mark.parametrize("name", list(SETS))
def test_stages_of_one_step(S, name):
    """Y from the GPU's X_n and b(Y, mu^Y) from the GPU's Y, every particle (FP64)."""
    N = 777
    s = _ctx(S, name, N, S.SSM_FP64, seed=60)
    s.run_steps(3)
    x0, n = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    b = s.get_stage(S.SSM_STAGE_B)
    s.close()
    P = _problem(name, N, seed=60)
    yo, it, bad = O.implicit_step(P, x0)
    assert bad == 0 and relerr(y, yo) < 1e-13
    bo = np.stack([O.drift_one(P, y, i) for i in range(N)])
    assert relerr(b, bo) < 1e-13


@pytest.mark.parametrize("name", list(SETS))
def test_fp32c_large_n_sampled_steps(S, name):
    N = 1 << 22
    s = _ctx(S, name, N, S.SSM_FP32C, seed=61)
    P = _problem(name, N, seed=61)
    rng = np.random.default_rng(2)
    for step in range(2):
        x0, n = s.get_state()
        s.step()
        y = s.get_stage(S.SSM_STAGE_Y)
        x1, _ = s.get_state()
        for i in np.concatenate([[0, N - 1], rng.integers(0, N, 5)]):
            yo, it = O.implicit_one(P, x0, int(i))
            assert np.max(np.abs(y[i] - yo)) < 1e-7 * max(1.0, np.abs(yo).max())
            xo = O.explicit_one(P, y, int(i), n)
            assert np.max(np.abs(x1[i] - xo)) < 1e-5 * max(1.0, np.abs(xo).max())
    s.close()


@pytest.mark.parametrize("name,gamma", [("gl1", None), ("gl2", None), ("cs", None), ("glstab", 2.0)])
def test_fp32c_cubic_roots_over_a_wide_range(S, name, gamma):
    """Step 1 of the cubic sets in the FP32C form (FP32 Cardano root, one Newton
    correction with the residual in double-float arithmetic) against the oracle's
    root for states over 1e-30 .. 1e6 of both signs, every particle: within 1e-12
    of the larger of |y| and |x| (absolute below 1e-15, where the dropped low half
    of a state smaller than 2^-74 in magnitude is < 2^-98)."""
    N = 4096
    rng = np.random.default_rng(7)
    if name == "glstab":
        d, gcoef, ocoef, p = 1, S.SSM_COEF_GLSTAB, O.COEF_GLSTAB, (gamma,)
    else:
        d, gname, ocoef, p = SETS[name][0], SETS[name][1], SETS[name][2], SETS[name][3]
        gcoef = getattr(S, gname)
    x = np.zeros((N, d))
    x[:, 0] = rng.choice([-1.0, 1.0], N) * 10.0 ** rng.uniform(-30, 6, N)
    x[:8, 0] = [0.0, -0.0, 1.0, -1.0, 1e6, -1e6, 2.0 ** -74, 3.0]
    if d == 2:
        x[:, 1] = rng.standard_normal(N)
    s = S.SSM(d=d, N=N, h=H, T=1.0, coef=gcoef, seed=63, precision=S.SSM_FP32C, coef_params=p, x0_mean=0.0,
              x0_std=1.0)
    s.set_state(x, 0)
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    s.close()
    # set_state recomputes the moments of the planted state in FP64, so GL2's measure
    # term is the oracle's
    P = O.problem(d=d, coef=ocoef, N=N, h=H, T=1.0, seed=63, p=p, x0_mean=0.0, x0_std=1.0)
    yo, it, bad = O.implicit_step(P, x)
    assert bad == 0
    # relative to the larger of the root and the state: GL2's x + c is formed to
    # ~2^-48 of its terms, which near a root y ~ 0 (x ~ -c) is large against |y|
    err = np.abs(y - yo) / np.maximum(np.maximum(np.abs(yo), np.abs(x[:, :1])), 1e-15)
    assert err.max() < 1e-12, (err.max(), x[np.argmax(err.max(axis=1))])
