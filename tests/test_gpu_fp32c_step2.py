"""Step 2 of the FP32C forms against the oracle: the FP32 evaluation of the
Box-Muller transform and the FP32 increment added to the FP64 state.

Bounds, derived from the arithmetic:
  * normals: the angle 2 pi u2 carries the FP32 rounding of the leading Philox word
    (<= pi 2^-23 absolute), times r = sqrt(-2 ln u1) <= 8.6, plus the FP32 rounding
    of r and a few ulps of the library log/sincospi: |z32 - z| < 5e-6, median ~1e-7;
  * one step: |dx| <= sigma sqrt(h) 5e-6 + 2^-24 |h b + sigma dW|; for the OU set
    below (eta = 0.5, h = 2^-6) that is < 3.2e-7 per step, so < 2.5e-5 after 64 steps
    (the implicit step contracts, the mean coupling lambda h = 2^-7 is small).
The FP64 form of every set is unchanged and checked at 1e-10 elsewhere.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

OU = dict(coef_params=(-1.0, 0.5, 0.5), x0_mean=1.0, x0_std=0.5)


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


def test_fp32_normals_within_bound(S):
    seed, N, step = 77, 1 << 16, 5
    z32 = S.ssm_normals_fp32(seed, 3, N, step, 1).astype(np.float64)
    z64 = S.ssm_normals(seed, 3, N, step, 1)
    err = np.abs(z32 - z64)
    assert err.max() < 5e-6, err.max()
    assert np.median(err) < 3e-7
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 2000)]))
    zo = np.stack([O.normals(seed, 3, int(i), step, 1) for i in idx])
    assert np.max(np.abs(z32[idx] - zo)) < 5e-6
    # both branches of ln u1 (u1 below and above 1/2) are exercised: |z| small and large
    r = np.sqrt(z64[:, 0] ** 2 + z64[:, 1] ** 2)
    assert (r < np.sqrt(-2 * np.log(0.5))).any() and (r > np.sqrt(-2 * np.log(0.5))).any()


@pytest.mark.parametrize("d", [1, 3])
def test_ou_fp32c_matches_oracle(S, d):
    N, h = 4096, 2.0 ** -6
    s = S.SSM(d=d, N=N, h=h, T=1.0, coef=S.SSM_COEF_OU, seed=31, precision=S.SSM_FP32C, **OU)
    s.run()
    x, n = s.get_state()
    m = s.moments()
    s.close()
    P = O.problem(d=d, coef=O.COEF_OU, N=N, h=h, seed=31, p=OU["coef_params"], x0_mean=1.0, x0_std=0.5)
    xo = O.run(P, O.init_x0(P), 0, 64)
    assert n == 64
    assert np.max(np.abs(x - xo)) < 2.5e-5
    mo = O.moments(P, xo)
    assert np.max(np.abs(m[0] - mo[0])) < 1e-5
    assert np.max(np.abs((m[1] - m[0] ** 2) - (mo[1] - mo[0] ** 2))) < 1e-5
    assert np.max(np.abs(m[2:] - mo[2:]) / np.maximum(1.0, np.abs(mo[2:]))) < 1e-5


def test_ou_fp32c_large_n_sampled_steps(S):
    """N = 2^22 (the grid-stride launch the O(N) benchmark uses): three steps; for
    sampled particles the oracle recomputes Y_i from the GPU's X_n and X_{n+1,i} from
    the GPU's Y (its b is a mean over all N, so each sample costs O(N)); per step
    within 3.2e-7 of the oracle."""
    N, h = 1 << 22, 2.0 ** -6
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_OU, seed=32, precision=S.SSM_FP32C, **OU)
    P = O.problem(d=3, coef=O.COEF_OU, N=N, h=h, seed=32, p=OU["coef_params"], x0_mean=1.0, x0_std=0.5)
    rng = np.random.default_rng(1)
    for step in range(3):
        x0, n = s.get_state()
        s.step()
        y = s.get_stage(S.SSM_STAGE_Y)
        x1, _ = s.get_state()
        for i in np.concatenate([[0, N - 1], rng.integers(0, N, 6)]):
            yo, it = O.implicit_one(P, x0, int(i))
            assert np.max(np.abs(y[i] - yo)) < 1e-15 * max(1.0, np.abs(yo).max())
            xo = O.explicit_one(P, y, int(i), n)
            assert np.max(np.abs(x1[i] - xo)) < 3.2e-7
    s.close()


def test_fp32c_and_fp64_share_the_brownian_path(S):
    """The two forms draw the same Philox words: their OU runs differ only by the
    FP32 rounding of z and of the increment."""
    N, h = 2000, 2.0 ** -6
    xs = []
    for prec in (S.SSM_FP64, S.SSM_FP32C):
        s = S.SSM(d=2, N=N, h=h, T=1.0, coef=S.SSM_COEF_OU, seed=33, precision=prec, **OU)
        s.run()
        xs.append(s.get_state()[0])
        s.close()
    assert np.max(np.abs(xs[0] - xs[1])) < 2.5e-5
    assert np.max(np.abs(xs[0] - xs[1])) > 0.0
