"""Step 1 against mu^Y (ssm_opts.measure_y = 1): the joint R^{dN} system of the
earlier implicit scheme that §1 sets the SSM against, on the GPU against the
oracle's Newton on the dense dN x dN system.

Tolerances: FP64 1e-10 relative per particle; FP32C per step within the step-1
tolerance plus the FP32 normals' effect (sigma sqrt(h) 5e-6 <= 1.2 * 2^-3 * 5e-6
= 7.5e-7 at h = 2^-6).  At sizes the dense oracle cannot solve, the joint residual
of sampled particles (an O(N) sum each) and the invariant
sum_i (Y_i - X_i + h Y_i |Y_i|^2) = 0 (the pair part sums to zero only when the
measure is the particles' own) are checked.
"""
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


def _coef(S, d):
    return (S.SSM_COEF_COUPLED1D, O.COEF_COUPLED1D) if d == 1 else (S.SSM_COEF_COUPLED3D, O.COEF_COUPLED3D)


@pytest.mark.parametrize("d,N", [(3, 150), (1, 300)])
def test_fp64_matches_joint_oracle(S, d, N):
    h, K = 2.0 ** -6, 8
    g, o = _coef(S, d)
    s = S.SSM(d=d, N=N, h=h, T=1.0, coef=g, seed=71, measure_y=1)
    s.run_steps(K)
    x, n = s.get_state()
    st = s.stats()
    s.close()
    P = O.problem(d=d, coef=o, N=N, h=h, seed=71, measure_y=1)
    xo = O.run(P, O.init_x0(P), 0, K)
    assert n == K and relerr(x, xo) < 1e-10
    assert 2 <= st["newton_passes"] / K <= 8
    Ps = O.problem(d=d, coef=o, N=N, h=h, seed=71)       # the SSM (mu^X) gives another result
    assert relerr(x, O.run(Ps, O.init_x0(Ps), 0, K)) > 1e-8


def test_fp32c_matches_joint_oracle(S):
    N, h, K = 150, 2.0 ** -6, 8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=72, precision=S.SSM_FP32C, measure_y=1)
    s.run_steps(K)
    x, _ = s.get_state()
    s.close()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=72, measure_y=1)
    xo = O.run(P, O.init_x0(P), 0, K)
    assert np.max(np.abs(x - xo)) < K * 7.5e-7


def test_fp64_invariant_and_joint_residual_at_larger_n(S):
    N, h = 1 << 14, 2.0 ** -6
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=73, measure_y=1)
    x0, _ = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    s.close()
    inv = np.sum(y - x0 + h * y * np.sum(y * y, axis=1, keepdims=True), axis=0)
    assert np.max(np.abs(inv)) < 1e-12 * N
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=73, measure_y=1)
    rng = np.random.default_rng(3)
    for i in np.concatenate([[0, N - 1], rng.integers(0, N, 30)]):
        assert np.max(np.abs(O.joint_residual_one(P, x0, y, int(i)))) < 2e-13


def test_fp32c_benchmark_size_joint_residual(S):
    """N = 2^18, h = 2^-8 (the benchmark workload), one step: sampled joint residuals
    within 64 x the FP32 tolerance (1e-10) plus the FP32 sums' error."""
    N, h = 1 << 18, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2, precision=S.SSM_FP32C, measure_y=1)
    x0, _ = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    st = s.stats()
    s.close()
    assert st["newton_passes"] <= 8
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2, measure_y=1)
    rng = np.random.default_rng(4)
    for i in np.concatenate([[0, N - 1], rng.integers(0, N, 12)]):
        assert np.max(np.abs(O.joint_residual_one(P, x0, y, int(i)))) < 1e-8
