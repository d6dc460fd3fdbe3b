"""Device-detected errors reach the host as sticky statuses (include/ssm.h: after a
device-detected error every call returns that status until ssm_destroy).

* a non-finite particle, planted through ssm_set_state, is reported as
  SSM_ENONFINITE by the next synchronising call, in the FP64 and FP32C forms of a
  pair set and of a moment set;
* an implicit step that cannot meet its tolerance within newton_kmax passes (one
  pass from the plain start Y = X) is reported as SSM_ENOCONV;
* once set, the status is returned by every later call and no further step runs.

The failures are made on the host (a planted value, a pass limit); no kernel is
made to fault.
"""
import numpy as np
import pytest

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


def _expect(S, status, fn, *args):
    with pytest.raises(S.SSMError) as e:
        fn(*args)
    assert e.value.status == status, (e.value.status, status)


@pytest.mark.parametrize("coef,d,prec,p", [("SSM_COEF_COUPLED3D", 3, "SSM_FP64", ()),
                                           ("SSM_COEF_COUPLED3D", 3, "SSM_FP32C", ()),
                                           ("SSM_COEF_OU", 2, "SSM_FP32C", (-1.0, 0.5, 0.5)),
                                           ("SSM_COEF_GL1", 1, "SSM_FP32C", (1.5, 0.5))])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_particle_is_reported_and_sticky(S, coef, d, prec, p, bad):
    N = 300
    s = S.SSM(d=d, N=N, h=2.0 ** -8, T=1.0, coef=getattr(S, coef), seed=31, precision=getattr(S, prec),
              coef_params=p)
    s.run_steps(2)
    x, n = s.get_state()
    assert np.all(np.isfinite(x)) and n == 2
    x[177, d - 1] = bad
    s.set_state(x, n)
    _expect(S, S.SSM_ENONFINITE, s.sync)
    _expect(S, S.SSM_ENONFINITE, s.step)
    _expect(S, S.SSM_ENONFINITE, s.moments)
    _expect(S, S.SSM_ENONFINITE, s.get_state)
    s.close()


def test_unconverged_implicit_step_is_reported(S):
    """One pass from Y = X cannot reach 1e-13 (FP64) at h = 2^-4: SSM_ENOCONV."""
    s = S.SSM(d=3, N=400, h=2.0 ** -4, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=32, newton_kmax=1)
    s.step()
    _expect(S, S.SSM_ENOCONV, s.sync)
    _expect(S, S.SSM_ENOCONV, s.step)
    s.close()


def test_the_same_problem_converges_with_the_default_pass_limit(S):
    s = S.SSM(d=3, N=400, h=2.0 ** -4, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=32)
    s.run_steps(2)
    s.sync()
    x, n = s.get_state()
    assert n == 2 and np.all(np.isfinite(x))
    s.close()
