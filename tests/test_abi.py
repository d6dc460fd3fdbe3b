"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function that include/ssm.h declares; argument validation and
the pure host helpers behave as documented."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ssm_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def S():
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


def test_library_exports_every_declared_symbol(S):
    names = _declared_functions()
    assert len(names) >= 17, names
    L = S.lib()
    for n in names:
        assert hasattr(L, n), n


def test_status_strings_and_defaults(S):
    assert S.ssm_status_str(S.SSM_OK) == "SSM_OK"
    assert "invalid" in S.ssm_status_str(S.SSM_EINVAL)
    o = S.ssm_opts_default()
    assert o.precision == S.SSM_FP64 and o.newton_kmax == 12 and o.x0_std == 1.0


def test_workspace_bytes_grows_with_N(S):
    a = S.ssm_workspace_bytes(3, 1 << 10, S.SSM_COEF_COUPLED3D)
    b = S.ssm_workspace_bytes(3, 1 << 14, S.SSM_COEF_COUPLED3D)
    assert 0 < a < b
    assert S.ssm_workspace_bytes(3, 0, S.SSM_COEF_COUPLED3D) == 0


@pytest.mark.parametrize("args", [
    (1, 0, 0.01, 1.0, 0),            # N = 0 (empty system)
    (1, 100, 0.5, 1.0, 0),           # h above 1/(1 + 2 L_v) = 1/3 (Theorem 2.3)
    (3, 100, 0.01, 1.0, 0),          # CUBIC1D needs d = 1
    (1, 100, 0.01, 1.0, 1),          # COUPLED3D needs d = 3
    (1, 100, 0.03, 1.0, 0),          # T/h not an integer
    (1, 100, -0.01, 1.0, 0),         # h <= 0
    (1, (1 << 26) + 1, 0.01, 1.0, 0),  # beyond the maximum N
    (1, 100, 0.01, 1.0, 9),          # unknown coefficient set
    (2, 100, 0.01, 1.0, 8),          # the GL stability set needs d = 1
    (1, 100, 0.01, 1.0, 7),          # Cucker-Smale needs d = 2
    (2, 100, 0.01, 1.0, 4),          # GL needs d = 1
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(S, args):
    d, N, h, T, coef = args
    with pytest.raises(S.SSMError) as e:
        S.ssm_create(d, N, h, T, coef, 0)
    assert e.value.status == S.SSM_EINVAL


def test_ou_step_bound_follows_rho(S):
    o = S.ssm_opts_default(coef_params=(1.0, 0.0, 0.0))   # L_v = rho = 1 -> h <= 1/3
    with pytest.raises(S.SSMError):
        S.ssm_create(1, 10, 0.5, 1.0, S.SSM_COEF_OU, 0, o)


def test_learned_form_needs_coupled_set(S):
    o = S.ssm_opts_default(precision=S.SSM_FP32C_LEARNED)
    with pytest.raises(S.SSMError):
        S.ssm_create(1, 10, 0.01, 1.0, S.SSM_COEF_CUBIC1D_GAUSS, 0, o)


@pytest.mark.parametrize("desc", [
    dict(d=2, N=100, h=0.1, T=1.0, seed=0),        # d must be 1 or 3
    dict(d=3, N=0, h=0.1, T=1.0, seed=0),          # empty ensemble
    dict(d=3, N=100, h=0.95, T=1.9, seed=0),       # h above 1/(1 + 2/16) (Theorem 2.3)
    dict(d=1, N=100, h=0.3, T=1.0, seed=0),        # T/h not an integer
    dict(d=1, N=100, h=2.0 ** -4, T=1.0, seed=0, fine_log2=3),   # fine grid coarser than h
])
def test_batch_rejects_bad_descriptors_before_touching_the_gpu(S, desc):
    good = dict(d=1, N=10, h=0.25, T=1.0, seed=1)
    with pytest.raises(S.SSMError) as e:
        S.Batch([good, desc])
    assert e.value.status == S.SSM_EINVAL


def test_batch_rejects_unsupported_precision(S):
    with pytest.raises(S.SSMError):
        S.Batch([dict(d=1, N=10, h=0.25, T=1.0, seed=1)], precision=S.SSM_FP32C_LEARNED)


def test_measure_y_option_is_validated(S):
    """Step 1 against mu^Y exists for the coupled sets in the FP64 and FP32C forms."""
    for coef, prec, flag in [(S.SSM_COEF_CUBIC1D_GAUSS, 0, 1), (S.SSM_COEF_OU, 0, 1),
                             (S.SSM_COEF_COUPLED3D, 2, 1), (S.SSM_COEF_COUPLED3D, 0, 2)]:
        d = 3 if coef == S.SSM_COEF_COUPLED3D else 1
        o = S.ssm_opts_default(precision=prec, measure_y=flag)
        with pytest.raises(S.SSMError) as e:
            S.ssm_create(d, 10, 2.0 ** -6, 1.0, coef, 0, o)
        assert e.value.status == S.SSM_EINVAL
