"""The binary64 <-> binary32 conversions the FP32C kernels do with integer
instructions (IEEE 754 bit manipulation, round to nearest even), run on the host
through the library and compared bit for bit with numpy's conversions.  Inputs
below the binary32 normal range (|v| < 2^-126) give a zero of the input's sign."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


def _cases():
    rng = np.random.default_rng(5)
    f32 = np.finfo(np.float32)
    # random values over the whole binary32 range and beyond, both signs
    r = rng.standard_normal(200000) * 2.0 ** rng.integers(-160, 160, 200000)
    # halfway cases: a binary32 value plus exactly half an ulp, and one binary64 ulp either side
    base = rng.standard_normal(20000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(base.astype(np.float32)).astype(np.float64)
    half = base + ulp / 2
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, f32.max, -f32.max, float(f32.max) * (1 + 2 ** -25),
                      float(f32.max) * (1 + 2 ** -24), f32.tiny, f32.tiny * (1 - 2 ** -30), f32.tiny / 2,
                      2.0 ** -149, 2.0 ** -150, 2.0 ** -151, 1.0, 1 + 2 ** -24, 1 + 2 ** -23 + 2 ** -24,
                      1 - 2 ** -25, 3.0 ** 0.5, 1e300, -1e-300])
    return np.concatenate([r, half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf), edges])


def test_double_to_float_matches_numpy_bit_for_bit(S):
    v = _cases()
    o32, _ = S.ssm_convert_check(v)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32)
    tiny = np.abs(v) < np.finfo(np.float32).tiny
    ref[tiny] = np.copysign(np.float32(0.0), v[tiny]).astype(np.float32)
    assert tiny.sum() > 1000 and (~tiny).sum() > 100000
    same = (o32.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(o32) & np.isnan(ref))
    assert same.all(), v[~same][:5]


def test_below_the_normal_range_gives_a_signed_zero(S):
    v = np.array([2.0 ** -126 * (1 - 2 ** -30), -2.0 ** -127, 2.0 ** -149, -2.0 ** -1074, 0.0, -0.0, 1e-300])
    o32, o64 = S.ssm_convert_check(v)
    assert (o32 == 0).all() and (np.signbit(o32) == np.signbit(v)).all()
    assert (o64 == 0).all() and (np.signbit(o64) == np.signbit(v)).all()


def test_float_to_double_is_exact(S):
    v = _cases()
    o32, o64 = S.ssm_convert_check(v)
    ref = o32.astype(np.float64)
    same = (o64.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(o64) & np.isnan(ref))
    assert same.all()


def test_conversion_check_validates_arguments(S):
    assert S.lib().ssm_convert_check(None, 3, None, None) == S.SSM_EINVAL
    assert S.lib().ssm_convert_check(None, 0, None, None) == S.SSM_OK
