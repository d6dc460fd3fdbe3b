"""ssm_pipe_probe, the measured basis of the pair kernels' roofline: the SM clock is
plausible, every rate is positive and within the nominal FP32 lanes of an SM (128
lane operations a clock), and the special-function unit is slower than the FMA pipe
(RCP at about an eighth and EX2 at about a quarter of it on this part)."""
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


def test_probe_rates_are_physical(S):
    p = S.ssm_pipe_probe()
    assert 0.5 < p["clock_ghz"] < 3.0
    for k in ("ffma", "ffma2", "rcp", "ex2"):
        assert 0.0 < p[k] <= 128.0 * 1.02, (k, p[k])
    assert p["rcp"] < p["ffma"] and p["ex2"] < p["ffma"]
