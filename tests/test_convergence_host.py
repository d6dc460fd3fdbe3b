"""Host-side checks of the error studies (no GPU): argument validation happens
before any device work."""
import pytest


def test_batch_study_rejects_a_step_not_coarser_than_the_reference():
    from paper_2105_09688_gb300 import convergence as C
    with pytest.raises(ValueError):
        C.batch_study([dict(d=1, N=8, h=2.0 ** -10, T=1.0, seed=0)], ref_log2=10)
    with pytest.raises(ValueError):
        C.batch_study([dict(d=3, N=8, h=2.0 ** -12, T=1.0, seed=0)], ref_log2=10)


def test_weak_and_strong_errors_follow_their_definitions():
    """epsilon_1 = |(1/N) sum_j (X^j - Xhat^j)|, epsilon_2 = ((1/N) sum_j |X^j - Xhat^j|^2)^(1/2)
    (§3): a common offset c gives both |c|; differences of zero mean give epsilon_1 = 0
    and their root mean square."""
    import numpy as np
    from paper_2105_09688_gb300 import convergence as C
    ref = np.random.default_rng(3).standard_normal((1000, 3))
    c = np.array([0.3, -0.4, 1.2])
    w, s = C.weak_strong(ref + c, ref)
    assert abs(w - 1.3) < 1e-12 and abs(s - 1.3) < 1e-12
    dev = np.zeros((1000, 3))
    dev[0::2, 1], dev[1::2, 1] = 0.5, -0.5
    w, s = C.weak_strong(ref + dev, ref)
    assert w < 1e-15 and abs(s - 0.5) < 1e-12
