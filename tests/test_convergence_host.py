"""Host-side checks of the error studies (no GPU): argument validation happens
before any device work."""
import pytest


def test_batch_study_rejects_a_step_not_coarser_than_the_reference():
    from paper_2105_09688_gb300 import convergence as C
    with pytest.raises(ValueError):
        C.batch_study([dict(d=1, N=8, h=2.0 ** -10, T=1.0, seed=0)], ref_log2=10)
    with pytest.raises(ValueError):
        C.batch_study([dict(d=3, N=8, h=2.0 ** -12, T=1.0, seed=0)], ref_log2=10)
