"""Weak (k = 1) and strong (k = 2) error rates of §3 on the GPU, against a run at
h = T 2^-11 on the same Brownian paths, for the paper's examples: the weak errors
decrease at a fitted rate of about 1 (the paper's figures) and the strong ones at
no less than 1/2 (Theorem 2.3).  One study is recomputed by the oracle."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

KS, KREF = range(3, 8), 11


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return S


@pytest.mark.parametrize("name", ["gl1", "gl2", "cs"])
def test_weak_rate_one_and_strong_rate_half(S, name):
    from paper_2105_09688_gb300 import convergence as C
    coef, d, p, m0, s0, T = {"gl1": (S.SSM_COEF_GL1, 1, (1.5, 0.5), 1.0, 0.0, 1.0),
                             "gl2": (S.SSM_COEF_GL2, 1, (1.5, 0.5), 1.0, 0.0, 1.0),
                             "cs": (S.SSM_COEF_CS, 2, (2.0, 4.0), 1.0, math.sqrt(2.0), 2.0)}[name]
    r = C.error_study(coef, d, T, KS, KREF, 1 << 14, seed=91, coef_params=p, x0_mean=m0, x0_std=s0)
    assert r["weak"][-1] < r["weak"][0] and r["strong"][-1] < r["strong"][0]
    assert r["weak_slope"] >= 0.8, r
    assert r["strong_slope"] >= 0.45, r


def test_study_matches_the_oracle(S):
    """GL version 1, N = 200: the study's errors recomputed from oracle runs."""
    from paper_2105_09688_gb300 import convergence as C
    N, T, p = 200, 1.0, (1.5, 0.5)
    r = C.error_study(S.SSM_COEF_GL1, 1, T, KS, KREF, N, seed=92, coef_params=p, x0_mean=1.0, x0_std=0.0)
    Pr = O.problem(d=1, coef=O.COEF_GL1, N=N, h=T * 2.0 ** -KREF, T=T, seed=92, p=p, x0_mean=1.0, x0_std=0.0,
                   fine_log2=KREF)
    x0 = O.init_x0(Pr)
    ref = O.run(Pr, x0, 0, 1 << KREF)
    for k, w, st in zip(KS, r["weak"], r["strong"]):
        P = O.problem(d=1, coef=O.COEF_GL1, N=N, h=T * 2.0 ** -k, T=T, seed=92, p=p, x0_mean=1.0, x0_std=0.0,
                      fine_log2=KREF)
        xk = O.run(P, x0, 0, 1 << k)
        assert abs(w - abs(np.mean(xk - ref))) < 1e-9
        assert abs(st - math.sqrt(np.mean((xk - ref) ** 2))) < 1e-9


def test_batch_study_rates_on_mixed_ensembles(S):
    """The study on the batched form: d = 1 and 3 ensembles of uneven N with
    h = 2^-2..2^-6, each against its own run at h = 2^-10 on the same path, all in
    one graph launch: weak rate about 1, strong rate at least 1/2; the errors of one
    ensemble agree with the same study done on single contexts."""
    from paper_2105_09688_gb300 import convergence as C
    descs = [dict(d=d, N=N, h=2.0 ** -k, T=1.0, seed=seed) for d, N, seed in ((1, 2048, 1200), (3, 1024, 1201))
             for k in range(2, 7)]
    r = C.batch_study(descs, ref_log2=10, precision=S.SSM_FP64)
    assert len(r["per_ensemble"]) == len(descs)
    assert r["weak_slope"] >= 0.8, r
    assert r["strong_slope"] >= 0.45, r
    for d in (1, 3):
        rows = [p for p in r["per_ensemble"] if p["d"] == d]
        assert rows[-1]["weak"] < rows[0]["weak"] and rows[-1]["strong"] < rows[0]["strong"], rows
    one = C.error_study(S.SSM_COEF_COUPLED3D, 3, 1.0, range(2, 7), 10, 1024, seed=1201)
    rows = [p for p in r["per_ensemble"] if p["d"] == 3]
    for p, w, st in zip(rows, one["weak"], one["strong"]):
        assert abs(p["weak"] - w) <= 1e-9 * max(1.0, w) and abs(p["strong"] - st) <= 1e-9 * max(1.0, st)


def test_batch_study_weak_error_matches_the_oracle(S):
    """d = 1, N = 256, h = 2^-3 against h = 2^-10: the weak and strong errors of the
    batched study recomputed from oracle runs on the same Brownian path."""
    from paper_2105_09688_gb300 import convergence as C
    N, L = 256, 10
    r = C.batch_study([dict(d=1, N=N, h=2.0 ** -3, T=1.0, seed=1100)], ref_log2=L, precision=S.SSM_FP64)
    P = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=2.0 ** -3, seed=1100, fine_log2=L)
    Pr = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=2.0 ** -L, seed=1100, fine_log2=L)
    x0 = O.init_x0(P)
    diff = O.run(P, x0, 0, 8) - O.run(Pr, x0, 0, 1 << L)
    p = r["per_ensemble"][0]
    assert abs(p["weak"] - abs(np.mean(diff))) < 1e-9
    assert abs(p["strong"] - math.sqrt(np.mean(diff ** 2))) < 1e-9
