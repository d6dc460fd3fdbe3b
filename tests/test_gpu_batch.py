"""The batched form (many ensembles, one graph launch) and the 1-d coupled set.

* every ensemble of a mixed batch (d = 1 and 3, uneven N, different h) ends where
  a single context of the same ensemble ends;
* small batches match the FP64 oracle per particle (FP64: 1e-10 relative;
  FP32C: 1e-4 absolute per particle at T, 1e-5 on mean and variance);
* the rMSE-vs-h study on shared Brownian paths gives the strong order of
  Theorem 2.3 (fitted slope >= 0.45), and one of its errors is recomputed with
  the oracle;
* partial runs stop at the requested batch step; the autotuner changes launch
  shapes, not results.
"""
import math

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
    return S.SSM_COEF_COUPLED1D if d == 1 else S.SSM_COEF_COUPLED3D


def _ocoef(d):
    return O.COEF_COUPLED1D if d == 1 else O.COEF_COUPLED3D


MIXED = [dict(d=3, N=700, h=2.0 ** -5, T=0.5, seed=1000),
         dict(d=1, N=1, h=2.0 ** -4, T=0.5, seed=1001),
         dict(d=1, N=2500, h=2.0 ** -6, T=0.5, seed=1002),
         dict(d=3, N=7, h=2.0 ** -3, T=0.5, seed=1003),
         dict(d=3, N=300, h=2.0 ** -6, T=0.5, seed=1004),
         dict(d=1, N=9000, h=2.0 ** -4, T=0.5, seed=1005)]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_single_contexts(S, prec):
    b = S.Batch(MIXED, precision=prec)
    b.run()
    b.sync()
    for e, dsc in enumerate(MIXED):
        xb, nb = b.get_state(e)
        s = S.SSM(d=dsc["d"], N=dsc["N"], h=dsc["h"], T=dsc["T"], coef=_coef(S, dsc["d"]), seed=dsc["seed"],
                  precision=prec)
        s.run()
        xs, ns = s.get_state()
        ms = s.moments()
        s.close()
        assert nb == ns == round(dsc["T"] / dsc["h"])
        if prec == 0:
            assert relerr(xb, xs) < 1e-11, e
        else:
            assert np.max(np.abs(xb - xs)) < 1e-7, e
        assert relerr(b.moments(e), ms) < (1e-11 if prec == 0 else 1e-7)
    st = b.stats()
    assert st["ensemble_steps"] == sum(round(d["T"] / d["h"]) for d in MIXED)
    assert st["batch_steps"] == max(round(d["T"] / d["h"]) for d in MIXED)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_carried_start_matches_single_contexts(S, prec):
    """ssm_opts.carry_start in the batched form: every ensemble ends where a single
    context of it with the carried start ends (same tolerances as from the plain
    start), with fewer step-1 pair rows than the batch from the plain start."""
    rows = []
    for carry in (0, 1):
        b = S.Batch(MIXED, precision=prec, carry_start=carry)
        b.run()
        b.sync()
        if carry:
            for e, dsc in enumerate(MIXED):
                xb, nb = b.get_state(e)
                s = S.SSM(d=dsc["d"], N=dsc["N"], h=dsc["h"], T=dsc["T"], coef=_coef(S, dsc["d"]),
                          seed=dsc["seed"], precision=prec, carry_start=1)
                s.run()
                xs, ns = s.get_state()
                s.close()
                assert nb == ns
                if prec == 0:
                    assert relerr(xb, xs) < 1e-11, e
                else:
                    assert np.max(np.abs(xb - xs)) < 1e-7, e
        rows.append(b.stats()["newton_rows"])
        b.close()
    # these ensembles take 4 to 32 steps of h = 2^-3 .. 2^-6 (the first step of each
    # starts plain): about 14% fewer rows here, a third fewer at the benchmark's h
    assert rows[1] < 0.9 * rows[0], rows


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle(S, prec):
    descs = [dict(d=1, N=333, h=2.0 ** -5, T=1.0, seed=7), dict(d=3, N=257, h=2.0 ** -4, T=1.0, seed=8)]
    b = S.Batch(descs, precision=prec)
    b.run()
    for e, dsc in enumerate(descs):
        xb, _ = b.get_state(e)
        P = O.problem(d=dsc["d"], coef=_ocoef(dsc["d"]), N=dsc["N"], h=dsc["h"], seed=dsc["seed"])
        xo = O.run(P, O.init_x0(P), 0, round(1.0 / dsc["h"]))
        if prec == 0:
            assert relerr(xb, xo) < 1e-10
        else:
            assert np.max(np.abs(xb - xo)) < 1e-4
            mb, mo = b.moments(e), O.moments(P, xo)
            assert np.max(np.abs(mb[0] - mo[0])) < 1e-5
            assert np.max(np.abs((mb[1] - mb[0] ** 2) - (mo[1] - mo[0] ** 2))) < 1e-5
    b.close()


def test_convergence_study_on_shared_paths(S):
    """rMSE at T of h = 2^-2..2^-6 against h = 2^-10 on the same Brownian paths
    (fine grid 2^-10), d = 1 and d = 3: decreasing errors, fitted slope >= 0.45."""
    L, N = 10, 256
    for d, seed in ((1, 1100), (3, 1101)):
        descs = [dict(d=d, N=N, h=2.0 ** -k, T=1.0, seed=seed, fine_log2=L) for k in range(2, 7)]
        descs.append(dict(d=d, N=N, h=2.0 ** -L, T=1.0, seed=seed, fine_log2=L))
        b = S.Batch(descs, precision=S.SSM_FP32C)
        b.run()
        ref, _ = b.get_state(len(descs) - 1)
        errs = []
        for e in range(len(descs) - 1):
            x, _ = b.get_state(e)
            errs.append(math.sqrt(np.mean(np.sum((x - ref) ** 2, axis=1))))
        b.close()
        hs = [2.0 ** -k for k in range(2, 7)]
        slope = np.polyfit(np.log2(hs), np.log2(errs), 1)[0]
        assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
        assert slope >= 0.45, (d, slope, errs)
    # one error of the study recomputed by the oracle (d = 1, h = 2^-3)
    P = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=2.0 ** -3, seed=1100, fine_log2=L)
    Pr = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=2.0 ** -L, seed=1100, fine_log2=L)
    x0 = O.init_x0(P)
    xo, xr = O.run(P, x0, 0, 8), O.run(Pr, x0, 0, 1 << L)
    e_o = math.sqrt(np.mean(np.sum((xo - xr) ** 2, axis=1)))
    b = S.Batch([dict(d=1, N=N, h=2.0 ** -3, T=1.0, seed=1100, fine_log2=L),
                 dict(d=1, N=N, h=2.0 ** -L, T=1.0, seed=1100, fine_log2=L)], precision=S.SSM_FP64)
    b.run()
    e_g = math.sqrt(np.mean(np.sum((b.get_state(0)[0] - b.get_state(1)[0]) ** 2, axis=1)))
    b.close()
    assert abs(e_g - e_o) < 1e-9 * max(1.0, e_o)


def test_partial_runs_and_autotune(S):
    descs = [dict(d=3, N=1500, h=2.0 ** -4, T=1.0, seed=5), dict(d=1, N=4000, h=2.0 ** -2, T=1.0, seed=6)]
    a = S.Batch(descs, precision=S.SSM_FP32C)
    a.run_steps(3)
    assert [a.get_state(e)[1] for e in range(2)] == [3, 3]
    a.run_steps(3)
    assert [a.get_state(e)[1] for e in range(2)] == [6, 4]
    a.run()
    xa = [a.get_state(e)[0] for e in range(2)]
    b = S.Batch(descs, precision=S.SSM_FP32C)
    best = b.autotune()
    assert best > 0
    plan = b.plan()
    assert plan["chunk_len"] in (4096, 8192, 16384)
    b.run()
    for e in range(2):
        d = descs[e]
        K = round(1.0 / d["h"])
        assert b.get_state(e)[1] == K
        # the tuned shapes sum the pair terms in another order (and, with 8 d = 1
        # targets a thread, take one reciprocal in eight on the FMA pipe), so the two
        # runs agree to what the FP32 forms' residual test admits: each root within
        # 64 tol of the exact one (the stagnation rule), tol = 2^-27 h (1 + 64/sqrt(N)),
        # so K steps differ by at most K x 2 x 64 tol
        tol = max(1e-10, 2.0 ** -27 * d["h"] * (1.0 + 64.0 / math.sqrt(d["N"])))
        assert np.max(np.abs(b.get_state(e)[0] - xa[e])) < K * 2 * 64 * tol
    a.close()
    b.close()


@pytest.mark.parametrize("N", [1, 5, 640])
def test_coupled1d_single_context_fp64(S, N):
    h = 2.0 ** -6
    s = S.SSM(d=1, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED1D, seed=3)
    s.run()
    x, _ = s.get_state()
    s.close()
    P = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=h, seed=3)
    assert relerr(x, O.run(P, O.init_x0(P), 0, 64)) < 1e-10


def test_coupled1d_single_context_fp32c(S):
    N, h = 3000, 2.0 ** -6
    s = S.SSM(d=1, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED1D, seed=4, precision=S.SSM_FP32C)
    s.run()
    x, _ = s.get_state()
    m = s.moments()
    s.close()
    P = O.problem(d=1, coef=O.COEF_COUPLED1D, N=N, h=h, seed=4)
    xo = O.run(P, O.init_x0(P), 0, 64)
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert abs(m[0, 0] - mo[0, 0]) < 1e-5 and abs((m[1, 0] - m[0, 0] ** 2) - (mo[1, 0] - mo[0, 0] ** 2)) < 1e-5


@pytest.mark.parametrize("N,h", [(7, 2.0 ** -3), (50, 2.0 ** -4), (400, 2.0 ** -2)])
def test_coupled3d_fp32c_large_h_small_n(S, N, h):
    """FP32 pair sums where their evaluation floor exceeds 1e-10 (large h, small N):
    the iteration stops at the floor and the run stays within the FP32 bar."""
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=9, precision=S.SSM_FP32C)
    s.run()
    x, _ = s.get_state()
    s.close()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=9)
    xo = O.run(P, O.init_x0(P), 0, round(1.0 / h))
    assert np.max(np.abs(x - xo)) < 1e-4
