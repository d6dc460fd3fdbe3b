"""The packed centred-expansion form of the FP32 pair kernels (d = 3), against the oracle.

The expansion evaluates the same pair sums of §2.3 (eq. SSTM:scheme 1 and 2) as
the difference form, with |x_j - y_i|^2 expanded about the centroid of each
block's targets; a block with a target far from that point falls back to the
difference form.
Checked here, through the C ABI on the same seeded inputs as the oracle:
  * one step at N = 3000 (several tiles, ragged tail) for every compiled shape of
    the form: Y (step 1) within 2e-9 relative of the oracle's implicit solve from
    the GPU's X_n, and b(Y, mu^Y) (step 2) within 5e-7 absolute of the oracle's
    drift at the GPU's Y, for every particle.  The b bound: the exponent
    -|s|^2 + 2 s.t is formed by three FP32 roundings of values up to |s|^2 + |t|^2,
    which is below ~16 for targets within 3 standard deviations of their block's
    centroid (scaled coordinates), so a term carries <= 3 * 2^-24 * 16 * ln 2 ~ 2e-6
    relative error and b = (1/N) sum (y_j - y_i) e_ij, |b| <~ 0.25 here, <= 5e-7;
  * the same with outlying particles planted (blocks that fall back, and a target
    inside the drift's bound but outside step 1's) and with the cloud far from the
    origin (the centring);
  * the full horizon at the FP32-compensated tolerances (1e-4 per particle, 1e-5
    on mean and variance);
  * the batched form with the expansion against single contexts and against its
    own difference form.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

H = 2.0 ** -8


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


def _ctx(S, N, seed, shape, **kw):
    s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=S.SSM_FP32C, **kw)
    s.set_plan(0, *shape)
    s.set_plan(1, *shape)
    assert s.plan(0)["form"] == shape[0] and s.plan(1)["form"] == shape[0]
    return s


def _check_one_step(S, s, P, tol_y=2e-9, tol_b=5e-7):
    x0, n = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    b = s.get_stage(S.SSM_STAGE_B)
    yo, it, bad = O.implicit_step(P, x0)
    assert bad == 0 and np.all(it >= 0)
    ey = relerr(y, yo)
    bo = np.stack([O.drift_one(P, y, i) for i in range(P.N)])
    eb = float(np.max(np.abs(b - bo)))
    assert ey < tol_y, ey
    assert eb < tol_b, eb
    return ey, eb


@pytest.mark.parametrize("shape", [(1, 128, 8), (2, 128, 8), (2, 128, 4), (2, 256, 4), (2, 256, 8)])
def test_one_step_every_shape(S, shape):
    N, seed = 3000, 21
    s = _ctx(S, N, seed, shape)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, seed=seed)
    _check_one_step(S, s, P)
    s.close()


def test_outliers_fall_back_per_block(S):
    """Particles at distance ~20, 12 and 9 from their block's centroid: the blocks fail the
    expansion's bound |t|^2 <= 64 in step 1 (all three) and in the drift (the
    first two; the third is inside the drift's scaled bound 0.72 * 81 = 58)."""
    N, seed = 3000, 22
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, seed=seed)
    x0 = O.init_x0(P)
    x0[0] = (20.0, -3.0, 5.0)
    x0[1777] = (0.0, 0.0, 12.0)
    x0[2999] = (-9.0, 0.0, 0.0)
    for shape in [(2, 128, 8), (2, 128, 4), (1, 128, 8)]:
        s = _ctx(S, N, seed, shape)
        s.set_state(x0, 0)
        _check_one_step(S, s, P)
        s.close()


def test_cloud_far_from_origin(S):
    """X_0 ~ N(6, I), and step 1 moves the cloud by ~1 per coordinate: the
    expansion is centred on each block's targets, so its accuracy does not
    depend on where the cloud sits."""
    N, seed = 3000, 23
    s = _ctx(S, N, seed, (2, 128, 8), x0_mean=6.0)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, seed=seed, x0_mean=6.0)
    xg, _ = s.get_state()
    assert relerr(xg, O.init_x0(P)) < 1e-14
    _check_one_step(S, s, P)
    _check_one_step(S, s, P)
    s.close()


@pytest.mark.parametrize("step1_rpt", [8, 4])
def test_full_horizon_tolerances(S, step1_rpt):
    """N = 1536, h = 2^-8, T = 1 with the expansion in both pair kinds (drift 128 x 8;
    step-1 sums 128 x 8, or 128 x 4 with the accumulators in shared memory)."""
    N, seed = 1536, 2
    s = _ctx(S, N, seed, (2, 128, 8))
    s.set_plan(0, 2, 128, step1_rpt)
    s.run()
    x, n = s.get_state()
    m = s.moments()
    st = s.stats()
    s.close()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, seed=seed)
    xo = O.run(P, O.init_x0(P), 0, 256)
    assert n == 256 and st["max_passes"] < 12
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert np.max(np.abs(m[0] - mo[0])) < 1e-5
    assert np.max(np.abs((m[1] - m[0] ** 2) - (mo[1] - mo[0] ** 2))) < 1e-5


DESCS = [dict(d=3, N=700, h=2.0 ** -5, T=0.25, seed=1200),
         dict(d=1, N=900, h=2.0 ** -4, T=0.25, seed=1201),
         dict(d=3, N=2100, h=2.0 ** -6, T=0.25, seed=1202)]


@pytest.mark.parametrize("r3", [8, 4])
def test_batch_expansion_matches_single_contexts(S, r3):
    """The batched expansion (d = 3 tiles of 8 targets a thread, accumulators in
    registers, or of 4 with them in shared memory, the shape the batched benchmark's
    autotuner picks) against single contexts and the batched difference form."""
    b = S.Batch(DESCS, precision=S.SSM_FP32C)
    b.set_plan(2, 8, r3, 4096)
    assert b.plan()["form"] == 2 and b.plan()["targets_per_thread_d3"] == r3
    b.run()
    c = S.Batch(DESCS, precision=S.SSM_FP32C)
    c.set_plan(1, 8, 8, 4096)
    c.run()
    for e, dsc in enumerate(DESCS):
        xb, nb = b.get_state(e)
        xc, _ = c.get_state(e)
        coef = S.SSM_COEF_COUPLED1D if dsc["d"] == 1 else S.SSM_COEF_COUPLED3D
        s = S.SSM(d=dsc["d"], N=dsc["N"], h=dsc["h"], T=dsc["T"], coef=coef, seed=dsc["seed"],
                  precision=S.SSM_FP32C)
        if dsc["d"] == 3:
            s.set_plan(0, 2, 128, 8)
            s.set_plan(1, 2, 128, 8)
        s.run()
        xs, ns = s.get_state()
        s.close()
        assert nb == ns == round(dsc["T"] / dsc["h"])
        assert np.max(np.abs(xb - xs)) < 1e-7, e
        assert np.max(np.abs(xb - xc)) < 1e-7, e
    b.close()
    c.close()


def test_batch_set_plan_rejects_unknown_shape(S):
    b = S.Batch(DESCS[:1], precision=S.SSM_FP32C)
    with pytest.raises(S.SSMError):
        b.set_plan(3, 8, 8, 4096)
    with pytest.raises(S.SSMError):
        b.set_plan(2, 8, 8, 5000)
    b.close()
    f = S.Batch(DESCS[:1], precision=S.SSM_FP64)
    with pytest.raises(S.SSMError):
        f.set_plan(2, 8, 8, 4096)
    f.close()


@pytest.mark.parametrize("N", [1, 2, 3, 7, 33, 129, 513])
def test_tiny_and_ragged_n_in_the_benchmark_shapes(S, N):
    """Degenerate and ragged sizes in the benchmark's shapes (step-1 sums 128 x 4,
    drift 128 x 8; one partly filled tile, N = 1 a single self-interacting
    particle), with T = h (a one-step horizon): Y and b of the step against the
    oracle, and no step past the horizon."""
    seed = 24
    s = S.SSM(d=3, N=N, h=H, T=H, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=S.SSM_FP32C)
    s.set_plan(0, 2, 128, 4)
    s.set_plan(1, 2, 128, 8)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, T=H, seed=seed)
    _check_one_step(S, s, P)
    x, n = s.get_state()
    assert n == 1 and np.all(np.isfinite(x))
    with pytest.raises(S.SSMError) as e:
        s.step()
    assert e.value.status == S.SSM_ESTATE
    s.close()
