"""Parity of the CUDA path with the FP64 CPU oracle, through the C ABI.

Tolerances (written per test):
  * integer work (Philox words) is bit-exact;
  * FP64 forms match per particle to 1e-10 relative, |a - b| <= 1e-10 max(1, |b|);
  * FP32-compensated forms match to 1e-4 absolute per particle at T and 1e-5 on
    the empirical mean and variance.
Sizes: small cases the oracle finishes in seconds over the full horizon (several
tiles, ragged tails), plus the full workload sizes checked step by step on
sampled particles, which the oracle computes one at a time.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import inputs

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


# ---------------------------------------------------------------------------
# Components
# ---------------------------------------------------------------------------

def test_philox_bit_exact(S):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xffffffff] * 4, [5, 6, 7, 8]]
    for seed in (0, 1, 0xa4093822299f31d0, 2 ** 64 - 1):
        key = np.array([seed & 0xffffffff, seed >> 32], dtype=np.uint32)
        assert np.array_equal(S.ssm_philox(seed, ctr), O.philox(ctr, key))


def test_philox_known_answer(S):
    """The published Philox4x32-10 vectors through the device kernel (key words are
    (seed mod 2^32, seed >> 32))."""
    rows = [([0, 0, 0, 0], 0, [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
            ([0xffffffff] * 4, 2 ** 64 - 1, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
            ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], (0x299f31d0 << 32) | 0xa4093822,
             [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1])]
    for ctr, seed, want in rows:
        assert [int(v) for v in S.ssm_philox(seed, [ctr])[0]] == want


@pytest.mark.parametrize("d", [1, 2, 3])
def test_normals_match_oracle(S, d):
    N, step, stream, seed = 3001, 17, 1, 99
    g = S.ssm_normals(seed, d, N, step, stream)
    o = np.array([O.normals(seed, d, i, step, stream) for i in range(N)])
    assert np.max(np.abs(g - o)) < 1e-13


def test_cardano_matches_oracle(S):
    xs = np.concatenate([inputs.uniform_points(5000, -6, 6, seed=4), [0.0, 1e-300, -1e-12, 7.5, -7.5]])
    for h in (0.01, 2.0 ** -10, 0.3):
        g = S.ssm_cardano(xs, h)
        o = np.array([O.cardano(v, h) for v in xs])
        assert np.all(np.abs(g - o) <= 4e-16 * np.maximum(np.abs(o), 1e-300) + 1e-320)


def test_empty_component_calls(S):
    assert S.ssm_philox(0, np.zeros((0, 4), np.uint32)).shape == (0, 4)
    assert S.ssm_cardano(np.zeros(0), 0.01).shape == (0,)


# ---------------------------------------------------------------------------
# Whole runs over [0, T], FP64
# ---------------------------------------------------------------------------

def _gpu_run(S, d, N, h, coef, seed, steps=None, **opt):
    s = S.SSM(d=d, N=N, h=h, T=1.0, coef=coef, seed=seed, **opt)
    if steps is None:
        s.run()
    else:
        s.run_steps(steps)
    x, n = s.get_state()
    m = s.moments()
    st = s.stats()
    s.close()
    return x, n, m, st


def test_config0_cubic1d_full_horizon_fp64(S):
    """N = 1000, h = 1/100, T = 1, seed 0: per particle 1e-10 relative."""
    N, h = 1000, 0.01
    x, n, m, _ = _gpu_run(S, 1, N, h, S.SSM_COEF_CUBIC1D_GAUSS, 0)
    P = O.problem(d=1, coef=O.COEF_CUBIC1D_GAUSS, N=N, h=h, seed=0)
    xo = O.run(P, O.init_x0(P), 0, 100)
    assert n == 100
    assert relerr(x, xo) < 1e-10
    assert relerr(m, O.moments(P, xo)) < 1e-10


def test_config1_cubic1d_ragged_full_horizon_fp64(S):
    """Config-1 coefficients and h = 2^-10 over T = 1 at N = 2000 (ragged tiles)."""
    N, h = 2000, 2.0 ** -10
    x, n, _, _ = _gpu_run(S, 1, N, h, S.SSM_COEF_CUBIC1D_GAUSS, 1)
    P = O.problem(d=1, coef=O.COEF_CUBIC1D_GAUSS, N=N, h=h, seed=1)
    xo = O.run(P, O.init_x0(P), 0, 1024)
    assert relerr(x, xo) < 1e-10


def _sampled_step_check(S, s, P, n_samples, tol_y, tol_x, seed=0):
    """One step on the GPU; for sampled particles the oracle recomputes Y_i from
    the GPU's X_n (all particles) and X_{n+1,i} from the GPU's Y (all particles)."""
    x0, n = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    x1, _ = s.get_state()
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, P.N - 1], rng.integers(0, P.N, n_samples)]))
    ey = ex = 0.0
    for i in idx:
        yo, it = O.implicit_one(P, x0, int(i))
        assert it >= 0
        ey = max(ey, relerr(y[i], yo))
        xo = O.explicit_one(P, y, int(i), n)
        ex = max(ex, relerr(x1[i], xo))
    assert ey < tol_y, ey
    assert ex < tol_x, ex
    return x1


def test_config1_full_size_sampled_fp64(S):
    """N = 65536, h = 2^-10, seed 1: two steps checked on sampled particles."""
    N, h = 65536, 2.0 ** -10
    s = S.SSM(d=1, N=N, h=h, T=1.0, coef=S.SSM_COEF_CUBIC1D_GAUSS, seed=1)
    P = O.problem(d=1, coef=O.COEF_CUBIC1D_GAUSS, N=N, h=h, seed=1)
    xg, _ = s.get_state()
    assert np.array_equal(xg, O.init_x0(P)) or relerr(xg, O.init_x0(P)) < 1e-14
    for _ in range(2):
        _sampled_step_check(S, s, P, 48, 1e-14, 1e-10)
    s.close()


@pytest.mark.parametrize("N", [1, 2, 3, 7, 33, 300, 777])
def test_coupled3d_fp64_small_and_ragged(S, N):
    h = 2.0 ** -8
    x, n, _, _ = _gpu_run(S, 3, N, h, S.SSM_COEF_COUPLED3D, 5, steps=6)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=5)
    xo = O.run(P, O.init_x0(P), 0, 6)
    assert relerr(x, xo) < 1e-10


def test_coupled3d_fp64_full_horizon(S):
    """Coupled implicit drift, N = 640, h = 2^-8, T = 1 (256 steps): 1e-10 relative."""
    N, h = 640, 2.0 ** -8
    x, n, m, st = _gpu_run(S, 3, N, h, S.SSM_COEF_COUPLED3D, 2)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    xo, mo, _ = O.run(P, O.init_x0(P), 0, 256, want_moments=True)
    assert n == 256
    assert relerr(x, xo) < 1e-10
    assert relerr(m, mo[-1]) < 1e-10
    assert st["steps"] == 256 and st["max_passes"] < 12


def test_ou_matches_oracle(S):
    N, h = 777, 2.0 ** -6
    opt = dict(coef_params=(-1.0, 0.5, 0.5), x0_mean=1.0, x0_std=0.5)
    x, n, _, _ = _gpu_run(S, 2, N, h, S.SSM_COEF_OU, 4, **opt)
    P = O.problem(d=2, coef=O.COEF_OU, N=N, h=h, seed=4, p=(-1.0, 0.5, 0.5), x0_mean=1.0, x0_std=0.5)
    xo = O.run(P, O.init_x0(P), 0, 64)
    assert relerr(x, xo) < 1e-12


def test_fine_brownian_grid(S):
    """dW summed from the grid T 2^-6 at h = 2^-4 (shared Brownian path, §3)."""
    N, h = 100, 2.0 ** -4
    x, n, _, _ = _gpu_run(S, 1, N, h, S.SSM_COEF_CUBIC1D_GAUSS, 8, fine_log2=6)
    P = O.problem(d=1, coef=O.COEF_CUBIC1D_GAUSS, N=N, h=h, seed=8, fine_log2=6)
    xo = O.run(P, O.init_x0(P), 0, 16)
    assert relerr(x, xo) < 1e-10


# ---------------------------------------------------------------------------
# FP32-compensated form of the coupled workload
# ---------------------------------------------------------------------------

def test_coupled3d_fp32c_full_horizon_tolerances(S):
    """N = 1536, h = 2^-8, T = 1: <= 1e-4 absolute per particle, <= 1e-5 on mean and variance."""
    N, h = 1536, 2.0 ** -8
    x, n, m, st = _gpu_run(S, 3, N, h, S.SSM_COEF_COUPLED3D, 2, precision=S.SSM_FP32C)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    xo = O.run(P, O.init_x0(P), 0, 256)
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert np.max(np.abs(m[0] - mo[0])) < 1e-5
    var_g, var_o = m[1] - m[0] ** 2, mo[1] - mo[0] ** 2
    assert np.max(np.abs(var_g - var_o)) < 1e-5


@pytest.mark.parametrize("shape", [(1, 128, 4), (1, 256, 8), (1, 128, 8), (2, 128, 4), (2, 256, 8), (0, 256, 2), (0, 128, 8)])
def test_coupled3d_fp32c_every_launch_shape(S, shape):
    """Packed and scalar FP32 pair kernels of each compiled shape give the oracle's
    result within FP32-compensated accuracy (N = 1000: ragged tiles and chunks):
    the first step's Y (step 1) and b (step 2) element by element, then the state
    after 8 steps, which also carries the FP32 normals of step 2 (|dz| < 5e-6, so
    |dx| < sigma sqrt(h) 5e-6 <= 1.2 * 2^-4 * 5e-6 = 3.8e-7 per step)."""
    N, h, K = 1000, 2.0 ** -8, 8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=11, precision=S.SSM_FP32C)
    s.set_plan(0, *shape)
    s.set_plan(1, *shape)
    assert s.plan(0)["form"] == shape[0] and s.plan(0)["targets_per_thread"] == shape[2]
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=11)
    x0, _ = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    b = s.get_stage(S.SSM_STAGE_B)
    yo, it, bad = O.implicit_step(P, x0)
    assert bad == 0 and relerr(y, yo) < 2e-9
    bo = np.stack([O.drift_one(P, y, i) for i in range(N)])
    assert np.max(np.abs(b - bo)) < 5e-7
    s.run_steps(K - 1)
    x, _ = s.get_state()
    s.close()
    xo = O.run(P, O.init_x0(P), 0, K)
    assert np.max(np.abs(x - xo)) < K * 3.8e-7


def test_autotune_changes_shape_not_results(S):
    """The tuned shape and chunk count sum the pair terms in another order; both runs
    pass the same residual test (each root within 64 tol of the exact one under the
    FP32 forms' stagnation rule), so K steps differ by at most K x 2 x 64 tol."""
    N, h, K = 5000, 2.0 ** -8, 3
    runs = []
    for tune in (False, True):
        s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=12, precision=S.SSM_FP32C)
        if tune:
            best = s.autotune()
            assert np.all(best > 0)
        s.run_steps(K)
        runs.append(s.get_state()[0])
        s.close()
    tol = max(1e-10, 2.0 ** -27 * h * (1.0 + 64.0 / math.sqrt(N)))
    assert np.max(np.abs(runs[0] - runs[1])) < K * 2 * 64 * tol


@pytest.mark.parametrize("chunks", [1, 2, 5, 40])
def test_source_chunks_change_grouping_not_results(S, chunks):
    """A pair pass splits the sources of every target tile into chunks, one set of
    partial sums each, added by the consumer in chunk order.  With another chunk
    count (ssm_opts.tile_chunks; 40 is capped at one 512-source sub-tile a chunk, and
    the step-1 passes over part of the particles re-pack their blocks into more
    chunks) the sums are grouped differently, but the step-1 roots pass the same
    residual test: the first step's Y within 1e-9 of the planned launch's; b, the
    FP32 drift at those two Y (each within 5e-7 of the oracle's, the bound of
    test_coupled3d_fp32c_every_launch_shape), within 1e-6; the state after 3 steps
    within 3 x 2 x 64 tol (N = 3000: a ragged last tile and a ragged last chunk)."""
    N, h, K = 3000, 2.0 ** -8, 3
    out = []
    for k in (0, chunks):
        s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=13, precision=S.SSM_FP32C, tile_chunks=k)
        s.set_plan(0, 2, 128, 4)
        s.set_plan(1, 2, 128, 8)
        if k:   # chunks of whole 512-source sub-tiles, at most one per 256 sources
            want = min(k, -(-N // 256))
            length = -(-(-(-N // want)) // 512) * 512
            assert s.plan(0)["chunks"] == -(-N // length)
        s.step()
        y, b = s.get_stage(S.SSM_STAGE_Y), s.get_stage(S.SSM_STAGE_B)
        s.run_steps(K - 1)
        out.append((y, b, s.get_state()[0]))
        s.close()
    (y0, b0, x0), (y1, b1, x1) = out
    tol = max(1e-10, 2.0 ** -27 * h * (1.0 + 64.0 / math.sqrt(N)))
    assert np.max(np.abs(y0 - y1)) < 1e-9
    assert np.max(np.abs(b0 - b1)) < 1e-6
    assert np.max(np.abs(x0 - x1)) < K * 2 * 64 * tol


def test_tuning_cache_restores_the_tuned_plan(S, tmp_path):
    """A second context of the same workload takes the tuned plans from the JSON cache
    (ssm_set_plan_chunks, no tuning): the same shapes and chunk counts, and the same
    states bit for bit after a few steps."""
    N, h, K = 5000, 2.0 ** -8, 2
    cache = str(tmp_path / "tune.json")
    runs = []
    for _ in range(2):
        s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=14, precision=S.SSM_FP32C)
        best = s.autotune(cache=cache)
        assert np.all(best > 0)
        plans = (s.plan(0), s.plan(1))
        s.run_steps(K)
        runs.append((plans, s.get_state()[0]))
        s.close()
    assert len(S.tune_cache_load(cache)) == 1
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_set_plan_chunks_rejects_out_of_range(S):
    s = S.SSM(d=3, N=3000, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=1, precision=S.SSM_FP32C)
    for bad in (0, -1, 10 ** 6):
        with pytest.raises(S.SSMError):
            S.ssm_set_plan_chunks(s.ctx, 0, 2, 128, 4, bad)
    with pytest.raises(S.SSMError):
        S.ssm_set_plan_chunks(s.ctx, 0, 2, 96, 4, 3)   # not a compiled shape
    s.set_plan(0, 2, 128, 4, chunks=3)
    assert s.plan(0)["chunks"] == 3
    s.close()


def test_carried_start_keeps_the_roots_and_saves_a_pass(S):
    """ssm_opts.carry_start: from the second step on, step 1 starts from the previous
    step's converged pair sums.  The FP64 form still matches the oracle to 1e-10 per
    particle after 12 steps; in the FP32C form every root passes the same residual
    test as from the plain start (within K x 2 x 64 tol of the plain run after K
    steps), with at most 80% of its pair rows."""
    N, h, K = 640, 2.0 ** -8, 12
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=15, carry_start=1)
    s.run_steps(K)
    x, _ = s.get_state()
    st = s.stats()
    s.close()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=15)
    xo = O.run(P, O.init_x0(P), 0, K)
    assert relerr(x, xo) < 1e-10
    N, K = 4096, 24
    runs = []
    for carry in (0, 1):
        s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=16, precision=S.SSM_FP32C, carry_start=carry)
        s.run_steps(K)
        runs.append((s.get_state()[0], s.stats()))
        s.close()
    (xp, sp), (xc, sc) = runs
    tol = max(1e-10, 2.0 ** -27 * h * (1.0 + 64.0 / math.sqrt(N)))
    assert np.max(np.abs(xc - xp)) < K * 2 * 64 * tol
    print("pair rows per step: plain %.0f, carried start %.0f" % (sp["newton_rows"] / K, sc["newton_rows"] / K))
    assert sc["newton_rows"] <= 0.8 * sp["newton_rows"]


def test_carried_start_is_rejected_where_it_does_not_apply(S):
    for kw in (dict(coef=S.SSM_COEF_OU, d=3), dict(coef=S.SSM_COEF_CUBIC1D_GAUSS, d=1),
               dict(coef=S.SSM_COEF_COUPLED3D, d=3, precision=S.SSM_FP32C_LEARNED),
               dict(coef=S.SSM_COEF_COUPLED3D, d=3, measure_y=1), dict(coef=S.SSM_COEF_COUPLED3D, d=3, carry_start=2)):
        kw.setdefault("carry_start", 1)
        with pytest.raises(S.SSMError):
            S.SSM(N=100, h=2.0 ** -8, T=1.0, seed=1, **kw)


def test_set_plan_rejects_unknown_shape(S):
    s = S.SSM(d=3, N=100, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=1)   # FP64: no packed kernels
    with pytest.raises(S.SSMError):
        s.set_plan(0, 1, 128, 4)
    with pytest.raises(S.SSMError):
        s.set_plan(0, 0, 96, 4)
    s.close()


def test_coupled3d_full_size_sampled_fp32c(S):
    """N = 2^18, h = 2^-8, seed 2 (the benchmark workload): one step, sampled."""
    N, h = 1 << 18, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2, precision=S.SSM_FP32C)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    _sampled_step_check(S, s, P, 24, 2e-9, 6e-7)   # x: + sigma sqrt(h) |dz| < 3.8e-7 from the FP32 normals
    st = s.stats()
    assert sum(st["hist"]) == N
    s.close()


@pytest.mark.parametrize("learned", [False, True])
def test_coupled3d_full_size_sampled_bench_configuration(S, learned):
    """N = 2^18, h = 2^-8, seed 2 in the launch configuration the benchmark times:
    step-1 sums on the packed expansion with 128 threads x 4 targets (two-sum
    accumulators in shared memory), the drift with 128 x 8, plain FP32C and the
    learned form (the shipped network): one step, sampled."""
    N, h = 1 << 18, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2,
              precision=S.SSM_FP32C_LEARNED if learned else S.SSM_FP32C)
    if learned:
        S.load_ws(s)
    s.set_plan(0, 2, 128, 4)
    s.set_plan(1, 2, 128, 8)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    _sampled_step_check(S, s, P, 24, 2e-9, 6e-7)
    s.close()


def test_coupled3d_learned_full_horizon_tolerances(S):
    """The learned + FP32C form (the shipped network) over the whole horizon against
    the FP64 oracle: N = 4096, h = 2^-8, T = 1 (256 steps), seed 2.  Bars: <= 1e-4
    absolute per particle at T and <= 1e-5 on the empirical mean and variance.  The
    learned start sees the late-time distribution of X here, not only X_0."""
    N, h = 4096, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2, precision=S.SSM_FP32C_LEARNED)
    S.load_ws(s)
    s.run()
    x, n = s.get_state()
    m = s.moments()
    st = s.stats()
    s.close()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    xo = O.run(P, O.init_x0(P), 0, 256)
    assert n == 256
    assert np.max(np.abs(x - xo)) < 1e-4
    mo = O.moments(P, xo)
    assert np.max(np.abs(m[0] - mo[0])) < 1e-5
    var_g, var_o = m[1] - m[0] ** 2, mo[1] - mo[0] ** 2
    assert np.max(np.abs(var_g - var_o)) < 1e-5
    # every implicit solve ended within the pass limit; the learned start saved passes
    assert st["steps"] == 256 and st["max_passes"] < 12
    assert st["newton_rows"] < 3 * N * 256
    print("learned N=4096 to T: max|dx| %.3e, passes %d, rows/step %.1f, fallbacks %d, floor accepts %d"
          % (np.max(np.abs(x - xo)), st["newton_passes"], st["newton_rows"] / 256, st["fallbacks"],
             st["floor_accepts"]))


@pytest.mark.parametrize("n_at", [128, 255])
def test_coupled3d_learned_full_size_late_steps_sampled(S, n_at):
    """N = 2^18 in the benchmark's launch configuration, learned form: the GPU runs
    to step n_at, then one more step is checked on sampled particles against the
    oracle from the GPU's own X_n (the late-time distribution the learned start
    meets in the benchmark)."""
    N, h = 1 << 18, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2, precision=S.SSM_FP32C_LEARNED)
    S.load_ws(s)
    s.set_plan(0, 2, 128, 4)
    s.set_plan(1, 2, 128, 8)
    s.run_steps(n_at)
    st0 = s.stats()
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    _sampled_step_check(S, s, P, 24, 2e-9, 6e-7, seed=n_at)
    st1 = s.stats()
    assert st1["steps"] == n_at + 1
    print("learned N=2^18 step %d: passes %d, rows %d, fallbacks %d, floor accepts %d (over the first %d steps: %d)"
          % (n_at, st1["newton_passes"] - st0["newton_passes"], st1["newton_rows"] - st0["newton_rows"],
             st1["fallbacks"] - st0["fallbacks"], st1["floor_accepts"] - st0["floor_accepts"], n_at,
             st0["floor_accepts"]))
    s.close()


def test_coupled3d_full_size_sampled_fp64(S):
    """N = 2^18 in FP64: one step, sampled, 1e-10 relative."""
    N, h = 1 << 18, 2.0 ** -8
    s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, seed=2)
    _sampled_step_check(S, s, P, 16, 1e-10, 1e-10)
    s.close()


# ---------------------------------------------------------------------------
# Host logic through the device: graphs, resume, invariants
# ---------------------------------------------------------------------------

def test_graph_replay_equals_single_steps_and_resume_is_bit_exact(S):
    N, h = 500, 2.0 ** -8
    a = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=9, precision=S.SSM_FP32C)
    a.run_steps(10)
    xa, _ = a.get_state()
    b = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=9, precision=S.SSM_FP32C)
    for _ in range(4):
        b.step()
    x4, n4 = b.get_state()
    c = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=9, precision=S.SSM_FP32C)
    c.set_state(x4, n4)
    c.run_steps(6)
    xc, nc = c.get_state()
    assert nc == 10 and np.array_equal(xa, xc)
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("learned", [False, True])
def test_device_pass_loop_equals_fixed_pass_launches(S, learned):
    """The step-1 passes as a device-driven conditional graph node (default) and as a
    fixed sequence of newton_kmax pass launches (ssm_opts.fixed_pass_launches) run the
    same kernels on the same data: bit-identical states and equal work counters."""
    N, h, K = 3000, 2.0 ** -8, 5
    prec = S.SSM_FP32C_LEARNED if learned else S.SSM_FP32C
    out = []
    for fixed in (0, 1):
        s = S.SSM(d=3, N=N, h=h, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=13, precision=prec,
                  fixed_pass_launches=fixed)
        if learned:
            S.load_ws(s)
        s.step()                      # ssm_step and ssm_run_steps share the step graph
        s.run_steps(K - 1)
        x, n = s.get_state()
        st = s.stats()
        s.close()
        out.append((x, n, st))
    (xa, na, sa), (xb, nb, sb) = out
    assert na == nb == K and np.array_equal(xa, xb)
    for k in ("newton_passes", "newton_rows", "fallbacks", "floor_accepts", "max_passes"):
        assert sa[k] == sb[k], k


@pytest.mark.parametrize("prec", [0, 1])
def test_drift_stage_is_antisymmetric(S, prec):
    N = 3000
    s = S.SSM(d=3, N=N, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=3, precision=prec)
    s.step()
    b = s.get_stage(S.SSM_STAGE_B)
    assert np.all(np.abs(b.sum(axis=0)) < N * (1e-15 if prec == 0 else 1e-6) * np.abs(b).max())
    s.close()


def test_step_past_horizon_is_rejected(S):
    s = S.SSM(d=1, N=10, h=0.25, T=0.5, coef=S.SSM_COEF_CUBIC1D_GAUSS, seed=0)
    s.run()
    with pytest.raises(S.SSMError) as e:
        s.step()
    assert e.value.status == S.SSM_ESTATE
    s.close()
