"""The learned initial guess of step 1 (SSM_FP32C_LEARNED) on the GPU.

* network kernels vs the FP64 network oracle (forward outputs, gradients);
* training-row collection vs the SSM oracle (rebuilt X_n, moments, label S(Y*));
* GPU training lowers the loss;
* the learned start changes no root beyond the Newton tolerance (plain Newton is
  the judge), saves pair passes, and falls back to the plain start when it must.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M

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


def _rows(S, N, seed, steps, stride):
    s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=S.SSM_FP32C)
    fs, ls = [], []
    for n in range(steps):
        s.step()
        f, l = s.ws_collect(stride, n % stride)
        fs.append(f)
        ls.append(l)
    s.close()
    return np.concatenate(fs), np.concatenate(ls)


@pytest.fixture(scope="module")
def trained(S):
    """A network trained on the GPU from plain-SSM rows (N = 4096, seeds 100..103)."""
    parts = [_rows(S, 4096, sd, 64, 2) for sd in range(100, 104)]
    feat = np.concatenate([p[0] for p in parts])
    lab = np.concatenate([p[1] for p in parts])
    blob, curve = S.ssm_ws_train(feat, lab, epochs=8, batch=4096, lr=3e-3, seed=0)
    return blob, curve, feat, lab


def test_predict_matches_oracle_forward(S, trained):
    blob, _, feat, _ = trained
    f = feat[:: max(1, feat.shape[0] // 4000)]
    g = S.ssm_ws_predict(blob, f).astype(np.float64)
    o = M.forward(M.parse_blob(blob), f.astype(np.float64))
    assert np.max(np.abs(g - o)) <= 1e-5 * max(1.0, np.max(np.abs(o)))


def test_gradient_matches_oracle_backward(S, trained):
    _, _, feat, lab = trained
    p = M.random_params(5)
    fm, fs = feat.mean(0).astype(np.float64), np.maximum(feat.std(0), 1e-12).astype(np.float64)
    ym, ys = lab.mean(0).astype(np.float64), lab.std(0).astype(np.float64)
    blob = M.make_blob(p, fm, fs, ym, ys)
    rows = np.random.default_rng(1).choice(feat.shape[0], 3000, replace=False)
    g, loss = S.ssm_ws_grad(blob, feat[rows], lab[rows])
    q = M.parse_blob(blob)
    lo, go = M.loss_and_grad(q, feat[rows].astype(np.float64), lab[rows].astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go)) + 1e-7
    assert np.allclose(S.ssm_ws_params(blob), M.flatten(q), rtol=1e-7, atol=0)


def test_gpu_training_lowers_the_loss(trained):
    _, curve, _, _ = trained
    assert curve[-1] < 0.25 * curve[0], curve
    assert curve[-1] <= min(curve[:-1]) * 1.05


def test_collected_rows_match_the_ssm_oracle(S):
    N = 1500
    s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=21, precision=S.SSM_FP32C)
    s.step()
    x1, _ = s.get_state()
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    f, l = s.ws_collect(7, 3)
    s.close()
    idx = np.arange(3, N, 7)
    assert f.shape == (idx.size, 16)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=H, seed=21)
    assert np.max(np.abs(f[:, :3] - x1[idx])) < 1e-6 * max(1.0, np.abs(x1).max())
    assert np.allclose(f[:, 3:15], O.moments(P, x1).ravel()[None, :], rtol=1e-6, atol=1e-7)
    assert np.all(f[:, 15] == np.float32(H))
    for r, i in enumerate(idx[:40]):
        Sref, _ = O.pair_sum_coupled(P, x1, y[i])
        assert np.max(np.abs(l[r] - Sref)) < 1e-6


def _run(S, N, seed, steps, prec, blob=None, **opt):
    s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=prec, **opt)
    if blob is not None:
        s.ws_load(blob)
    s.run_steps(steps)
    x, _ = s.get_state()
    st = s.stats()
    s.close()
    return x, st


def test_learned_start_keeps_the_roots_and_saves_passes(S, trained):
    blob = trained[0]
    N, seed, K = 4096, 7, 24
    xp, sp = _run(S, N, seed, K, S.SSM_FP32C)
    xl, sl = _run(S, N, seed, K, S.SSM_FP32C_LEARNED, blob)
    # every root passes the same residual test: residual <= tol = 1e-10, or the FP32
    # forms' stagnation rule, which accepts up to 64 tol.  The implicit map is strongly
    # monotone (1 - h L_v ~ 1), so each step's roots of the two runs differ by at most
    # 2 x 64 tol, and over K steps by about K x 2 x 64 tol = 3.1e-7 (growth over T =
    # 3/32 is a few percent): far below the 1e-4 accuracy bar of the FP32 forms
    assert np.max(np.abs(xl - xp)) < 4e-7
    rows_plain, rows_learned = sp["newton_rows"] / K, sl["newton_rows"] / K
    print("pair rows per step: plain %.0f, learned %.0f (%.2fx); fallbacks %d"
          % (rows_plain, rows_learned, rows_plain / rows_learned, sl["fallbacks"]))
    assert rows_learned <= 0.9 * rows_plain
    assert sl["fallbacks"] <= 0.01 * N * K


def test_bad_network_falls_back_to_the_plain_start(S):
    """A network whose prediction is off by 1e6: in the first step every particle
    misses the tolerance within ws_passes passes and restarts from the plain start;
    from the second step on the start carries each particle's previous error, which
    cancels this network's constant offset, so no particle restarts.  Both runs reach
    the plain form's roots."""
    p = {n: np.zeros(s) for n, s in M.SHAPES}
    p["b4"] = np.array([1e6, -1e6, 1e6])
    blob = M.make_blob(p, np.zeros(16), np.ones(16), np.zeros(3), np.ones(3))
    N, seed, K = 1000, 9, 5
    xp, _ = _run(S, N, seed, K, S.SSM_FP32C)
    xl, sl = _run(S, N, seed, K, S.SSM_FP32C_LEARNED, blob, ws_passes=2)
    assert sl["fallbacks"] == N
    assert np.max(np.abs(xl - xp)) < 1e-8
    # without the carried error (dropped before every step) every step restarts
    s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=seed, precision=S.SSM_FP32C_LEARNED,
              ws_passes=2)
    s.ws_load(blob)
    for _ in range(K):
        s.pair_pass(2)                 # the start alone drops the carried error
        s.step()
    st = s.stats()
    x, _ = s.get_state()
    s.close()
    assert st["fallbacks"] == N * K
    assert np.max(np.abs(x - xp)) < 1e-8


def test_learned_form_without_weights_runs_plain(S):
    N, seed, K = 700, 4, 3
    xp, _ = _run(S, N, seed, K, S.SSM_FP32C)
    xl, sl = _run(S, N, seed, K, S.SSM_FP32C_LEARNED)
    assert np.array_equal(xl, xp) and sl["fallbacks"] == 0


def test_tensor_core_and_cuda_core_starts_agree(S):
    """The learned start on the tensor cores (mma.sync, BF16 activations) and on the
    CUDA cores (FFMA, FP32 activations), from the shipped network at N = 2^16: the two
    starts differ by the BF16 rounding of the activations only (well below the
    network's own error), and the steps that follow reach the same roots to the
    residual tolerance with the same pass counts."""
    N, K = 1 << 16, 3
    starts, runs = [], []
    for fwd in (0, 1):
        s = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2, precision=S.SSM_FP32C_LEARNED,
                  ws_forward=fwd)
        S.load_ws(s)
        s.pair_pass(2)                       # the learned start alone, from X_0 into Y
        starts.append(s.get_stage(S.SSM_STAGE_Y))
        s.run_steps(K)
        x, _ = s.get_state()
        runs.append((x, s.stats()))
        s.close()
    x0 = S.SSM(d=3, N=N, h=H, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=2).get_state()[0]
    move = np.max(np.abs(starts[1] - x0))          # the start's own step away from X
    assert move > 1e-3
    assert np.max(np.abs(starts[0] - starts[1])) < 2e-5
    assert np.max(np.abs(runs[0][0] - runs[1][0])) < K * 2 * 64 * 1e-10
    assert runs[0][1]["newton_passes"] == runs[1][1]["newton_passes"]
