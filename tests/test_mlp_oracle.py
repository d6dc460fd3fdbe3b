"""Pins of the FP64 network oracle (learned initial guess), CPU only.

The backward pass is checked against central finite differences of the loss; the
blob writer/reader round-trips parameters through BF16 rounding; a network with
zero weights outputs its bias, unstandardised.
"""
import numpy as np

from oracle import mlp as M


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 16)) * 0.7 + 0.2, rng.standard_normal((n, 3)) * 0.3


def test_backward_matches_central_differences():
    p = M.random_params(1)
    p["fm"], p["fs"] = np.full(16, 0.1), np.full(16, 1.3)
    p["ym"], p["ys"] = np.array([0.01, -0.02, 0.03]), np.array([0.2, 0.3, 0.25])
    feat, label = _data(40, 2)
    loss, g = M.loss_and_grad(p, feat, label)
    v = M.flatten(p)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(M.NPARAM, 60, replace=False), [0, M.NPARAM - 1, 1024, 1088]])
    eps = 1e-6
    for k in idx:
        vp, vm = v.copy(), v.copy()
        vp[k] += eps
        vm[k] -= eps
        pp, pm = dict(p, **M.unflatten(vp)), dict(p, **M.unflatten(vm))
        fd = (M.loss_only(pp, feat, label) - M.loss_only(pm, feat, label)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, g[k])
    assert abs(loss - M.loss_only(p, feat, label)) < 1e-15


def test_zero_weights_give_the_unstandardised_bias():
    p = {n: np.zeros(s) for n, s in M.SHAPES}
    p["b4"] = np.array([0.5, -1.0, 2.0])
    blob = M.make_blob(p, np.zeros(16), np.ones(16), np.array([1.0, 2.0, 3.0]), np.array([2.0, 2.0, 2.0]))
    q = M.parse_blob(blob)
    out = M.forward(q, np.random.default_rng(0).standard_normal((5, 16)))
    assert np.allclose(out, [2.0, 0.0, 7.0])   # b4 * ys + ym


def test_blob_round_trip_rounds_weights_to_bf16():
    p = M.random_params(4)
    blob = M.make_blob(p, np.zeros(16), np.ones(16), np.zeros(3), np.ones(3))
    assert len(blob) == M.BLOB_WORDS * 4
    q = M.parse_blob(blob)
    for n in ("W1", "W2", "W3", "W4"):
        rel = np.abs(q[n] - p[n]) / np.maximum(np.abs(p[n]), 1e-30)
        assert np.all(rel <= 2.0 ** -8)            # BF16: 8 significant bits
        assert np.any(q[n] != p[n])
    for n in ("b1", "b2", "b3", "b4"):
        assert np.allclose(q[n], p[n], rtol=1e-7)  # biases stay FP32
