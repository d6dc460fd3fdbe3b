"""Pins of three oracle functions that the GPU tests use as judges, each against
facts that do not come from the function itself (CPU only, no GPU marker):

* ``orc_moments`` (the raw empirical moments (1/N) sum_i x_{i,c}^k, k = 1..4, of
  the empirical measure of §2.3 that the learned start and the moment checks read):
  hand-worked values on small point sets, the exact scaling m_k(a x) = a^k m_k(x),
  and the Gaussian moments E Z^2 = 1, E Z^4 = 3 within their standard errors.
* ``orc_joint_residual_one`` (G_i = Y_i - X_i - h v(Y_i, mu^Y), the joint system of
  the earlier implicit scheme that §1 contrasts with the SSM): zero at the 40-digit
  fixed point of a tiny system and at the closed-form root of a single particle;
  the pair parts cancel in the sum over i; and at the SSM's own root (measure mu^X)
  it equals h/2 (S^X_i - S^Y_i), the gap between the two measures.
* ``oracle/mlp.py`` ``forward`` (the learned start's network: SiLU hidden layers,
  standardised features in, standardised labels out): hand-computed outputs of a
  one-path network with unit weights, the order of both standardisations, and a
  linear output layer.

Each group also runs its checks on deliberately wrong variants of the function
(a power k+1 for k, a dropped or sign-flipped pair term, another activation or a
swapped standardisation) and requires every variant to fail, so the pins are
shown to catch those slips.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from tests import inputs


# ---------------------------------------------------------------------------
# orc_moments
# ---------------------------------------------------------------------------

# Hand-worked moments, one column per coordinate:
#   column 0: {0, 1, 2, 3}    m_k = (0 + 1 + 2^k + 3^k) / 4 = 1.5, 3.5, 9, 24.5
#   column 1: {-1, 1, -1, 1}  m_k = 0, 1, 0, 1
#   column 2: {2, 2, 2, 2}    m_k = 2^k = 2, 4, 8, 16
_PTS = np.array([[0.0, -1.0, 2.0], [1.0, 1.0, 2.0], [2.0, -1.0, 2.0], [3.0, 1.0, 2.0]])
_WANT = np.array([[1.5, 0.0, 2.0], [3.5, 1.0, 4.0], [9.0, 0.0, 8.0], [24.5, 1.0, 16.0]])


def _oracle_moments(x):
    P = O.problem(d=x.shape[1], coef=O.COEF_OU, N=x.shape[0], h=0.01)
    return O.moments(P, x)


def _moment_pins_hold(fn):
    """True when fn(x) -> [4, d] meets every moment pin."""
    if not np.array_equal(fn(_PTS), _WANT):                 # exact: small integers
        return False
    x = inputs.gaussian_cloud(257, 3, seed=61)
    m, ms = fn(x), fn(-0.5 * x)
    for k in range(4):                                      # m_k(a x) = a^k m_k(x), a = -1/2
        if not np.allclose(ms[k], (-0.5) ** (k + 1) * m[k], rtol=1e-13, atol=1e-15):
            return False
    return True


def test_moments_hand_worked_and_scaling():
    assert _moment_pins_hold(_oracle_moments)


def test_moments_of_gaussian_particles():
    """X_0 ~ N(0, I_3): m_1 = 0, m_2 = 1, m_3 = 0, m_4 = 3 within 5 standard errors
    (the variances of Z^k are 1, 2, 15, 96)."""
    N = 1 << 16
    P = O.problem(d=3, coef=O.COEF_OU, N=N, h=0.01, seed=77)
    m = O.moments(P, O.init_x0(P))
    for k, (mu, var) in enumerate(((0.0, 1.0), (1.0, 2.0), (0.0, 15.0), (3.0, 96.0))):
        assert np.all(np.abs(m[k] - mu) < 5.0 * math.sqrt(var / N)), (k, m[k])


def test_moment_pins_reject_planted_slips():
    def power_shift(x):      # x^(k+2) where x^(k+1) is meant
        return np.array([np.mean(x ** (k + 2), axis=0) for k in range(4)])

    def bessel(x):           # 1/(N-1) instead of the measure's 1/N
        return np.array([np.sum(x ** (k + 1), axis=0) / (x.shape[0] - 1) for k in range(4)])

    def transposed(x):       # coordinates taken in reverse order
        return np.array([np.mean(x[:, ::-1] ** (k + 1), axis=0) for k in range(4)])

    for bad in (power_shift, bessel, transposed):
        assert not _moment_pins_hold(bad), bad.__name__


# ---------------------------------------------------------------------------
# orc_joint_residual_one
# ---------------------------------------------------------------------------

def _oracle_g(P, x, y, i):
    return O.joint_residual_one(P, x, y, i)


def _fixed_point_40(x, h):
    """Root of Y_i = X_i + h(-Y_i|Y_i|^2 + (1/(2N)) sum_j (Y_j - Y_i)/(1 + |Y_j - Y_i|^2))
    by the contraction iterated in 40-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    N, d = x.shape
    X = [[mp.mpf(float(v)) for v in row] for row in x]
    Y = [list(r) for r in X]
    for _ in range(200):
        new = []
        for i in range(N):
            r2 = sum(c * c for c in Y[i])
            S = [mp.mpf(0)] * d
            for j in range(N):
                dd = [Y[j][a] - Y[i][a] for a in range(d)]
                w = 1 / (1 + sum(c * c for c in dd))
                S = [S[a] + dd[a] * w for a in range(d)]
            new.append([X[i][a] + h * (-Y[i][a] * r2 + S[a] / (2 * N)) for a in range(d)])
        Y = new
    return np.array([[float(c) for c in row] for row in Y])


def _joint_pins_hold(g):
    """True when g(P, x, y, i) meets every pin of the joint residual."""
    h = 2.0 ** -6
    # (1) zero at the 40-digit root of a three-particle system (d = 3 and d = 1)
    for d, coef in ((3, O.COEF_COUPLED3D), (1, O.COEF_COUPLED1D)):
        x = inputs.gaussian_cloud(3, d, seed=62)
        y = _fixed_point_40(x, h)
        P = O.problem(d=d, coef=coef, N=3, h=h, measure_y=1)
        if max(np.max(np.abs(g(P, x, y, i))) for i in range(3)) > 1e-15:
            return False
    # (2) one particle: no pair term, Y = s X with s the real root of h|X|^2 s^3 + s = 1
    x1 = np.array([[1.3, -0.7, 2.1]])
    s = O.cardano_gl(1.0, h * float(np.dot(x1[0], x1[0])))
    P1 = O.problem(d=3, coef=O.COEF_COUPLED3D, N=1, h=h, measure_y=1)
    if np.max(np.abs(g(P1, x1, s * x1, 0))) > 1e-15:
        return False
    # (3) at any Y the pair parts cancel: sum_i G_i = sum_i (Y_i - X_i + h Y_i |Y_i|^2)
    N = 40
    x = inputs.gaussian_cloud(N, 3, seed=63)
    y = x + 0.3 * inputs.gaussian_cloud(N, 3, seed=64)
    P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h, measure_y=1)
    tot = sum(g(P, x, y, i) for i in range(N))
    local = np.sum(y - x + h * y * np.sum(y * y, axis=1, keepdims=True), axis=0)
    if np.max(np.abs(tot - local)) > 1e-13:
        return False
    # (4) at the SSM's root (step 1 against mu^X) G_i = h/2 (S^X_i - S^Y_i)
    Px = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=h)
    ys, _, bad = O.implicit_step(Px, x)
    assert bad == 0
    for i in (0, 7, N - 1):
        sx, _ = O.pair_sum_coupled(Px, x, ys[i])
        sy, _ = O.pair_sum_coupled(Px, ys, ys[i])
        if np.max(np.abs(g(P, x, ys, i) - 0.5 * h * (sx - sy))) > 1e-15:
            return False
    return True


def test_joint_residual_pins():
    assert _joint_pins_hold(_oracle_g)


def _g_variant(sign=1.0, self_skip_norm=False, src_x=False):
    """A deliberately wrong joint residual: pair term with the sign flipped, divided
    by N - 1, or taken against X instead of Y (for the slip checks only)."""
    def g(P, x, y, i):
        d = x.shape[1]
        src = x if src_x else y
        dd = src - y[i]
        w = 1.0 / (1.0 + np.sum(dd * dd, axis=1, keepdims=True))
        N = x.shape[0]
        S = np.sum(dd * w, axis=0) / ((N - 1) if (self_skip_norm and N > 1) else N)
        return y[i] - x[i] - P.h * (-y[i] * float(np.dot(y[i], y[i])) + 0.5 * sign * S[:d])
    return g


def test_joint_residual_pins_reject_planted_slips():
    pytest.importorskip("mpmath")
    assert _joint_pins_hold(_g_variant())          # the variant machinery itself is sound
    for bad in (_g_variant(sign=-1.0), _g_variant(self_skip_norm=True), _g_variant(src_x=True)):
        assert not _joint_pins_hold(bad)


# ---------------------------------------------------------------------------
# oracle/mlp.py forward
# ---------------------------------------------------------------------------

# Logistic sigma(s) = 1/(1 + e^-s) and SiLU(s) = s sigma(s), evaluated to 30 digits:
SILU_1 = 0.731058578630004879251159241822      # SiLU(1) = sigma(1)
SILU_M1 = -0.268941421369995120748840758178    # SiLU(-1) = -sigma(-1)
SILU_2 = 1.76159415595576488811945828260       # SiLU(2) = 2 sigma(2)
SILU_3X = 0.306423334019726887718340782662     # SiLU(SiLU(SiLU(1)))
SILU_3X_M1 = -0.0548592440071005351912440078478   # SiLU(SiLU(SiLU(-1)))
SILU_3X_2 = 1.2298620380264055409498916794        # SiLU(SiLU(SiLU(2)))


def _one_path(fm0=1.0, fs0=2.0, ys=(2.0, 3.0, 4.0), ym=(10.0, 20.0, 30.0), w4=(1.0, -2.0, 0.5)):
    """Network whose only path is feature 0 -> unit 0 -> unit 0 -> unit 0 -> outputs,
    all weights +-1, +-2 or 1/2 (exact in BF16), zero biases."""
    p = {n: np.zeros(s) for n, s in M.SHAPES}
    p["W1"][0, 0] = p["W2"][0, 0] = p["W3"][0, 0] = 1.0
    p["W4"][:, 0] = w4
    fm, fs = np.zeros(16), np.ones(16)
    fm[0], fs[0] = fm0, fs0
    return M.parse_blob(M.make_blob(p, fm, fs, np.array(ym), np.array(ys)))


def _mlp_pins_hold(forward):
    """True when forward(params, feat) meets every pin of the network oracle."""
    q = _one_path()
    # feature 0 = 3 standardises to (3 - 1)/2 = 1; three SiLU layers; output
    # raw * ys + ym with raw = w4 * SiLU(SiLU(SiLU(1)))
    f = np.zeros((1, 16))
    f[0, 0] = 3.0
    want = np.array([1.0, -2.0, 0.5]) * SILU_3X * np.array([2.0, 3.0, 4.0]) + np.array([10.0, 20.0, 30.0])
    if not np.allclose(forward(q, f)[0], want, rtol=0, atol=1e-14):
        return False
    # the same path at x = -1 and x = 2 (and x = 0, where every layer gives 0)
    f2 = np.zeros((3, 16))
    f2[:, 0] = [1.0 + 2.0 * -1.0, 1.0 + 2.0 * 2.0, 1.0]       # x = -1, 2, 0
    out = forward(q, f2)
    raw = (out - np.array([10.0, 20.0, 30.0])) / np.array([2.0, 3.0, 4.0])
    for row, s3x in ((0, SILU_3X_M1), (1, SILU_3X_2)):
        if not np.allclose(raw[row], np.array([1.0, -2.0, 0.5]) * s3x, rtol=0, atol=1e-14):
            return False
    if np.max(np.abs(raw[2])) != 0.0:                           # SiLU(0) = 0 all the way through
        return False
    # the output layer is linear: doubling W4 doubles the raw output
    q2 = _one_path(w4=(2.0, -4.0, 1.0))
    raw2 = (forward(q2, f) - np.array([10.0, 20.0, 30.0])) / np.array([2.0, 3.0, 4.0])
    raw1 = (forward(q, f) - np.array([10.0, 20.0, 30.0])) / np.array([2.0, 3.0, 4.0])
    return bool(np.allclose(raw2, 2.0 * raw1, rtol=1e-13, atol=0))


def test_mlp_forward_pins():
    assert abs(M.silu(np.array([1.0]))[0] - SILU_1) < 1e-16
    assert _mlp_pins_hold(M.forward)


def test_mlp_forward_pins_reject_planted_slips(monkeypatch):
    def swapped_label_order(p, feat):            # (raw + ym) * ys instead of raw * ys + ym
        x = (np.asarray(feat, np.float64) - p["fm"]) / p["fs"]
        a = M.silu(M.silu(M.silu(x @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"])
        return (a @ p["W4"].T + p["b4"] + p["ym"]) * p["ys"]

    def swapped_feature_order(p, feat):          # f / std - mean instead of (f - mean) / std
        x = np.asarray(feat, np.float64) / p["fs"] - p["fm"]
        a = M.silu(M.silu(M.silu(x @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"])
        return (a @ p["W4"].T + p["b4"]) * p["ys"] + p["ym"]

    def activated_output(p, feat):               # SiLU on the output layer too
        x = (np.asarray(feat, np.float64) - p["fm"]) / p["fs"]
        a = M.silu(M.silu(M.silu(x @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"])
        return M.silu(a @ p["W4"].T + p["b4"]) * p["ys"] + p["ym"]

    for bad in (swapped_label_order, swapped_feature_order, activated_output):
        assert not _mlp_pins_hold(bad), bad.__name__
    # another activation planted in the oracle's own forward
    for act in (np.tanh, lambda s: np.maximum(s, 0.0), lambda s: 1.0 / (1.0 + np.exp(-s)),
                lambda s: s * (1.0 / (1.0 + np.exp(-1.702 * s)))):
        monkeypatch.setattr(M, "silu", act)
        assert not _mlp_pins_hold(M.forward)
