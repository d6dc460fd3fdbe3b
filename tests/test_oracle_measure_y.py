"""Pins of the oracle's step 1 against mu^Y (the joint R^{dN} system that §1
contrasts with the SSM, for the coupled sets) by facts that do not come from its
own solver: the invariant that holds only when the measure is the particles' own,
the closed form of a single particle, and 40-digit brute force on tiny systems.
CPU only (no GPU marker).
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs


def _pair_part_sum(x, y, h):
    """sum_i (Y_i - X_i + h Y_i |Y_i|^2): h/2 times the sum over i of S_i(Y), which is
    zero when S_i is taken against mu^Y (each pair appears once with each sign)."""
    return np.sum(y - x + h * y * np.sum(y * y, axis=1, keepdims=True), axis=0)


@pytest.mark.parametrize("d,coef", [(3, O.COEF_COUPLED3D), (1, O.COEF_COUPLED1D)])
def test_pair_part_sums_to_zero_only_for_the_own_measure(d, coef):
    N, h = 120, 2.0 ** -5
    x = inputs.gaussian_cloud(N, d, seed=31, scale=1.3)
    P = O.problem(d=d, coef=coef, N=N, h=h, measure_y=1)
    y, it, bad = O.implicit_step(P, x)
    assert bad == 0 and it[0] > 0
    assert np.max(np.abs(_pair_part_sum(x, y, h))) < 1e-13 * N
    Ps = O.problem(d=d, coef=coef, N=N, h=h)                  # the SSM's step 1 (mu^X)
    ys, _, _ = O.implicit_step(Ps, x)
    assert np.max(np.abs(_pair_part_sum(x, ys, h))) > 1e-6


def test_single_particle_closed_form():
    """N = 1: the pair term vanishes, Y + h |Y|^2 Y = X, so Y = s X with s the real
    root of h |X|^2 s^3 + s = 1."""
    h = 2.0 ** -4
    for x in inputs.gaussian_cloud(6, 3, seed=32, scale=2.0):
        P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=1, h=h, measure_y=1)
        y, _, bad = O.implicit_step(P, x.reshape(1, 3))
        s = O.cardano_gl(1.0, h * float(np.dot(x, x)))
        assert bad == 0
        assert np.max(np.abs(y[0] - s * x)) < 4e-16 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("d,coef", [(3, O.COEF_COUPLED3D), (1, O.COEF_COUPLED1D)])
def test_tiny_systems_match_high_precision_fixed_point(d, coef):
    """N = 3: the contraction Y <- X + h v(Y, mu^Y) iterated to 40 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    N, h = 3, 2.0 ** -6
    x = inputs.gaussian_cloud(N, d, seed=33)
    P = O.problem(d=d, coef=coef, N=N, h=h, measure_y=1)
    y, _, bad = O.implicit_step(P, x)
    assert bad == 0
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
    exact = np.array([[float(c) for c in row] for row in Y])
    assert np.max(np.abs(y - exact)) < 1e-15
