"""FP64 CPU oracle of the split-step method (SSM) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the CUDA library.  The arithmetic lives in
``ssm_oracle.c`` (plain C, IEEE double); this module is a ctypes wrapper that
moves numpy arrays in and out, plus the MLP oracle in ``mlp.py``.

Arrays are particle-major: ``x[i, c]`` with shape ``(N, d)``.
"""
import ctypes
import numpy as np

from .build import build_oracle

COEF_CUBIC1D_GAUSS = 0
COEF_COUPLED3D = 1
COEF_OU = 2
COEF_COUPLED1D = 3
COEF_GL1 = 4          # §3.2, SSM version 1: v = -x^3, b = s^2/2 y + c mean, sigma = s y
COEF_GL2 = 5          # §3.2, SSM version 2: v = -x^3 + c mean, b = s^2/2 y, sigma = s y
COEF_POLY = 6         # §3.3: v = gamma x - x mean(x^2), b = mean, sigma = y
COEF_CS = 7           # §3.4 Cucker-Smale, x = (V, X): v = (-V^3, 0), b = (1 + lambda (mean V - V), V)
COEF_GLSTAB = 8       # §3.4.2: v = -(5/2 + gamma) x - x^3/4, b = mean + gamma y, sigma = y

_c_int, _c_i64, _c_dbl, _c_u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64


class Problem(ctypes.Structure):
    _fields_ = [("d", _c_int), ("coef", _c_int), ("N", _c_i64), ("h", _c_dbl), ("T", _c_dbl),
                ("seed", _c_u64), ("p", _c_dbl * 4), ("x0_mean", _c_dbl), ("x0_std", _c_dbl),
                ("fine_log2", _c_int), ("measure_y", _c_int)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER(Problem)
        dp = ctypes.POINTER(_c_dbl)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        ip = ctypes.POINTER(_c_int)
        sig = {
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_normals": (None, [_c_u64, _c_int, _c_i64, _c_i64, _c_int, dp]),
            "orc_brownian": (None, [P, _c_i64, _c_i64, dp]),
            "orc_cardano_cubic": (_c_dbl, [_c_dbl, _c_dbl]),
            "orc_cardano_gl": (_c_dbl, [_c_dbl, _c_dbl]),
            "orc_implicit_one": (_c_int, [P, dp, _c_i64, dp]),
            "orc_implicit_point": (_c_int, [P, dp, dp, dp]),
            "orc_explicit_one": (None, [P, dp, _c_i64, _c_i64, dp]),
            "orc_drift_one": (None, [P, dp, _c_i64, dp]),
            "orc_pair_sum_coupled": (None, [P, dp, dp, dp, dp]),
            "orc_implicit_step": (_c_int, [P, dp, dp, ip]),
            "orc_explicit_step": (None, [P, dp, _c_i64, dp]),
            "orc_init_x0": (None, [P, dp]),
            "orc_moments": (None, [P, dp, dp]),
            "orc_run": (_c_int, [P, dp, _c_i64, _c_i64, dp, ctypes.POINTER(_c_i64)]),
            "orc_num_threads": (_c_int, []),
            "orc_joint_residual_one": (None, [P, dp, dp, _c_i64, dp]),
            "orc_sample_step": (None, [P, dp, dp, ctypes.POINTER(_c_i64), _c_i64, _c_i64, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(_c_dbl))


def problem(d, coef, N, h, T=1.0, seed=0, p=(0.0, 0.0, 0.0, 0.0), x0_mean=0.0, x0_std=1.0,
            fine_log2=0, measure_y=0):
    P = Problem()
    P.measure_y = int(measure_y)
    P.d, P.coef, P.N, P.h, P.T, P.seed = int(d), int(coef), int(N), float(h), float(T), int(seed)
    for k in range(4):
        P.p[k] = float(p[k]) if k < len(p) else 0.0
    P.x0_mean, P.x0_std, P.fine_log2 = float(x0_mean), float(x0_std), int(fine_log2)
    return P


def num_threads():
    return int(lib().orc_num_threads())


def philox(ctr, key):
    """Philox4x32-10 of each counter row (uint32 [n, 4]) under one key (uint32 [2])."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    f = lib().orc_philox4x32_10
    kp = key.ctypes.data_as(u32p)
    for r in range(ctr.shape[0]):
        f(ctr[r].ctypes.data_as(u32p), kp, out[r].ctypes.data_as(u32p))
    return out


def normals(seed, d, i, step, stream):
    z = np.empty(3)
    lib().orc_normals(int(seed), int(d), int(i), int(step), int(stream), _dp(z))
    return z[:d].copy()


def brownian(P, i, n):
    dw = np.empty(3)
    lib().orc_brownian(ctypes.byref(P), int(i), int(n), _dp(dw))
    return dw[:P.d].copy()


def cardano(x, h):
    return float(lib().orc_cardano_cubic(float(x), float(h)))


def cardano_gl(x, h):
    """Root of y + h y^3 = x."""
    return float(lib().orc_cardano_gl(float(x), float(h)))


def init_x0(P):
    x = np.empty((P.N, P.d))
    lib().orc_init_x0(ctypes.byref(P), _dp(x))
    return x


def _c(x, P):
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (P.N, P.d), (x.shape, P.N, P.d)
    return x


def implicit_one(P, x, i):
    x = _c(x, P)
    y = np.empty(3)
    it = lib().orc_implicit_one(ctypes.byref(P), _dp(x), int(i), _dp(y))
    return y[:P.d].copy(), int(it)


def implicit_point(P, x, xpoint):
    """F_h(xpoint; mu^X) of Lemma 4.1 for an arbitrary point."""
    x = _c(x, P)
    xp = np.zeros(3)
    xp[:P.d] = np.asarray(xpoint, dtype=np.float64).reshape(P.d)
    y = np.empty(3)
    it = lib().orc_implicit_point(ctypes.byref(P), _dp(x), _dp(xp), _dp(y))
    return y[:P.d].copy(), int(it)


def explicit_one(P, y, i, n):
    y = _c(y, P)
    out = np.empty(3)
    lib().orc_explicit_one(ctypes.byref(P), _dp(y), int(i), int(n), _dp(out))
    return out[:P.d].copy()


def drift_one(P, y, i):
    y = _c(y, P)
    out = np.empty(3)
    lib().orc_drift_one(ctypes.byref(P), _dp(y), int(i), _dp(out))
    return out[:P.d].copy()


def pair_sum_coupled(P, x, y_point):
    x = _c(x, P)
    yp = np.zeros(3)
    yp[:P.d] = np.asarray(y_point, dtype=np.float64).reshape(P.d)
    S = np.empty(3)
    JS = np.empty(9)
    lib().orc_pair_sum_coupled(ctypes.byref(P), _dp(x), _dp(yp), _dp(S), _dp(JS))
    return S[:P.d].copy(), JS[:P.d * P.d].reshape(P.d, P.d)


def joint_residual_one(P, x, y, i):
    """G_i = Y_i - X_i - h v(Y_i, mu^Y) of step 1 against the measure of Y itself."""
    x, y = _c(x, P), _c(y, P)
    g = np.empty(3)
    lib().orc_joint_residual_one(ctypes.byref(P), _dp(x), _dp(y), int(i), _dp(g))
    return g[:P.d].copy()


def implicit_step(P, x):
    x = _c(x, P)
    y = np.empty_like(x)
    it = np.empty(P.N, dtype=np.int32)
    bad = lib().orc_implicit_step(ctypes.byref(P), _dp(x), _dp(y),
                                  it.ctypes.data_as(ctypes.POINTER(_c_int)))
    return y, it, int(bad)


def explicit_step(P, y, n):
    y = _c(y, P)
    x = np.empty_like(y)
    lib().orc_explicit_step(ctypes.byref(P), _dp(y), int(n), _dp(x))
    return x


def sample_step(P, x, idx, n):
    """Step n restricted to the target particles idx (for timing a bounded sample):
    returns X_{n+1} of those targets.  Particles outside the sample enter step 2's
    measure at their X_n."""
    x = _c(x, P)
    y = x.copy()
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((idx.size, P.d))
    lib().orc_sample_step(ctypes.byref(P), _dp(x), _dp(y), idx.ctypes.data_as(ctypes.POINTER(_c_i64)),
                          idx.size, int(n), _dp(out))
    return out


def moments(P, x):
    x = _c(x, P)
    m = np.empty((4, P.d))
    lib().orc_moments(ctypes.byref(P), _dp(x), _dp(m))
    return m


def run(P, x, n0, nsteps, want_moments=False):
    """Advance a copy of x through nsteps SSM steps starting at step index n0."""
    x = _c(x, P).copy()
    mom = np.empty((max(int(nsteps), 1), 4, P.d)) if want_moments else None
    tot = _c_i64(0)
    bad = lib().orc_run(ctypes.byref(P), _dp(x), int(n0), int(nsteps),
                        _dp(mom) if mom is not None else None, ctypes.byref(tot))
    if bad:
        raise RuntimeError("oracle: %d implicit solves did not converge" % bad)
    return (x, mom, int(tot.value)) if want_moments else x
