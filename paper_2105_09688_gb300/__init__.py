"""Python binding of the GB300 split-step-method library (``libssm.so``).

Thin ctypes marshalling over the C ABI of ``include/ssm.h``: the functions here
carry the same names and move numpy arrays and plain numbers across; every step
of the method runs in the library's CUDA kernels.  PyTorch is used only to hand
the library device memory (a workspace tensor) and a CUDA stream.

The library must have been built (``paper_2105_09688_gb300.build.build()``); if
it is missing, loading fails with an error -- there is no CPU fallback.

Method: Chen & dos Reis, "A flexible split-step scheme for solving McKean-Vlasov
stochastic differential equations", arXiv:2105.09688, §2.3.
"""
import ctypes
import os

import numpy as np

__all__ = [
    "SSM_OK", "SSM_EINVAL", "SSM_ENOMEM", "SSM_ECUDA", "SSM_ENOCONV", "SSM_ENONFINITE", "SSM_ETIMEOUT",
    "SSM_ESTATE", "SSM_COEF_CUBIC1D_GAUSS", "SSM_COEF_COUPLED3D", "SSM_COEF_OU", "SSM_FP64", "SSM_FP32C",
    "SSM_FP32C_LEARNED", "SSM_STAGE_Y", "SSM_STAGE_B", "SSMError", "ssm_opts", "ssm_stats_t", "lib",
    "ssm_opts_default", "ssm_workspace_bytes", "ssm_create", "ssm_step", "ssm_run_steps", "ssm_run", "ssm_sync",
    "ssm_moments", "ssm_get_state", "ssm_set_state", "ssm_get_stage", "ssm_stats", "ssm_destroy",
    "ssm_status_str", "ssm_philox", "ssm_normals", "ssm_normals_fp32", "ssm_convert_check", "ssm_cardano", "ssm_pair_pass", "ssm_autotune", "ssm_get_plan",
    "ssm_set_plan", "ssm_set_plan_chunks", "tune_cache_key", "tune_cache_load", "tune_cache_store", "ssm_drift_noalloc", "ssm_pipe_probe", "SSM", "Batch", "ssm_ens_desc", "SSM_COEF_COUPLED1D", "SSM_COEF_GL1", "SSM_COEF_GL2", "SSM_COEF_POLY", "SSM_COEF_CS", "SSM_COEF_GLSTAB", "ssm_stability_beta", "load_ws",
    "ssm_ws_train", "ssm_ws_predict", "ssm_ws_grad", "ssm_ws_collect", "ssm_ws_load", "ssm_ws_params", "ssm_ws_blob_bytes",
    "ssm_ws_num_params",
]

SSM_OK, SSM_EINVAL, SSM_ENOMEM, SSM_ECUDA, SSM_ENOCONV, SSM_ENONFINITE, SSM_ETIMEOUT, SSM_ESTATE, SSM_EBOUNDS = range(9)
SSM_BUILD_CHECK_BOUNDS = 1
SSM_COEF_CUBIC1D_GAUSS, SSM_COEF_COUPLED3D, SSM_COEF_OU, SSM_COEF_COUPLED1D = 0, 1, 2, 3
SSM_COEF_GL1, SSM_COEF_GL2, SSM_COEF_POLY, SSM_COEF_CS, SSM_COEF_GLSTAB = 4, 5, 6, 7, 8
SSM_FP64, SSM_FP32C, SSM_FP32C_LEARNED = 0, 1, 2
SSM_STAGE_Y, SSM_STAGE_B = 0, 1

# SSM_LIB_VARIANT=check selects the debug build libssm_check.so (bounds-checked
# kernels, see ssm_build_flags); the default is the release library.
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libssm_check.so" if os.environ.get("SSM_LIB_VARIANT") == "check" else "libssm.so")
# Learned-start network trained by train_ws.py (rows from plain-SSM runs, seeds 100..163).
WS_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ws_weights.bin")


def load_ws(s, path=WS_WEIGHTS):
    """Load the shipped learned-start network into an SSM context."""
    with open(path, "rb") as f:
        s.ws_load(f.read())

_i32, _i64, _u64, _dbl, _sz, _vp = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_size_t, ctypes.c_void_p)


class ssm_opts(ctypes.Structure):
    _fields_ = [("precision", _i32), ("newton_tol", _dbl), ("newton_kmax", _i32), ("fine_log2", _i32),
                ("x0_mean", _dbl), ("x0_std", _dbl), ("coef_params", _dbl * 4), ("stream", _vp),
                ("workspace", _vp), ("workspace_bytes", _sz), ("tile_chunks", _i32), ("ws_passes", _i32),
                ("measure_y", _i32), ("ws_forward", _i32), ("fixed_pass_launches", _i32), ("inject", _i32),
                ("carry_start", _i32)]


class ssm_stats_t(ctypes.Structure):
    _fields_ = [("steps", _i64), ("newton_passes", _i64), ("newton_rows", _i64), ("drift_rows", _i64),
                ("fallbacks", _i64), ("max_passes", _i64), ("hist", _i64 * 16), ("floor_accepts", _i64)]


class SSMError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__("%s%s" % (where + ": " if where else "", ssm_status_str(status)))


_LIB = None
_DP = ctypes.POINTER(_dbl)
_U32P = ctypes.POINTER(ctypes.c_uint32)

_SIGS = {
    "ssm_opts_default": (None, [ctypes.POINTER(ssm_opts)]),
    "ssm_workspace_bytes": (_sz, [_i32, _i64, _i32, ctypes.POINTER(ssm_opts)]),
    "ssm_create": (_i32, [_i32, _i64, _dbl, _dbl, _i32, _u64, ctypes.POINTER(ssm_opts), ctypes.POINTER(_vp)]),
    "ssm_step": (_i32, [_vp]),
    "ssm_run_steps": (_i32, [_vp, _i64]),
    "ssm_run": (_i32, [_vp]),
    "ssm_sync": (_i32, [_vp]),
    "ssm_moments": (_i32, [_vp, _DP]),
    "ssm_get_state": (_i32, [_vp, _DP, ctypes.POINTER(_i64)]),
    "ssm_set_state": (_i32, [_vp, _DP, _i64]),
    "ssm_get_stage": (_i32, [_vp, _i32, _DP]),
    "ssm_stats": (_i32, [_vp, ctypes.POINTER(ssm_stats_t)]),
    "ssm_destroy": (None, [_vp]),
    "ssm_status_str": (ctypes.c_char_p, [_i32]),
    "ssm_build_flags": (_i32, []),
    "ssm_pipe_probe": (_i32, [_DP]),
    "ssm_philox": (_i32, [_u64, _U32P, _i64, _U32P]),
    "ssm_normals": (_i32, [_u64, _i32, _i64, _i64, _i32, _DP]),
    "ssm_normals_fp32": (_i32, [_u64, _i32, _i64, _i64, _i32, ctypes.POINTER(ctypes.c_float)]),
    "ssm_convert_check": (_i32, [_DP, _i64, ctypes.POINTER(ctypes.c_float), _DP]),
    "ssm_stability_beta": (_i32, [_dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _DP]),
    "ssm_cardano": (_i32, [_DP, _i64, _dbl, _DP]),
    "ssm_pair_pass": (_i32, [_vp, _i32, ctypes.POINTER(_i64)]),
    "ssm_autotune": (_i32, [_vp, _DP]),
    "ssm_get_plan": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "ssm_set_plan": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "ssm_set_plan_chunks": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "ssm_drift_noalloc": (_i32, [_i32, _i32, _i64, _vp, _i64, _vp, _vp]),
    "ssm_ws_blob_bytes": (_sz, []),
    "ssm_ws_num_params": (_i32, []),
    "ssm_ws_load": (_i32, [_vp, _vp, _sz]),
    "ssm_ws_collect": (_i32, [_vp, _i64, _i64, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(_i64)]),
    "ssm_ws_predict": (_i32, [_vp, _sz, ctypes.POINTER(ctypes.c_float), _i64, ctypes.POINTER(ctypes.c_float)]),
    "ssm_ws_grad": (_i32, [_vp, _sz, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _i64,
                           ctypes.POINTER(ctypes.c_float), _DP]),
    "ssm_ws_train": (_i32, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _i64, _i32, _i32,
                            ctypes.c_float, _u64, _vp, _sz, _DP]),
    "ssm_ws_params": (_i32, [_vp, _sz, ctypes.POINTER(ctypes.c_float)]),
    "ssm_batch_create": (_i32, [_i32, _vp, ctypes.POINTER(ssm_opts), ctypes.POINTER(_vp)]),
    "ssm_batch_run_steps": (_i32, [_vp, _i64]),
    "ssm_batch_run": (_i32, [_vp]),
    "ssm_batch_sync": (_i32, [_vp]),
    "ssm_batch_get_state": (_i32, [_vp, _i32, _DP, ctypes.POINTER(_i64)]),
    "ssm_batch_moments": (_i32, [_vp, _i32, _DP]),
    "ssm_batch_stats": (_i32, [_vp, ctypes.POINTER(ssm_stats_t)]),
    "ssm_batch_autotune": (_i32, [_vp, _DP]),
    "ssm_batch_get_plan": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "ssm_batch_set_plan": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "ssm_batch_destroy": (None, [_vp]),
}


class ssm_ens_desc(ctypes.Structure):
    _fields_ = [("d", _i32), ("N", _i64), ("h", _dbl), ("T", _dbl), ("seed", _u64), ("fine_log2", _i32)]


class Batch:
    """Many independent ensembles (coupled coefficient set at d = 1 or 3) advanced by
    one graph launch.  ``descs``: iterable of dicts with keys d, N, h, T, seed and
    optionally fine_log2."""

    def __init__(self, descs, stream=None, **opt):
        descs = list(descs)
        arr = (ssm_ens_desc * len(descs))()
        for k, dsc in enumerate(descs):
            arr[k].d, arr[k].N, arr[k].h, arr[k].T = int(dsc["d"]), int(dsc["N"]), float(dsc["h"]), float(dsc["T"])
            arr[k].seed, arr[k].fine_log2 = int(dsc["seed"]), int(dsc.get("fine_log2", 0))
        self.descs = descs
        self.opts = ssm_opts_default(**opt)
        if stream is not None:
            self._stream = stream
            self.opts.stream = int(stream.cuda_stream) or None
        out = _vp()
        _check(lib().ssm_batch_create(len(descs), ctypes.cast(arr, _vp), ctypes.byref(self.opts), ctypes.byref(out)),
               "ssm_batch_create")
        self.b = out

    def run(self):
        _check(lib().ssm_batch_run(self.b), "ssm_batch_run")

    def run_steps(self, k):
        _check(lib().ssm_batch_run_steps(self.b, int(k)), "ssm_batch_run_steps")

    def sync(self):
        _check(lib().ssm_batch_sync(self.b), "ssm_batch_sync")

    def get_state(self, e):
        dsc = self.descs[e]
        x = np.empty((int(dsc["N"]), int(dsc["d"])))
        n = _i64(0)
        _check(lib().ssm_batch_get_state(self.b, int(e), _dp(x), ctypes.byref(n)), "ssm_batch_get_state")
        return x, int(n.value)

    def moments(self, e):
        out = np.empty((4, int(self.descs[e]["d"])))
        _check(lib().ssm_batch_moments(self.b, int(e), _dp(out)), "ssm_batch_moments")
        return out

    def stats(self):
        s = ssm_stats_t()
        _check(lib().ssm_batch_stats(self.b, ctypes.byref(s)), "ssm_batch_stats")
        return {"ensemble_steps": s.steps, "newton_passes": s.newton_passes, "newton_rows": s.newton_rows,
                "drift_rows": s.drift_rows, "batch_steps": s.max_passes, "floor_accepts": s.floor_accepts}

    def autotune(self):
        best = _dbl(0.0)
        _check(lib().ssm_batch_autotune(self.b, ctypes.byref(best)), "ssm_batch_autotune")
        return float(best.value)

    def set_plan(self, form, targets_per_thread_d1, targets_per_thread_d3, chunk_len):
        arr = (_i32 * 4)(int(form), int(targets_per_thread_d1), int(targets_per_thread_d3), int(chunk_len))
        _check(lib().ssm_batch_set_plan(self.b, arr), "ssm_batch_set_plan")

    def plan(self):
        out = (_i32 * 5)()
        _check(lib().ssm_batch_get_plan(self.b, out), "ssm_batch_get_plan")
        return dict(zip(("form", "threads", "targets_per_thread_d1", "targets_per_thread_d3", "chunk_len"),
                        list(out)))

    def close(self):
        if getattr(self, "b", None):
            lib().ssm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

_FP = ctypes.POINTER(ctypes.c_float)


def _fp(a):
    return a.ctypes.data_as(_FP)


def _blob_arg(blob):
    b = np.ascontiguousarray(np.frombuffer(bytes(blob), dtype=np.uint8))
    return b, b.ctypes.data_as(_vp), b.size


def ssm_ws_blob_bytes():
    return int(lib().ssm_ws_blob_bytes())


def ssm_ws_num_params():
    return int(lib().ssm_ws_num_params())


def ssm_ws_load(ctx, blob):
    keep, p, n = _blob_arg(blob)
    _check(lib().ssm_ws_load(ctx, p, n), "ssm_ws_load")


def ssm_ws_collect(ctx, N, stride, offset):
    rows = max(0, (N - offset + stride - 1) // stride)
    feat = np.empty((rows, 16), np.float32)
    label = np.empty((rows, 3), np.float32)
    got = _i64(0)
    _check(lib().ssm_ws_collect(ctx, int(stride), int(offset), _fp(feat), _fp(label), ctypes.byref(got)),
           "ssm_ws_collect")
    return feat[:got.value], label[:got.value]


def ssm_ws_predict(blob, feat):
    keep, p, n = _blob_arg(blob)
    feat = np.ascontiguousarray(feat, np.float32).reshape(-1, 16)
    out = np.empty((feat.shape[0], 3), np.float32)
    _check(lib().ssm_ws_predict(p, n, _fp(feat), feat.shape[0], _fp(out)), "ssm_ws_predict")
    return out


def ssm_ws_grad(blob, feat, label):
    keep, p, n = _blob_arg(blob)
    feat = np.ascontiguousarray(feat, np.float32).reshape(-1, 16)
    label = np.ascontiguousarray(label, np.float32).reshape(-1, 3)
    g = np.empty(ssm_ws_num_params(), np.float32)
    loss = _dbl(0.0)
    _check(lib().ssm_ws_grad(p, n, _fp(feat), _fp(label), feat.shape[0], _fp(g), ctypes.byref(loss)), "ssm_ws_grad")
    return g, float(loss.value)


def ssm_ws_train(feat, label, epochs=20, batch=8192, lr=2e-3, seed=0):
    """Train the learned-start network on the GPU; returns (blob bytes, per-epoch losses)."""
    feat = np.ascontiguousarray(feat, np.float32).reshape(-1, 16)
    label = np.ascontiguousarray(label, np.float32).reshape(-1, 3)
    blob = np.zeros(ssm_ws_blob_bytes(), np.uint8)
    curve = np.zeros(int(epochs))
    _check(lib().ssm_ws_train(_fp(feat), _fp(label), feat.shape[0], int(epochs), int(batch), float(lr), int(seed),
                              blob.ctypes.data_as(_vp), blob.size, _dp(curve)), "ssm_ws_train")
    return blob.tobytes(), curve


def ssm_ws_params(blob):
    keep, p, n = _blob_arg(blob)
    out = np.empty(ssm_ws_num_params(), np.float32)
    _check(lib().ssm_ws_params(p, n, _fp(out)), "ssm_ws_params")
    return out


def lib():
    """Load libssm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built; run paper_2105_09688_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status, where):
    if status != SSM_OK:
        raise SSMError(status, where)


def _dp(a):
    return a.ctypes.data_as(_DP)


def ssm_status_str(status):
    return lib().ssm_status_str(int(status)).decode()


def ssm_opts_default(**kw):
    o = ssm_opts()
    lib().ssm_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "coef_params":
            for i, p in enumerate(v):
                o.coef_params[i] = float(p)
        else:
            setattr(o, k, v)
    return o


def ssm_workspace_bytes(d, N, coef, opts=None):
    return int(lib().ssm_workspace_bytes(int(d), int(N), int(coef), ctypes.byref(opts) if opts else None))


def ssm_create(d, N, h, T, coef, seed, opts=None):
    out = _vp()
    _check(lib().ssm_create(int(d), int(N), float(h), float(T), int(coef), int(seed),
                            ctypes.byref(opts) if opts else None, ctypes.byref(out)), "ssm_create")
    return out


def ssm_step(ctx):
    _check(lib().ssm_step(ctx), "ssm_step")


def ssm_run_steps(ctx, k):
    _check(lib().ssm_run_steps(ctx, int(k)), "ssm_run_steps")


def ssm_run(ctx):
    _check(lib().ssm_run(ctx), "ssm_run")


def ssm_sync(ctx):
    _check(lib().ssm_sync(ctx), "ssm_sync")


def ssm_moments(ctx, d):
    out = np.empty((4, d))
    _check(lib().ssm_moments(ctx, _dp(out)), "ssm_moments")
    return out


def ssm_get_state(ctx, N, d, out=None):
    """Current state as an (N, d) array (or into ``out``, e.g. a pinned buffer) and step index."""
    x = np.empty((N, d)) if out is None else out
    n = _i64(0)
    _check(lib().ssm_get_state(ctx, _dp(x), ctypes.byref(n)), "ssm_get_state")
    return x, int(n.value)


def ssm_set_state(ctx, x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    _check(lib().ssm_set_state(ctx, _dp(x), int(n)), "ssm_set_state")


def ssm_get_stage(ctx, which, N, d):
    out = np.empty((N, d))
    _check(lib().ssm_get_stage(ctx, int(which), _dp(out)), "ssm_get_stage")
    return out


def ssm_stats(ctx):
    s = ssm_stats_t()
    _check(lib().ssm_stats(ctx, ctypes.byref(s)), "ssm_stats")
    return {"steps": s.steps, "newton_passes": s.newton_passes, "newton_rows": s.newton_rows,
            "drift_rows": s.drift_rows, "fallbacks": s.fallbacks, "max_passes": s.max_passes,
            "hist": [int(v) for v in s.hist], "floor_accepts": s.floor_accepts}


def ssm_destroy(ctx):
    if ctx:
        lib().ssm_destroy(ctx)


def ssm_philox(seed, ctr):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    _check(lib().ssm_philox(int(seed), ctr.ctypes.data_as(_U32P), ctr.shape[0], out.ctypes.data_as(_U32P)),
           "ssm_philox")
    return out


def ssm_normals(seed, d, N, step, stream):
    out = np.empty((int(N), int(d)))
    _check(lib().ssm_normals(int(seed), int(d), int(N), int(step), int(stream), _dp(out)), "ssm_normals")
    return out


def ssm_stability_beta(Lv, Lvt, Lb, Lbt, Ls, Lst, h):
    """beta of the mean-square stability theorem (see include/ssm.h)."""
    out = _dbl()
    _check(lib().ssm_stability_beta(float(Lv), float(Lvt), float(Lb), float(Lbt), float(Ls), float(Lst), float(h),
                                    ctypes.byref(out)), "ssm_stability_beta")
    return float(out.value)


def ssm_pipe_probe():
    """Measured FP32 pipe rates of the current device: dict of lane operations per clock
    per SM (ffma, ffma2, rcp, ex2) and the SM clock in GHz during the probe."""
    out = np.zeros(5)
    _check(lib().ssm_pipe_probe(_dp(out)), "ssm_pipe_probe")
    return {"ffma": float(out[0]), "ffma2": float(out[1]), "rcp": float(out[2]), "ex2": float(out[3]),
            "clock_ghz": float(out[4])}


def ssm_convert_check(values):
    """The library's integer-pipe conversions run on the host: (float32 of each
    value, float64 of that float32)."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    o32 = np.empty(v.size, dtype=np.float32)
    o64 = np.empty(v.size, dtype=np.float64)
    _check(lib().ssm_convert_check(_dp(v), v.size, o32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(o64)),
           "ssm_convert_check")
    return o32, o64


def ssm_normals_fp32(seed, d, N, step, stream):
    out = np.empty((int(N), int(d)), dtype=np.float32)
    _check(lib().ssm_normals_fp32(int(seed), int(d), int(N), int(step), int(stream),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "ssm_normals_fp32")
    return out


def ssm_pair_pass(ctx, which):
    """Enqueue one full pair-sum pass (0: step-1 sums, 1: step-2 drift); returns the pair count."""
    pairs = _i64(0)
    _check(lib().ssm_pair_pass(ctx, int(which), ctypes.byref(pairs)), "ssm_pair_pass")
    return int(pairs.value)


def ssm_autotune(ctx):
    """Tune the pair-sum launch shapes on the context's state; returns the best pass times (ms)."""
    best = np.zeros(2)
    _check(lib().ssm_autotune(ctx, _dp(best)), "ssm_autotune")
    return best


def ssm_get_plan(ctx, which):
    out = (_i32 * 5)()
    _check(lib().ssm_get_plan(ctx, int(which), out), "ssm_get_plan")
    return dict(zip(("form", "threads", "targets_per_thread", "chunks", "chunk_len"), list(out)))


def ssm_set_plan(ctx, which, form, threads, targets_per_thread):
    """form: 0 scalar kernel, 1 packed-FP32 difference form, 2 packed-FP32 centred expansion."""
    arr = (_i32 * 3)(int(form), int(threads), int(targets_per_thread))
    _check(lib().ssm_set_plan(ctx, int(which), arr), "ssm_set_plan")


def ssm_set_plan_chunks(ctx, which, form, threads, targets_per_thread, chunks):
    """ssm_set_plan with the source chunk count fixed (chunks >= 1)."""
    arr = (_i32 * 4)(int(form), int(threads), int(targets_per_thread), int(chunks))
    _check(lib().ssm_set_plan_chunks(ctx, int(which), arr), "ssm_set_plan_chunks")


# Tuning cache: the autotuner's choice per device, library build and workload, kept
# in a JSON file so that later contexts of the same workload take it without tuning.
def tune_cache_key(device_name, sms, library_digest, d, N, coef, precision):
    """Key of a tuned plan: the device (name, SM count), the library build (a digest
    of libssm.so) and the workload (d, N, coefficient set, precision)."""
    return "|".join(str(v) for v in (device_name, int(sms), library_digest, int(d), int(N), int(coef),
                                     int(precision)))


def tune_cache_load(path):
    """The cache's entries ({} if the file is missing or not a JSON object)."""
    import json
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def tune_cache_store(path, key, entry):
    """Adds or replaces one entry; the file is rewritten through a temporary file in
    the same directory and renamed over the old one, so readers see either file."""
    import json
    import tempfile
    data = tune_cache_load(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tune", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def _library_digest():
    import hashlib
    h = hashlib.sha256()
    with open(LIB_PATH, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def ssm_drift_noalloc(coef, precision, N, y_ptr, ld, b_ptr, stream_ptr=0):
    """Step-2 drift of the device arrays at y_ptr into b_ptr (SoA, leading dimension ld)
    without allocating (scratch is a fixed static device array; see include/ssm.h).
    For callers that cannot allocate device memory at the point of use."""
    _check(lib().ssm_drift_noalloc(int(coef), int(precision), int(N), _vp(int(y_ptr)), int(ld), _vp(int(b_ptr)),
                                   _vp(int(stream_ptr)) if stream_ptr else None), "ssm_drift_noalloc")


def ssm_cardano(x, h):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.empty_like(x)
    _check(lib().ssm_cardano(_dp(x), x.size, float(h), _dp(y)), "ssm_cardano")
    return y


class SSM:
    """A context whose device workspace is a torch tensor and whose stream is
    torch's current CUDA stream (or one passed in).

    >>> s = SSM(d=3, N=1 << 12, h=2**-8, T=1.0, coef=SSM_COEF_COUPLED3D, seed=2, precision=SSM_FP32C)
    >>> s.run(); m = s.moments()
    """

    def __init__(self, d, N, h, T, coef, seed, stream=None, **opt):
        import torch
        self.d, self.N, self.h, self.T, self.coef = int(d), int(N), float(h), float(T), int(coef)
        self.opts = ssm_opts_default(**opt)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.opts.stream = int(stream.cuda_stream) or None
        nbytes = ssm_workspace_bytes(d, N, coef, self.opts)
        if nbytes == 0:
            raise SSMError(SSM_EINVAL, "ssm_workspace_bytes")
        # 256-byte aligned device workspace owned by torch's allocator
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        self.opts.workspace = (base + 255) // 256 * 256
        self.opts.workspace_bytes = nbytes
        self.ctx = ssm_create(d, N, h, T, coef, seed, self.opts)

    def step(self):
        ssm_step(self.ctx)

    def run_steps(self, k):
        ssm_run_steps(self.ctx, k)

    def run(self):
        ssm_run(self.ctx)

    def sync(self):
        ssm_sync(self.ctx)

    def moments(self):
        return ssm_moments(self.ctx, self.d)

    def get_state(self, out=None):
        return ssm_get_state(self.ctx, self.N, self.d, out)

    def set_state(self, x, n):
        ssm_set_state(self.ctx, x, n)

    def get_stage(self, which):
        return ssm_get_stage(self.ctx, which, self.N, self.d)

    def stats(self):
        return ssm_stats(self.ctx)

    def pair_pass(self, which):
        return ssm_pair_pass(self.ctx, which)

    def autotune(self, cache=None):
        """Tune the pair-sum launch shapes; returns the best pass times [step 1, drift]
        in ms.  cache: path of a JSON tuning cache: a plan tuned earlier for this
        device, library build and workload (d, N, coefficient set, precision) is
        restored with ssm_set_plan_chunks instead of tuning (its recorded times are
        returned), and a newly tuned one is added to the file."""
        pair_kinds = {SSM_COEF_COUPLED3D: (0, 1), SSM_COEF_COUPLED1D: (0, 1), SSM_COEF_CUBIC1D_GAUSS: (1,)}
        if cache is None or self.coef not in pair_kinds:
            return ssm_autotune(self.ctx)
        import torch
        dev = torch.cuda.current_device()
        key = tune_cache_key(torch.cuda.get_device_name(dev), torch.cuda.get_device_properties(dev).multi_processor_count,
                             _library_digest(), self.d, self.N, self.coef, self.opts.precision)
        entry = tune_cache_load(cache).get(key)
        if entry:
            try:
                for which, p in enumerate(entry["plans"]):
                    if p is not None:
                        self.set_plan(which, p["form"], p["threads"], p["targets_per_thread"], chunks=p["chunks"])
                return np.array(entry["best_ms"], dtype=float)
            except (KeyError, TypeError, SSMError):
                pass   # an entry this library cannot take: tune afresh
        best = ssm_autotune(self.ctx)
        plans = [self.plan(which) if which in pair_kinds[self.coef] else None for which in (0, 1)]
        tune_cache_store(cache, key, {"plans": plans, "best_ms": [float(v) for v in best]})
        return best

    def plan(self, which):
        return ssm_get_plan(self.ctx, which)

    def set_plan(self, which, form, threads, targets_per_thread, chunks=0):
        """chunks: 0 = planned (or ssm_opts.tile_chunks); >= 1 fixes the source chunks."""
        if chunks:
            ssm_set_plan_chunks(self.ctx, which, form, threads, targets_per_thread, chunks)
        else:
            ssm_set_plan(self.ctx, which, form, threads, targets_per_thread)

    def ws_load(self, blob):
        ssm_ws_load(self.ctx, blob)

    def ws_collect(self, stride, offset=0):
        return ssm_ws_collect(self.ctx, self.N, stride, offset)

    def close(self):
        if getattr(self, "ctx", None):
            ssm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
