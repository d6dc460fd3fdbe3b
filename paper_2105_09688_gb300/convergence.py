"""Weak and strong errors of the SSM against a finer step on the same Brownian paths,
as §3 measures them (the paper's eq. for epsilon_k):
    epsilon_1 = | (1/N) sum_j (X_T^j - Xhat_T^j) |_2      (weak, k = 1)
    epsilon_2 = ( (1/N) sum_j |X_T^j - Xhat_T^j|^2 )^(1/2)  (strong, k = 2)
where X_T is the run at the fine step (the paper's proxy for the true solution)
and Xhat_T the run at step h; every run samples its increments from the Brownian
path on the fine grid (ssm_opts.fine_log2), so all of them share one path.
Every step runs in the library's GPU kernels.

``batch_study`` does the same for many independent ensembles at once (the batched
form): each ensemble is compared with its own run at the fine step, all of them
advanced together by one graph launch.
"""
import math

import numpy as np

from . import SSM, SSM_FP32C, SSM_FP64, Batch, ssm_philox


def weak_strong(x, ref):
    """(epsilon_1, epsilon_2) of §3 between particle arrays x and ref, shape (N, d):
    the norm of the mean difference and the root mean square of the differences."""
    diff = np.asarray(x, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.mean(diff, axis=0))), math.sqrt(float(np.mean(np.sum(diff * diff, axis=1))))


def error_study(coef, d, T, ks, k_ref, N, seed, coef_params=(), x0_mean=0.0, x0_std=1.0, precision=SSM_FP64,
                measure_y=0):
    """epsilon_1 and epsilon_2 at T for h = T 2^-k (k in ks) against h = T 2^-k_ref.
    Returns dict(h, weak, strong, weak_slope, strong_slope) (slopes of log2 error
    against log2 h, least squares)."""
    def run(k):
        s = SSM(d=d, N=N, h=T * 2.0 ** -k, T=T, coef=coef, seed=seed, precision=precision,
                coef_params=coef_params, x0_mean=x0_mean, x0_std=x0_std, fine_log2=k_ref, measure_y=measure_y)
        s.run()
        x, _ = s.get_state()
        s.close()
        return x

    ref = run(k_ref)
    hs, weak, strong = [], [], []
    for k in ks:
        x = run(k)
        hs.append(T * 2.0 ** -k)
        w, st = weak_strong(x, ref)
        weak.append(w)
        strong.append(st)
    lh = np.log2(hs)
    return dict(h=hs, weak=weak, strong=strong, weak_slope=float(np.polyfit(lh, np.log2(weak), 1)[0]),
                strong_slope=float(np.polyfit(lh, np.log2(strong), 1)[0]))


def mixed_ensembles(count=64, seed=3):
    """The mixed ensemble workload of the batched form: ensemble e has
    N_e = round(2^(10 + 6 u_e)), u_e the FP64 uniform of Philox(seed, counter (e, 0, 2, 0))
    (N log-uniform in [2^10, 2^16]), d_e = 1 for the first half and 3 for the second,
    h_e = 2^-(4 + e mod 7), T = 1 and seed 1000 + e."""
    out = []
    for e in range(count):
        w = ssm_philox(seed, [[e, 0, 2, 0]])[0]
        u = (((int(w[0]) << 32 | int(w[1])) >> 11) + 1) * 2.0 ** -53
        out.append(dict(d=1 if e < count // 2 else 3, N=int(round(2.0 ** (10 + 6 * u))), h=2.0 ** -(4 + e % 7),
                        T=1.0, seed=1000 + e))
    return out


def batch_study(descs, ref_log2=14, precision=SSM_FP32C, stream=None):
    """epsilon_1 and epsilon_2 at T of every ensemble in ``descs`` (dicts d, N, h, T,
    seed of the coupled set) against the same ensemble at h = T 2^-ref_log2 on the
    same Brownian path.  Every ensemble and one reference per distinct (d, N, T, seed)
    run in one Batch (one graph launch).

    Returns dict(per_ensemble=[dict(e, d, N, h, weak, strong)], by_h={h: (geometric
    mean weak, geometric mean strong)}, weak_slope, strong_slope, particle_steps);
    the slopes are least-squares fits of log2 error against log2 h over all ensembles
    (None with a single step size)."""
    runs = []
    for dsc in descs:
        if dsc["h"] <= dsc["T"] * 2.0 ** -ref_log2:
            raise ValueError("every ensemble needs a step coarser than the reference step")
        runs.append(dict(dsc, fine_log2=ref_log2))
    ref_of = {}
    for dsc in descs:
        key = (dsc["d"], dsc["N"], dsc["T"], dsc["seed"])
        if key not in ref_of:
            ref_of[key] = len(runs)
            runs.append(dict(d=dsc["d"], N=dsc["N"], T=dsc["T"], seed=dsc["seed"], h=dsc["T"] * 2.0 ** -ref_log2,
                             fine_log2=ref_log2))
    b = Batch(runs, stream=stream, precision=precision)
    try:
        b.run()
        b.sync()
        refs = {k: b.get_state(i)[0] for k, i in ref_of.items()}
        per = []
        for e, dsc in enumerate(descs):
            w, st = weak_strong(b.get_state(e)[0], refs[(dsc["d"], dsc["N"], dsc["T"], dsc["seed"])])
            per.append(dict(e=e, d=dsc["d"], N=dsc["N"], h=dsc["h"], weak=w, strong=st))
    finally:
        b.close()
    by_h = {}
    for h in sorted({r["h"] for r in per}, reverse=True):
        rows = [r for r in per if r["h"] == h]
        by_h[h] = tuple(float(2.0 ** np.mean(np.log2([max(r[k], 1e-300) for r in rows]))) for k in ("weak", "strong"))
    lh = np.log2([r["h"] for r in per])
    if len(set(lh)) > 1:
        slope = {k: float(np.polyfit(lh, np.log2([max(r[k], 1e-300) for r in per]), 1)[0]) for k in ("weak", "strong")}
    else:   # a single step size: no rate
        slope = {"weak": None, "strong": None}
    steps = sum(r["N"] * round(r["T"] / r["h"]) for r in runs)
    return dict(per_ensemble=per, by_h=by_h, weak_slope=slope["weak"], strong_slope=slope["strong"],
                particle_steps=steps)


def paper_examples(N=1 << 14, ks=range(3, 8), k_ref=11, seed=91):
    """The study for the §3 examples the library builds in: dict name -> result."""
    from . import SSM_COEF_CS, SSM_COEF_GL1, SSM_COEF_GL2, SSM_COEF_POLY
    cases = {"gl1": (SSM_COEF_GL1, 1, (1.5, 0.5), 1.0, 0.0, 1.0),
             "gl2": (SSM_COEF_GL2, 1, (1.5, 0.5), 1.0, 0.0, 1.0),
             "poly": (SSM_COEF_POLY, 1, (-1.0,), 1.0, 0.0, 2.0),
             "cs": (SSM_COEF_CS, 2, (2.0, 4.0), 1.0, math.sqrt(2.0), 2.0)}
    return {name: error_study(coef, d, T, ks, k_ref, N, seed, coef_params=p, x0_mean=m0, x0_std=s0)
            for name, (coef, d, p, m0, s0, T) in cases.items()}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="weak and strong error studies of the SSM on the GPU")
    ap.add_argument("--batch", action="store_true",
                    help="the mixed ensemble workload (64 ensembles) against h = 2^-REF_LOG2, one graph launch")
    ap.add_argument("--ref-log2", type=int, default=14)
    a = ap.parse_args()
    if a.batch:
        r = batch_study(mixed_ensembles(), ref_log2=a.ref_log2)
        r["by_h"] = {str(h): v for h, v in r["by_h"].items()}
        print(json.dumps(r))
    else:
        print(json.dumps(paper_examples()))
