"""Weak and strong errors of the SSM against a finer step on the same Brownian paths,
as §3 measures them (the paper's eq. for epsilon_k):
    epsilon_1 = | (1/N) sum_j (X_T^j - Xhat_T^j) |_2      (weak, k = 1)
    epsilon_2 = ( (1/N) sum_j |X_T^j - Xhat_T^j|^2 )^(1/2)  (strong, k = 2)
where X_T is the run at the fine step (the paper's proxy for the true solution)
and Xhat_T the run at step h; every run samples its increments from the Brownian
path on the fine grid (ssm_opts.fine_log2), so all of them share one path.
Every step runs in the library's GPU kernels.
"""
import math

import numpy as np

from . import SSM, SSM_FP64


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
        weak.append(float(np.linalg.norm(np.mean(x - ref, axis=0))))
        strong.append(math.sqrt(float(np.mean(np.sum((x - ref) ** 2, axis=1)))))
    lh = np.log2(hs)
    return dict(h=hs, weak=weak, strong=strong, weak_slope=float(np.polyfit(lh, np.log2(weak), 1)[0]),
                strong_slope=float(np.polyfit(lh, np.log2(strong), 1)[0]))


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
    import json
    print(json.dumps(paper_examples()))
