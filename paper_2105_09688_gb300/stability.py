"""Mean-square stability of the SSM: the constant beta of the stability theorem of §2
(eq. (SSTM:beta formula)) for the paper's two examples, and the curves of §3.4.2 --
t -> E|X_t|^2 and the mean-square distance of two runs driven by the same noise --
computed with the library's GPU kernels (the Ginzburg-Landau stability example is
SSM_COEF_GLSTAB).  Every step runs on the device; these functions only read the
state or the moments back after each step.
"""
import numpy as np

from . import SSM, SSM_COEF_GLSTAB, SSM_FP64, ssm_stability_beta


def ou_constants(rho, lam):
    """§3.4.1: L_v = rho, L_bt = lambda^2, the others zero."""
    return dict(Lv=rho, Lvt=0.0, Lb=0.0, Lbt=lam * lam, Ls=0.0, Lst=0.0)


def glstab_constants(gamma):
    """§3.4.2: L_v = -5/2 - gamma, L_bt = L_s = 1, L_b = gamma^2, L_vt = L_st = 0."""
    return dict(Lv=-2.5 - gamma, Lvt=0.0, Lb=gamma * gamma, Lbt=1.0, Ls=1.0, Lst=0.0)


def beta(h, Lv, Lvt, Lb, Lbt, Ls, Lst):
    return ssm_stability_beta(Lv, Lvt, Lb, Lbt, Ls, Lst, h)


def _glstab(gamma, h, T, N, x0, seed, precision, stream=None):
    return SSM(d=1, N=N, h=h, T=T, coef=SSM_COEF_GLSTAB, seed=seed, stream=stream, precision=precision,
               coef_params=(gamma,), x0_mean=x0, x0_std=0.0)


def second_moment_curve(gamma, h, T, N=1000, x0=1.0, seed=0, precision=SSM_FP64):
    """(t_n, (1/N) sum_i |X_n^i|^2) for n = 0..M of the GL stability example."""
    s = _glstab(gamma, h, T, N, x0, seed, precision)
    M = int(round(T / h))
    out = [float(s.moments()[1, 0])]
    for _ in range(M):
        s.step()
        out.append(float(s.moments()[1, 0]))
    s.close()
    return np.arange(M + 1) * h, np.array(out)


def contraction_curve(gamma, h, T, x0, z0, N=1000, seed=0, precision=SSM_FP64):
    """(t_n, (1/N) sum_i |X_n^i - Z_n^i|^2) for two runs from X_0 = x0 and Z_0 = z0
    driven by the same Brownian paths (same seed)."""
    a = _glstab(gamma, h, T, N, x0, seed, precision)
    b = _glstab(gamma, h, T, N, z0, seed, precision)
    M = int(round(T / h))
    out = [float((x0 - z0) ** 2)]
    for _ in range(M):
        a.step()
        b.step()
        out.append(float(np.mean((a.get_state()[0] - b.get_state()[0]) ** 2)))
    a.close()
    b.close()
    return np.arange(M + 1) * h, np.array(out)


def gamma_sweep(gammas=(-12.0, -8.0, -4.0, 0.0, 2.0, 4.0, 6.0, 8.0, 12.0), h=0.1, T=3.0, N=1000, seed=0):
    """The §3.4.2 experiment at the paper's step h = 0.1: for each gamma, beta of the
    stability theorem and, from two runs X_0 = 1, Z_0 = 5 on the same Brownian paths,
    the observed mean-square contraction factor per step
    ((1/N) sum |X_M - Z_M|^2 / |1 - 5|^2)^(1/M), next to the theorem's 1 + beta h
    (a bound where theorem_applies, i.e. 1 - h (2 L_v + 1) > 0, and beta < 0),
    and E|X_T|^2 from X_0 = 1.  Returns a list of dicts."""
    out = []
    for g in gammas:
        b = beta(h, **glstab_constants(g))
        t, d2 = contraction_curve(g, h, T, 1.0, 5.0, N=N, seed=seed)
        _, m2 = second_moment_curve(g, h, T, N=N, x0=1.0, seed=seed)
        M = t.size - 1
        k = glstab_constants(g)
        out.append(dict(gamma=g, beta=b, theorem_applies=bool(1.0 - h * (2.0 * k["Lv"] + 1.0) > 0.0),
                        theorem_factor=1.0 + b * h, observed_factor=float((d2[-1] / d2[0]) ** (1.0 / M)),
                        m2_T=float(m2[-1])))
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(gamma_sweep()))
