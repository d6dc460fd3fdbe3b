"""The bounds-checked debug build on the GPU, on small and ragged cases.

Run in a child process that loads libssm_check.so (SSM_LIB_VARIANT=check): the
coupled set at N in {1, 2, 3, 7, 8, 33} (FP64 against the oracle per particle to
1e-10 relative, FP32C to 2e-6 over four steps), the cubic set at N = 7,
and the batched form at two small ensembles, must run without an index leaving its
array (status SSM_OK); then a context whose step-1 start plants particle index N
in its active list (ssm_opts.inject = 1; inside the padded arrays, so nothing
outside an allocation is touched even if a check were missing) must report
SSM_EBOUNDS at its next synchronising call.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _child():
    sys.path.insert(0, ROOT)
    import oracle as O
    import paper_2105_09688_gb300 as S
    out = {"flags": int(S.lib().ssm_build_flags())}
    worst = 0.0
    for N in (1, 2, 3, 7, 8, 33):
        for prec in (S.SSM_FP64, S.SSM_FP32C):
            s = S.SSM(d=3, N=N, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=5, precision=prec)
            s.run_steps(4)
            x, _ = s.get_state()
            s.close()
            P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=2.0 ** -8, seed=5)
            xo = O.run(P, O.init_x0(P), 0, 4)
            err = float(np.max(np.abs(x - xo) / np.maximum(1.0, np.abs(xo))))
            if prec == S.SSM_FP64:
                assert err < 1e-10, (N, err)
            else:
                assert err < 2e-6, (N, err)
            worst = max(worst, err)
    # several target tiles: passes over part of the particles repack the pair kernel's
    # blocks and partial sums (the partial-pass chunking), here under the index checks
    for N in (3000, 5000):
        s = S.SSM(d=3, N=N, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=6, precision=S.SSM_FP32C)
        s.run_steps(3)
        x, _ = s.get_state()
        st = s.stats()
        s.close()
        P = O.problem(d=3, coef=O.COEF_COUPLED3D, N=N, h=2.0 ** -8, seed=6)
        xo = O.run(P, O.init_x0(P), 0, 3)
        assert np.max(np.abs(x - xo)) < 2e-6
        assert st["newton_rows"] < st["newton_passes"] * N     # some passes were partial
    s = S.SSM(d=1, N=7, h=0.01, T=1.0, coef=S.SSM_COEF_CUBIC1D_GAUSS, seed=0)
    s.run_steps(3)
    s.sync()
    s.close()
    b = S.Batch([dict(d=1, N=33, h=2.0 ** -4, T=0.25, seed=1), dict(d=3, N=7, h=2.0 ** -5, T=0.25, seed=2)],
                precision=S.SSM_FP32C)
    b.run()
    b.sync()
    b.close()
    out["clean_worst_rel_err"] = worst
    # the planted index
    s = S.SSM(d=3, N=33, h=2.0 ** -8, T=1.0, coef=S.SSM_COEF_COUPLED3D, seed=5, precision=S.SSM_FP32C, inject=1)
    s.step()
    try:
        s.sync()
        out["planted"] = "SSM_OK"
    except S.SSMError as e:
        out["planted"] = S.ssm_status_str(e.status).split(":")[0]
    print("CHILD_RESULT " + json.dumps(out))


def test_debug_build_small_cases_and_planted_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_09688_gb300 import build as B
    B.build(check_bounds=True)
    env = dict(os.environ, SSM_LIB_VARIANT="check")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "child"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("CHILD_RESULT ")][-1]
    res = json.loads(line[len("CHILD_RESULT "):])
    assert res["flags"] == 1
    assert res["planted"] == "SSM_EBOUNDS", res


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "child":
    _child()
