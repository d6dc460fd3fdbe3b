"""ssm_drift_noalloc, the drift entry point that allocates nothing.

Callers that cannot allocate device memory where they need the drift (host
callbacks, real-time loops that must not block on the allocator, runtimes with one
pre-reserved pool) use ssm_drift_noalloc, whose scratch is a fixed static device
array inside the library.  Here it is called through the C ABI on device arrays
the test owns, twice in a row, and compared with the drift the context's own step
reports through ssm_get_stage(SSM_STAGE_B) for the same Y.  Tolerances: FP64
1e-10 relative (the FP64 parity bound of the other tests); FP32C 1e-9 absolute
(the two paths group the same FP32 sub-tile sums differently).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    return torch, S


@pytest.mark.parametrize("case", ["cubic1d_fp64", "coupled3d_fp32c", "coupled3d_fp64"])
def test_noalloc_drift_matches_the_context_drift_twice(env, case):
    torch, S = env
    coef, d, prec, N, h = {
        "cubic1d_fp64": (S.SSM_COEF_CUBIC1D_GAUSS, 1, S.SSM_FP64, 2000, 2.0 ** -10),
        "coupled3d_fp32c": (S.SSM_COEF_COUPLED3D, 3, S.SSM_FP32C, 3000, 2.0 ** -8),
        "coupled3d_fp64": (S.SSM_COEF_COUPLED3D, 3, S.SSM_FP64, 700, 2.0 ** -8),
    }[case]
    s = S.SSM(d=d, N=N, h=h, T=1.0, coef=coef, seed=7, precision=prec)
    s.step()
    y = s.get_stage(S.SSM_STAGE_Y)
    b_ref = s.get_stage(S.SSM_STAGE_B)
    s.close()

    ld = N + 5                                   # leading dimension != N
    ydev = torch.zeros((d, ld), dtype=torch.float64, device="cuda")
    ydev[:, :N] = torch.from_numpy(np.ascontiguousarray(y.T)).cuda()
    bdev = torch.empty((d, ld), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        bdev.fill_(float("nan") if call == 0 else 1e300)   # the output is fully rewritten each call
        S.ssm_drift_noalloc(coef, prec, N, ydev.data_ptr(), ld, bdev.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        b = bdev[:, :N].cpu().numpy().T
        assert np.all(np.isfinite(b))
        if prec == S.SSM_FP64:
            assert np.max(np.abs(b - b_ref) / np.maximum(1.0, np.abs(b_ref))) < 1e-10, call
        else:
            assert np.max(np.abs(b - b_ref)) < 1e-9, call


@pytest.mark.parametrize("case", ["cubic1d_fp64", "coupled3d_fp32c"])
def test_noalloc_drift_matches_the_oracle(env, case):
    """The same entry point against the FP64 oracle's drift b(Y_i, mu^Y) of every
    particle, on a seeded cloud: FP64 1e-10 relative; FP32C 5e-7 absolute (the
    bound the pair-kernel shapes meet against the oracle)."""
    import oracle as O
    from tests import inputs
    torch, S = env
    coef, ocoef, d, prec, N = {
        "cubic1d_fp64": (S.SSM_COEF_CUBIC1D_GAUSS, O.COEF_CUBIC1D_GAUSS, 1, S.SSM_FP64, 1500),
        "coupled3d_fp32c": (S.SSM_COEF_COUPLED3D, O.COEF_COUPLED3D, 3, S.SSM_FP32C, 2500),
    }[case]
    y = inputs.heavy_cloud(N, d, seed=81)
    ydev = torch.from_numpy(np.ascontiguousarray(y.T)).cuda()
    bdev = torch.empty((d, N), dtype=torch.float64, device="cuda")
    S.ssm_drift_noalloc(coef, prec, N, ydev.data_ptr(), N, bdev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    b = bdev.cpu().numpy().T
    P = O.problem(d=d, coef=ocoef, N=N, h=2.0 ** -8)
    bo = np.stack([O.drift_one(P, y, i) for i in range(N)])
    if prec == S.SSM_FP64:
        assert np.max(np.abs(b - bo) / np.maximum(1.0, np.abs(bo))) < 1e-10
    else:
        assert np.max(np.abs(b - bo)) < 5e-7


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, S = env
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SSMError) as e:
        S.ssm_drift_noalloc(S.SSM_COEF_COUPLED3D, S.SSM_FP32C, 349526, buf.data_ptr(), 349526, buf.data_ptr())
    assert e.value.status == S.SSM_ENOMEM
    with pytest.raises(S.SSMError) as e:
        S.ssm_drift_noalloc(S.SSM_COEF_COUPLED3D, S.SSM_FP32C, 100, buf.data_ptr(), 50, buf.data_ptr())
    assert e.value.status == S.SSM_EINVAL
