"""nadmm_spectral_solve_noalloc against nadmm_spectral_solve.

The no-allocation entry point serves callers that may not allocate device
memory themselves (a library inside an application that owns every device
allocation, or a latency-critical caller that cannot risk cudaMalloc's
device synchronisation).  It keeps its scratch in one static device array
shared by every call.  This file is collected last so that, in a run that
stops at the first failure, every other test has already run; it also passes
when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


@pytest.mark.parametrize("dims,n", [((32, 32, 24), 2), ((128, 128, 96), 3), ((20, 12, 14), 1)])
def test_noalloc_matches_workspace_entry_on_two_calls(lib, dims, n):
    nx, ny, nz = dims
    lam, theta = 10.0, 0.1
    stream = torch.cuda.current_stream()
    reg = lib.Registration(dims, device="cuda:0", order_n=n, lam=lam, theta=theta)
    for call, seed in enumerate((11, 12)):        # two calls in a row, different inputs
        y = torch.from_numpy(synth.random_field((3, nz, ny, nx), seed=seed)).cuda()
        w_ref = torch.empty_like(y)
        w_new = torch.full_like(y, float("nan"))
        lib.nadmm_spectral_solve(reg.handle, y, w_ref, stream)
        lib.nadmm_spectral_solve_noalloc(nx, ny, nz, n, lam, theta, y, w_new, stream)
        torch.cuda.synchronize()
        a = w_new.cpu().numpy().astype(np.float64)
        b = w_ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all(), call
        # same tolerance as the spectral-solve parity tests against the oracle
        assert np.abs(a - b).max() <= 2e-6 * float(y.abs().max()), call
        assert rel_l2(a, b) <= 1e-6, call
    reg.close()


def test_noalloc_rejects_grids_beyond_its_array(lib):
    y = torch.zeros(16, device="cuda:0")
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve_noalloc(160, 160, 112, 2, 10.0, 0.1, y, y)
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert "24 MiB" in str(e.value)
