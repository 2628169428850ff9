"""Adaptive restart of the Nesterov momentum (reading R20) on the GPU against
the FP64 oracle's admm_restart, through the C ABI.

The restart test of iteration k needs the grid-wide residual c_k, which is
complete only after the pass that already forms w_hat^{k+1}; the decision
therefore restarts the momentum at iteration k + 2, on both sides.
"""
import math

import numpy as np
import pytest

import oracle as O
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _oracle_with_counts(pair, lam, theta, n, outer, inner, eta):
    """oracle.register with restart, also counting the restarts (the loop of
    oracle.register spelled out with the oracle's own steps)."""
    I0 = pair["fixed"].astype(np.float64)
    I1 = pair["moving"].astype(np.float64)
    u = np.zeros((3,) + I0.shape)
    J, c, _ = O.linearise(I0, I1, u)
    count = 0
    for o in range(outer):
        h = O.admm_restart(J, c, lam, theta, n, inner, eta=eta, history=True)
        count += sum(1 for k in h["restart"] if k + 2 < inner)  # decisions that take effect
        sc, _, _ = O.bound_scale(h["w"][-1], 0.5, 1.0)
        u = O.compose(u, sc * h["w"][-1])
        if o + 1 < outer:
            J, c, _ = O.linearise(I0, I1, u)
    ref = O.register(I0, I1, lam=lam, theta=theta, n=n, outer=outer, inner=inner, restart_eta=eta)
    assert np.array_equal(ref, u)
    return u, count


# (dims, n, lambda, theta, outer, inner); the 128x128x96 case restarts at
# iterations 21-25 of its first outer step, each test decided by a margin of
# at least 3.8 % (FP64), far above FP32 rounding
@pytest.mark.parametrize("dims,n,lam,theta,outer,inner", [((32, 32, 24), 2, 10.0, 0.02, 3, 20),
                                                          ((32, 32, 24), 1, 10.0, 0.01, 2, 25),
                                                          ((128, 128, 96), 1, 1.0, 0.01, 2, 30)])
def test_restart_registration_matches_oracle(lib, dims, n, lam, theta, outer, inner):
    """A weakly convex setting (theta well below |grad I|^2 at the edges),
    where restarts happen: same displacement (1e-3 voxel) and the same
    number of restarts as the oracle."""
    pair = synth.make_pair(dims, seed=5)
    u_ref, count = _oracle_with_counts(pair, lam, theta, n, outer, inner, 0.999)
    reg = lib.Registration(dims, device="cuda:0", order_n=n, lam=lam, theta=theta, outer=outer,
                           inner=inner, restart_eta=0.999)
    u = reg.register(_dev(pair["fixed"]), _dev(pair["moving"]))
    stream = torch.cuda.current_stream()
    assert lib.nadmm_get_status(reg.handle, stream) == lib.NADMM_OK
    got = lib.nadmm_get_restarts(reg.handle, stream)
    assert count >= 1
    assert got == count
    assert np.abs(u.cpu().numpy().astype(np.float64) - u_ref).max() <= 1e-3


def test_restart_extremes(lib):
    """eta = inf never restarts: bit-identical to the handle without restart;
    eta = 0 restarts at every test: plain ADMM (every factor 0) as in the
    oracle with accelerate=False."""
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed=2)
    I0, I1 = _dev(pair["fixed"]), _dev(pair["moving"])
    kw = dict(device="cuda:0", order_n=2, lam=10.0, theta=0.1, outer=2, inner=8)
    # restart runs on the slab path; the handle without it is put there too
    plain_gpu = lib.Registration(dims, flags=lib.NADMM_FLAG_SLAB_PATH, **kw).register(I0, I1)
    never = lib.Registration(dims, restart_eta=math.inf, **kw)
    u_never = never.register(I0, I1)
    torch.cuda.synchronize()
    assert torch.equal(u_never, plain_gpu)
    assert lib.nadmm_get_restarts(never.handle, torch.cuda.current_stream()) == 0
    always = lib.Registration(dims, restart_eta=0.0, **kw)
    u_always = always.register(I0, I1).cpu().numpy().astype(np.float64)
    ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=8,
                     accelerate=False)
    assert np.abs(u_always - ref).max() <= 1e-3
    # the momentum was restarted after each of the first inner - 2 tests per outer step
    assert lib.nadmm_get_restarts(always.handle, torch.cuda.current_stream()) == 2 * (8 - 2)
