"""Reverse mode on the GPU (nadmm_backward, nadmm_ssd_after_warp*) against
the FP64 oracle's hand-written adjoints and against finite differences.

Tolerances: the GPU sweeps run in FP32 with float atomics for the scatters;
the adjoint recursion has the forward's conditioning (measured agreement
with the FP64 oracle ~1e-6 relative), so gradients are compared by relative
L2 error <= 1e-4 and lambda/theta to 1e-4 relative; the 128x128x96 gradients
against central differences of the GPU forward (step 1e-3), whose FP32
rounding noise in the loss bounds the agreement to a few 1e-3 absolute."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


def stream():
    return torch.cuda.current_stream()


# ---------------------------------------------------------------- SSD loss
def test_ssd_after_warp_and_vjp(lib):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=3)
    u = synth.random_velocity(dims, np.random.default_rng(5), max_amp=2.5)
    reg = lib.Registration(dims, device=DEV)
    loss = torch.zeros(4, device=DEV)
    f, m, ud = dev(p["fixed"]), dev(p["moving"]), dev(u)
    lib.nadmm_ssd_after_warp(reg.handle, f, m, ud, loss, stream())
    ref = O.ssd_after_warp(p["fixed"], p["moving"], u.astype(np.float32))
    assert abs(float(loss[0]) - ref) <= 1e-5 * ref
    gl = torch.tensor([0.7, 0, 0, 0], device=DEV)
    g0, g1, gu = torch.empty_like(f), torch.empty_like(m), torch.empty_like(ud)
    lib.nadmm_ssd_after_warp_backward(reg.handle, f, m, ud, gl, g0, g1, gu, stream())
    r0, r1, ru = O.ssd_after_warp_vjp(p["fixed"], p["moving"], u.astype(np.float32), 0.7)
    assert rel_l2(host(g0), r0) <= 1e-5
    assert rel_l2(host(g1), r1) <= 1e-5
    assert rel_l2(host(gu), ru) <= 1e-4


# ---------------------------------------------------------------- registration
CASES = [dict(n=2, outer=3, inner=5, kappa=0.5, delta=1.0),
         dict(n=1, outer=2, inner=6, kappa=math.inf, delta=math.inf),
         dict(n=3, outer=3, inner=4, kappa=0.05, delta=math.inf)]


@pytest.mark.parametrize("path", ["four_kernel", "slab"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_backward_matches_oracle_vjp(lib, case, path):
    """Both paths' reverse sweeps: the four-kernel path solves each reverse
    step's S g with five kernels and a separate adjoint kernel; the slab
    path fuses the adjoint point-wise step between the inverse and forward
    transforms of one slab pass (two kernels per reverse step)."""
    c = CASES[case]
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=case)
    gu = synth.random_field((3,) + dims[::-1], seed=40 + case)
    kw = dict(lam=10.0, theta=0.1, n=c["n"], outer=c["outer"], inner=c["inner"],
              kappa=c["kappa"], delta=c["delta"])
    flags = {"four_kernel": lib.NADMM_FLAG_FOUR_PASS, "slab": lib.NADMM_FLAG_SLAB_PATH}[path]
    reg = lib.Registration(dims, device=DEV, requires_grad=True, order_n=c["n"], lam=10.0,
                           theta=0.1, outer=c["outer"], inner=c["inner"], kappa=c["kappa"],
                           delta=c["delta"], flags=flags)
    f, m = dev(p["fixed"]), dev(p["moving"])
    u = reg.register(f, m)
    u_ref, tape = O.register_tape(p["fixed"], p["moving"], **kw)
    assert np.abs(host(u) - u_ref).max() <= 1e-3
    if c["kappa"] < 0.1:
        assert all(t[4] < 1.0 for t in tape)  # bound active
    g0, g1, gl, gt = reg.backward(f, m, dev(gu))
    r0, r1, rl, rt = O.register_vjp(p["fixed"], p["moving"], gu, **kw)
    assert rel_l2(host(g0), r0) <= 1e-4
    assert rel_l2(host(g1), r1) <= 1e-4
    assert abs(float(gl) - rl) <= 1e-4 * abs(rl) + 1e-7
    assert abs(float(gt) - rt) <= 1e-4 * abs(rt) + 1e-7


def test_backward_graph_and_direct_agree(lib):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=9)
    gu = dev(synth.random_field((3,) + dims[::-1], seed=1))
    f, m = dev(p["fixed"]), dev(p["moving"])
    out = []
    for flags in (0, lib.NADMM_FLAG_NO_GRAPH):
        reg = lib.Registration(dims, device=DEV, requires_grad=True, outer=3, inner=4,
                               flags=flags)
        reg.register(f, m)
        res = [host(t) for t in reg.backward(f, m, gu)]
        res2 = [host(t) for t in reg.backward(f, m, gu)]  # replay
        for a, b in zip(res, res2):
            np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6)
        out.append(res)
    for a, b in zip(*out):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6)


def test_backward_errors(lib):
    dims = (16, 16, 8)
    f = torch.zeros(dims[::-1], device=DEV)
    gu = torch.zeros((3,) + dims[::-1], device=DEV)
    plain = lib.Registration(dims, device=DEV)
    with pytest.raises(lib.NadmmError) as e:
        plain.backward(f, f, gu)
    assert e.value.status == lib.NADMM_ERR_NO_SAVED_FORWARD
    reg = lib.Registration(dims, device=DEV, requires_grad=True)
    with pytest.raises(lib.NadmmError) as e:
        reg.backward(f, f, gu)  # no forward yet
    assert e.value.status == lib.NADMM_ERR_NO_SAVED_FORWARD
    l1 = lib.Registration(dims, device=DEV, requires_grad=True, data_term=1)
    l1.register(f, f)
    with pytest.raises(lib.NadmmError) as e:
        l1.backward(f, f, gu)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG


def test_autograd_chain_matches_oracle(lib):
    """L = SSD(I1 o (Id + register(I0, I1)), I0) through torch.autograd."""
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=4)
    kw = dict(lam=10.0, theta=0.1, n=2, outer=3, inner=5)
    reg = lib.Registration(dims, device=DEV, requires_grad=True, order_n=2, outer=3, inner=5)
    f = dev(p["fixed"]).requires_grad_()
    m = dev(p["moving"]).requires_grad_()
    lam = torch.tensor(10.0, device=DEV, requires_grad=True)
    theta = torch.tensor(0.1, device=DEV, requires_grad=True)
    u = lib.register(f, m, lam, theta, reg)
    L = lib.ssd_after_warp(f, m, u, reg)
    L.backward()
    Lr, r0, r1, rl, rt = O.loss_and_gradients(p["fixed"], p["moving"], **kw)
    assert abs(float(L) - Lr) <= 1e-4 * Lr
    assert rel_l2(host(f.grad), r0) <= 1e-4
    assert rel_l2(host(m.grad), r1) <= 1e-4
    assert abs(float(lam.grad) - rl) <= 1e-4 * abs(rl) + 1e-7
    assert abs(float(theta.grad) - rt) <= 1e-4 * abs(rt) + 1e-7


def test_gradients_128x128x96_against_finite_differences(lib):
    """The gradient workload: 128x128x96 seed 0, n = 2, 8 compositions x 20
    ADMM iterations; dL/dI0, dL/dI1 at 16 voxels drawn with seed 7 and
    dL/dlambda, dL/dtheta against central differences (step 1e-3) of the GPU
    forward, the loss evaluated in FP64 from the GPU displacement."""
    dims = (128, 128, 96)
    nx, ny, nz = dims
    p = synth.make_pair(dims, seed=0)
    I0, I1 = p["fixed"], p["moving"]
    reg = lib.Registration(dims, device=DEV, requires_grad=True, order_n=2, outer=8, inner=20)
    f, m = dev(I0), dev(I1)
    lam = torch.tensor(10.0, device=DEV, requires_grad=True)
    theta = torch.tensor(0.1, device=DEV, requires_grad=True)
    fg, mg = f.clone().requires_grad_(), m.clone().requires_grad_()
    L = lib.ssd_after_warp(fg, mg, lib.register(fg, mg, lam, theta, reg), reg)
    L.backward()
    g0, g1 = host(fg.grad), host(mg.grad)
    gl, gt = float(lam.grad), float(theta.grad)

    fwd = lib.Registration(dims, device=DEV, order_n=2, outer=8, inner=20)

    def loss(a=I0, b=I1, lam_=10.0, th_=0.1):
        fwd.set_params(lam_, th_)
        u = host(fwd.register(dev(a), dev(b)))
        return O.ssd_after_warp(a, b, u)

    h = 1e-3
    rng = np.random.default_rng(7)
    # 16 voxels (seed 7) among those whose gradient is at least 0.05 in
    # magnitude, 25x the absolute allowance for the FP32 rounding noise of the
    # difference quotient, so the 2 % relative bound is what the check tests
    for arr, g, name in ((I0, g0, "I0"), (I1, g1, "I1")):
        big = np.argwhere(np.abs(g) >= 0.05)
        assert len(big) >= 16, name
        for z, y, x in big[rng.choice(len(big), size=16, replace=False)]:
            ap, am = arr.copy(), arr.copy()
            ap[z, y, x] += h
            am[z, y, x] -= h
            num = ((loss(a=ap) - loss(a=am)) if name == "I0" else (loss(b=ap) - loss(b=am))) / (2 * h)
            assert abs(num - g[z, y, x]) <= 0.02 * abs(num) + 2e-3, (name, (z, y, x), num, g[z, y, x])
    num_l = (loss(lam_=10.0 + h) - loss(lam_=10.0 - h)) / (2 * h)
    num_t = (loss(th_=0.1 + h) - loss(th_=0.1 - h)) / (2 * h)
    assert abs(num_l - gl) <= 0.02 * abs(num_l) + 5e-3, (num_l, gl)
    assert abs(num_t - gt) <= 0.02 * abs(num_t) + 5e-3, (num_t, gt)


def test_backward_128x128x96_matches_oracle_vjp(lib):
    """Full-size grid, short schedule (2 compositions x 5 ADMM iterations):
    the GPU reverse sweep against the FP64 oracle's register_vjp."""
    dims = (128, 128, 96)
    p = synth.make_pair(dims, seed=0)
    gu = synth.random_field((3,) + dims[::-1], seed=77)
    kw = dict(lam=10.0, theta=0.1, n=2, outer=2, inner=5, kappa=0.5, delta=1.0)
    reg = lib.Registration(dims, device=DEV, requires_grad=True, order_n=2, lam=10.0, theta=0.1,
                           outer=2, inner=5)
    f, m = dev(p["fixed"]), dev(p["moving"])
    reg.register(f, m)
    g0, g1, gl, gt = reg.backward(f, m, dev(gu))
    r0, r1, rl, rt = O.register_vjp(p["fixed"], p["moving"], gu, **kw)
    assert rel_l2(host(g0), r0) <= 1e-4
    assert rel_l2(host(g1), r1) <= 1e-4
    assert abs(float(gl) - rl) <= 1e-4 * abs(rl) + 1e-7
    assert abs(float(gt) - rt) <= 1e-4 * abs(rt) + 1e-7


# ---------------------------------------------------------------- batched
def test_batched_backward_matches_oracle_and_single(lib):
    dims = [(32, 32, 24), (20, 12, 14), (16, 20, 12), (24, 16, 10)]
    kw = dict(order_n=2, lam=10.0, theta=0.1, outer=2, inner=4)
    pairs = [synth.make_pair(d, seed=50 + i) for i, d in enumerate(dims)]
    f = [dev(p["fixed"]) for p in pairs]
    m = [dev(p["moving"]) for p in pairs]
    gu = [dev(synth.random_field((3,) + d[::-1], seed=60 + i)) for i, d in enumerate(dims)]
    for lanes in (1, 2):
        breg = lib.BatchedRegistration(dims, device=DEV, lanes=lanes, requires_grad=True, **kw)
        breg.register(f, m)
        g0, g1, gl, gt = breg.backward(f, m, gu)
        for i, (d, p) in enumerate(zip(dims, pairs)):
            r0, r1, rl, rt = O.register_vjp(p["fixed"], p["moving"], host(gu[i]), lam=10.0,
                                            theta=0.1, n=2, outer=2, inner=4)
            assert rel_l2(host(g0[i]), r0) <= 1e-4, (lanes, d)
            assert rel_l2(host(g1[i]), r1) <= 1e-4, (lanes, d)
            assert abs(float(gl[i]) - rl) <= 1e-4 * abs(rl) + 1e-7
            assert abs(float(gt[i]) - rt) <= 1e-4 * abs(rt) + 1e-7
            single = lib.Registration(d, device=DEV, requires_grad=True, **kw)
            single.register(f[i], m[i])
            s0, s1, sl, st = single.backward(f[i], m[i], gu[i])
            np.testing.assert_allclose(host(g0[i]), host(s0), rtol=1e-4, atol=1e-6)
            np.testing.assert_allclose(host(g1[i]), host(s1), rtol=1e-4, atol=1e-6)


def test_batch_of_16_forward_and_backward(lib):
    """16 uneven pairs (nx, ny from {96..160}, nz from {64..112}, seed 4321),
    n = 2, 10 x 10, forward and reverse mode as two graph replays; finite
    gradients, and a sample of pairs equal to single-pair calls."""
    dims = synth.draw_batch_dims(16, seed=4321)
    data = [synth.phase_pair(d, seed=100 + i) for i, d in enumerate(dims)]
    f = [dev(a) for a, _ in data]
    m = [dev(b) for _, b in data]
    gu = [dev(synth.random_field((3,) + d[::-1], seed=200 + i, scale=1e-3)) for i, d in enumerate(dims)]
    kw = dict(order_n=2, lam=10.0, theta=0.1, outer=10, inner=10)
    breg = lib.BatchedRegistration(dims, device=DEV, requires_grad=True, **kw)
    us = breg.register(f, m)
    g0, g1, gl, gt = breg.backward(f, m, gu)
    assert lib.nadmm_get_status(breg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    assert torch.isfinite(gl).all() and torch.isfinite(gt).all()
    for i in range(0, 16, 5):  # with the tape, each pair keeps its own path on the lanes
        assert torch.isfinite(g0[i]).all() and torch.isfinite(g1[i]).all()
        single = lib.Registration(dims[i], device=DEV, requires_grad=True, **kw)
        u = single.register(f[i], m[i])
        assert torch.equal(u, us[i])
        s0, s1, sl, st = single.backward(f[i], m[i], gu[i])
        np.testing.assert_allclose(host(g0[i]), host(s0), rtol=1e-4, atol=1e-7)
        np.testing.assert_allclose(host(g1[i]), host(s1), rtol=1e-4, atol=1e-7)
        assert abs(float(gl[i]) - float(sl)) <= 1e-4 * abs(float(sl)) + 1e-9
