"""The benchmarked configuration against the FP64 oracle, element by element.

bench.py times three 128x128x96 registrations per step: the phantom pairs of
seeds 1, 2, 3 with regulariser orders n = 1, 2, 3, s = 2, lambda = 10,
theta = 0.1, kappa = 0.5, delta = 1, 10 compositions x 10 ADMM iterations,
each registration on its own stream, in the faster of two plans (the slab
path or the four-kernel path).  Here the same pairs run the same way in both
plans (three streams, one graph replay each) and every displacement is compared
with the oracle's free-running registration (Sec. 2 outer loop after Eq. 2,
Eq. 5 and Eq. 6): max |u_gpu - u_oracle| <= 1e-3 voxel, and the Jacobian
determinant is positive everywhere on both.  One s = 1 pair at the same size
and schedule covers the L1 data term.  The concurrent results are also
checked bit for bit against the same registrations run one after another.

The oracle registrations run in a pool of spawned processes (about 30 s each
on one host core), started before any GPU work of this module.
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = (128, 128, 96)
LAM, THETA, OUTER, INNER = 10.0, 0.1, 10, 10
# (seed, order n, data term s): the bench's three pairs, then the s = 1 pair
CASES = [(1, 1, 2), (2, 2, 2), (3, 3, 2), (0, 2, 1)]


def _oracle_job(case):
    seed, n, s = case
    pair = synth.make_pair(DIMS, seed=seed)
    u = O.register(pair["fixed"], pair["moving"], lam=LAM, theta=THETA, n=n, outer=OUTER,
                   inner=INNER, s=s, kappa=0.5, delta=1.0)
    return case, u.astype(np.float64), float(O.jacobian_determinant(u).min())


@pytest.fixture(scope="module")
def oracle_results():
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(CASES)) as pool:
        res = pool.map(_oracle_job, CASES)
    return {case: (u, dmin) for case, u, dmin in res}


@pytest.fixture(scope="module")
def lib(oracle_results):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


def _nonpositive(lib, reg, u, stream):
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    lib.nadmm_jacobian_det(reg.handle, u, None, cnt, stream)
    torch.cuda.synchronize()
    return int(cnt.item())


def _run(lib, cases, concurrent, flags=0):
    dev = torch.device("cuda:0")
    nx, ny, nz = DIMS
    regs, I0, I1, U = [], [], [], []
    for seed, n, s in cases:
        pair = synth.make_pair(DIMS, seed=seed)
        I0.append(torch.from_numpy(pair["fixed"]).to(dev))
        I1.append(torch.from_numpy(pair["moving"]).to(dev))
        U.append(torch.full((3, nz, ny, nx), float("nan"), device=dev))
        regs.append(lib.Registration(DIMS, device=dev, order_n=n, lam=LAM, theta=THETA,
                                     outer=OUTER, inner=INNER, data_term=s, flags=flags))
    main = torch.cuda.current_stream(dev)
    if concurrent:  # as bench.py: one stream per registration, forked from the main one
        side = [torch.cuda.Stream(dev) for _ in cases]
        fork = torch.cuda.Event()
        fork.record(main)
        for r, a, b, u, sd in zip(regs, I0, I1, U, side):
            sd.wait_event(fork)
            lib.nadmm_register(r.handle, a, b, u, sd)
        for sd in side:
            main.wait_stream(sd)
    else:
        for r, a, b, u in zip(regs, I0, I1, U):
            lib.nadmm_register(r.handle, a, b, u, main)
    torch.cuda.synchronize()
    for r in regs:
        assert lib.nadmm_get_status(r.handle, main) == lib.NADMM_OK
    return regs, U


@pytest.mark.parametrize("plan", ["slab", "four_kernel"])
def test_benchmarked_registrations_match_oracle(lib, oracle_results, plan):
    bench_cases = CASES[:3]
    flags = {"slab": lib.NADMM_FLAG_SLAB_PATH, "four_kernel": lib.NADMM_FLAG_FOUR_PASS}[plan]
    regs, U = _run(lib, bench_cases, concurrent=True, flags=flags)
    stream = torch.cuda.current_stream()
    for case, reg, u in zip(bench_cases, regs, U):
        u_ref, det_min_ref = oracle_results[case]
        got = u.cpu().numpy().astype(np.float64)
        err = float(np.abs(got - u_ref).max())
        assert err <= 1e-3, (case, err)
        assert det_min_ref > 0.0, case
        assert _nonpositive(lib, reg, u, stream) == 0, case
    # the same registrations one after another on one stream: bit-identical
    _, U_seq = _run(lib, bench_cases, concurrent=False, flags=flags)
    for case, a, b in zip(bench_cases, U, U_seq):
        assert torch.equal(a, b), case


def test_l1_data_term_full_size_matches_oracle(lib, oracle_results):
    case = CASES[3]
    regs, U = _run(lib, [case], concurrent=False)
    u_ref, det_min_ref = oracle_results[case]
    err = float(np.abs(U[0].cpu().numpy().astype(np.float64) - u_ref).max())
    assert err <= 1e-3, err
    assert det_min_ref > 0.0
    assert _nonpositive(lib, regs[0], U[0], torch.cuda.current_stream()) == 0
