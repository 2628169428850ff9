"""FFT plans and stage arithmetic on the host (no GPU): the kernels' plan
(plan.h) and stages (fft_device.cuh, host build of the same functions)
against a direct DFT for smooth lengths, lane plans, and lengths with prime
factors above 7 (direct-sum stages).  The device-only part (the generic
stage's rounds between block barriers) is covered by the GPU tests."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_12688_gb300", "csrc")
SMOOTH = [4, 6, 8, 12, 20, 24, 96, 112, 128, 160, 192, 256]
PRIME = [11, 13, 23, 26, 34, 44, 97, 104, 143, 194, 251, 508, 858]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_plan_check")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "host", "fft_plan_check.cu")], check=True)
    out = subprocess.run([exe] + [str(n) for n in SMOOTH + PRIME], check=True,
                         capture_output=True, text=True).stdout
    res = {}
    for line in out.strip().splitlines():
        head, _, tail = line.partition("|")
        fields = head.split()
        err, rt, twc = tail.split()
        res[int(fields[0])] = (fields[1:], float(err), float(rt), int(twc))
    return res


@pytest.mark.parametrize("n", SMOOTH + PRIME)
def test_forward_stages_are_the_dft_and_invert(results, n):
    radices, err, rt, _ = results[n]
    prod = 1
    for r in radices:
        prod *= int(r.rstrip("g"))
    assert prod == n
    assert err <= 1e-6       # relative to the largest |X_k|
    assert rt <= 5e-6        # inverse stages / n give the input back


@pytest.mark.parametrize("n", PRIME)
def test_primes_above_7_are_generic_stages_first(results, n):
    radices, _, _, twc = results[n]
    generic = [int(r[:-1]) for r in radices if r.endswith("g")]
    codelet = [int(r) for r in radices if not r.endswith("g")]
    assert generic and all(r > 7 for r in generic)
    assert all(r <= 16 for r in codelet)
    assert radices[:len(generic)] == [f"{r}g" for r in generic]  # generic stages lead
    assert twc >= sum(generic)  # the roots w_r^q follow the stage twiddles


@pytest.mark.parametrize("n", [96, 128, 112])
def test_lane_plans_are_two_stages(results, n):
    radices, _, _, _ = results[n]
    assert len(radices) == 2 and int(radices[1]) in (8, 16)
