"""The hardware facts the kernels' design rests on, measured by a small CUDA
program (tests/probes/fp64_pipe.cu): the FP64 FMA peak the roofline uses, a
masked lane costing as much as an active one, one warp per SM sub-partition
sufficing for the FP64 pipe, and FP64 tensor-core MMA being slower than
DFMA and sharing its pipe (so it is not used, not even beside DFMA)."""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
PEAK_GFLOPS = 152 * 2 * 2 * 2.070


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "fp64_pipe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "probes", "fp64_pipe.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=300).stdout
    res = json.loads(out.strip().splitlines()[-1])
    print(json.dumps(res))
    assert "error" not in res
    return res


def test_dfma_peak_close_to_the_derived_unit_count(probe):
    # 152 SMs x 2 FP64 FMA lanes x 2 flops x 2.07 GHz; clocks may sit below the maximum
    assert 0.85 * PEAK_GFLOPS <= probe["dfma_full_gflops"] <= 1.02 * PEAK_GFLOPS


def test_a_masked_lane_costs_as_much_as_an_active_one(probe):
    assert 0.9 <= probe["dfma_1lane_ratio"] <= 1.1


def test_one_warp_per_sm_subpartition_feeds_the_fp64_pipe(probe):
    assert probe["dfma_ilp1_4warps_gflops"] >= 0.85 * probe["dfma_full_gflops"]


def test_fp64_mma_is_slower_than_dfma(probe):
    assert probe["dmma_gflops"] < probe["dfma_full_gflops"]


def test_fp64_mma_and_dfma_share_one_pipe(probe):
    # half the warps in each loop: together they take about the sum of their
    # times alone, not the longer of the two
    both, f, m = probe["mixed_ms_both"], probe["mixed_ms_dfma_only"], probe["mixed_ms_mma_only"]
    assert both >= 0.85 * (f + m)
