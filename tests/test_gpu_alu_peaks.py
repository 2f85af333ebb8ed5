"""The ALU roofline denominators are upper bounds of what the GPU delivers.

bench.py reports the near-field pair kernel against a peak derived from unit
counts and the maximum clock (16 MUFU rsqrt and 128 FP32 FMA per clock per
SM).  A microbenchmark (tests/alu_peaks.cu: independent chains of rsqrt, FP32
and FP64 FMA in bounded loops over 8 CTAs per SM) must not exceed those
figures, and should come within a few percent of them at the clock it ran at:
otherwise the derived peak is not the bound of the unit it names."""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_alu_peaks_bound_the_derived_roofline(tmp_path):
    import torch

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "alu_peaks")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "alu_peaks.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    m = json.loads(r.stdout)
    print(m)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert m["sms"] == sms
    fmax = 2070e6  # the SM clock limit of the part (MHz in nvidia-smi), the clock the roofline assumes
    mufu_peak = 16 * sms * fmax / 1e12      # T rsqrt/s
    fp32_peak = 2 * 128 * sms * fmax / 1e12  # TFLOP/s
    fp64_peak = 2 * 2 * sms * fmax / 1e12
    assert m["mufu_rsqrt_tops"] <= 1.02 * mufu_peak
    assert m["fp32_fma_tflops"] <= 1.02 * fp32_peak
    assert m["fp64_fma_tflops"] <= 1.02 * fp64_peak
    # packed FP32x2 FMA: at most two lanes' FMAs per FP32 lane and clock
    assert m["fp32x2_fma_tflops"] <= 1.02 * 2 * fp32_peak
    # and the units do run at their nominal widths (a clock of at least 1.5 GHz under this load)
    assert m["mufu_rsqrt_tops"] >= 16 * sms * 1.5e9 / 1e12
    assert m["fp32_fma_tflops"] >= 2 * 128 * sms * 1.5e9 / 1e12
