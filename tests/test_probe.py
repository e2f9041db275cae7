"""fr_probe_fp32_peak: the measured FP32 FMA rate that checks the insertion's
ALU roofline denominator (SMs x 128 lanes x 2 flops x SM clock).

* CPU: argument errors are returned before any CUDA call.
* GPU: the scalar FMA-chain rate lies between half of and just above the
  nominal rate at the device's maximum SM clock (it cannot exceed it), and
  the packed two-lane form is no slower than the scalar one.
"""
import shutil
import subprocess

import pytest
import torch

from paper_1910_08498_gb300 import _lib as L


def test_probe_rejects_bad_arguments():
    lib = L.lib()
    import ctypes
    tf = ctypes.c_double()
    assert lib.fr_probe_fp32_peak(2, 5, ctypes.byref(tf), None, None) == L.FR_ERR_INVALID_ARG
    assert lib.fr_probe_fp32_peak(0, 0, ctypes.byref(tf), None, None) == L.FR_ERR_INVALID_ARG
    assert lib.fr_probe_fp32_peak(0, 101, ctypes.byref(tf), None, None) == L.FR_ERR_INVALID_ARG
    assert lib.fr_probe_fp32_peak(0, 5, None, None, None) == L.FR_ERR_INVALID_ARG


def _max_sm_mhz():
    smi = shutil.which("nvidia-smi")
    if not smi:
        return None
    try:
        out = subprocess.run([smi, "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(torch.cuda.current_device())],
                             capture_output=True, text=True, timeout=30).stdout
        return float(out.strip().splitlines()[0])
    except Exception:
        return None


@pytest.mark.gpu
def test_probe_fp32_peak_is_plausible():
    tf1, ms1 = L.fr_probe_fp32_peak(False, 5)
    tf2, ms2 = L.fr_probe_fp32_peak(True, 5)
    assert tf1 > 0 and ms1 > 0 and tf2 > 0 and ms2 > 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = _max_sm_mhz()
    if mhz:
        nominal = sms * 128 * 2 * mhz * 1e6 / 1e12
        assert 0.5 * nominal <= tf1 <= 1.02 * nominal, (tf1, nominal)
    assert tf2 >= 0.9 * tf1, (tf1, tf2)
