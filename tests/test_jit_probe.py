"""Run-time specialisation works on this machine without a GPU: NVRTC and
the kernel sources are found and a sample few-groups shape compiles."""
import ctypes.util
import glob
import os

import pytest


def _nvrtc_available():
    return bool(ctypes.util.find_library("nvrtc") or glob.glob("/usr/local/cuda/lib64/libnvrtc.so*"))


def test_sample_shape_compiles(tmp_path, monkeypatch):
    if not _nvrtc_available():
        pytest.skip("NVRTC not installed")
    import paper_2203_01877_gb300 as tqp
    try:
        tqp.lib()
    except OSError as e:  # libcudart missing on a machine without CUDA
        pytest.skip(f"cannot load libtqp.so here: {e}")
    monkeypatch.setenv("TQP_JIT_CACHE", str(tmp_path))  # a fresh cache: the compile runs
    before = tqp.tqp_jit_stats()
    tqp.tqp_jit_probe()
    after = tqp.tqp_jit_stats()
    assert after["compiled"] == before["compiled"] + 1
    assert len(os.listdir(tmp_path)) == 1
    tqp.tqp_jit_probe()  # now from the disk cache
    assert tqp.tqp_jit_stats()["from_disk"] == after["from_disk"] + 1
