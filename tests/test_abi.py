"""The C ABI library builds, loads and exports every function include/gid.h declares (CPU)."""
import ctypes
import os
import re

import pytest

from paper_1908_01961_b300 import build, gid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gid_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(gid.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 22
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert set(gid.EXPORTS) <= set(syms)


def test_weights_struct_matches_defaults():
    w = gid.default_weights([[1, 2], [-1, 0]], temporal=1)
    assert (w.lambda_data, w.lambda_clustering, w.lambda_rsparsity, w.p) == (5000, 200, 20, 1)
    assert (w.lambda_isparsity, w.lambda_smoothness, w.lambda_nonneg) == (3, 3, 1000)
    assert (w.lambda_IR, w.lambda_CR, w.lambda_rconsistency, w.lambda_monochrome) == (10, 100, 10, 10)
    assert w.eps == pytest.approx(0.002) and w.retinex_sharpness == 50
    assert w.n_spatial_pairs == 2 and list(w.spatial_offsets[:4]) == [1, 2, -1, 0] and w.temporal == 1
    assert w.nonneg_strict == 1 and w.refine_base_colors == 1 and w.rcluster_follows_b == 0
    assert ctypes.sizeof(gid.Weights) == 14 * 4 + 7 * 4 + 2 * 16 * 4


def test_create_without_device_fails_cleanly():
    """No GPU here: gid_create must report GID_ERR_CUDA, never fall back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    lib = gid.load()
    h = ctypes.c_void_p()
    rc = lib.gid_create(8, 8, 2, None, None, ctypes.byref(h))
    assert rc == -2 and not h.value
    assert b"device" in lib.gid_last_error(None).lower()


def test_invalid_sizes_rejected_before_any_device_call():
    lib = gid.load()
    h = ctypes.c_void_p()
    assert lib.gid_create(8, 8, 11, None, None, ctypes.byref(h)) == -1
    assert lib.gid_create(0, 8, 2, None, None, ctypes.byref(h)) == -1
    w = gid.default_weights([[4, 0]])                     # offset beyond the 3-pixel radius
    assert lib.gid_create(8, 8, 2, ctypes.byref(w), None, ctypes.byref(h)) == -1


def test_network_create_rejects_bad_arguments_and_missing_device():
    import torch
    lib = gid.load()
    h = ctypes.c_void_p()
    assert lib.gid_net_create(11, None, 0, None, ctypes.byref(h)) == -1
    bad = (ctypes.c_int * 4)(32, 48, 96, 128)
    assert lib.gid_net_create(3, bad, 0, None, ctypes.byref(h)) == -1
    assert lib.gid_net_num_params(None) == 0
    if not torch.cuda.is_available():
        assert lib.gid_net_create(3, None, 0, None, ctypes.byref(h)) == -2 and not h.value
