"""The C ABI library builds, loads without a GPU and exports every symbol include/lr.h declares."""
import os
import re
import subprocess

import pytest

import paper_1501_06663_gb300 as lr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lr_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib_path():
    return lr.build_library()


def test_header_declares_the_binding_names():
    assert _declared() == set(lr.EXPORTED)


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lr_[a-z_0-9]+)", out))
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_without_gpu(lib_path):
    lib = lr.load()
    for name in _declared():
        assert hasattr(lib, name)
    assert lr.status_str(lr.LR_ERR_CAPACITY) == "LR_ERR_CAPACITY"


def test_argument_errors_need_no_gpu(lib_path):
    import ctypes
    lib = lr.load()
    h = ctypes.c_void_p()
    assert lib.lr_create(None, 0) == lr.LR_ERR_ARG
    assert lib.lr_create(ctypes.byref(h), -1) == lr.LR_ERR_ARG
    null = ctypes.c_void_p(0)
    assert lib.lr_query_all(null, null, null, null, null, 5, null, null, null, null, 0, None) == lr.LR_ERR_ARG
    assert lib.lr_destroy(null) == lr.LR_ERR_ARG


def test_kernels_target_sm103a(lib_path):
    """The fat binary carries sm_103a code (listing the ELF names only)."""
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_server_entry_points_without_gpu(lib_path):
    """With no device the server refuses to start; NULL handles are argument errors."""
    import ctypes
    lib = lr.load()
    h = ctypes.c_void_p()
    cfg = lr.ServerConfig(device=0)
    st = lib.lr_server_start(ctypes.byref(cfg), ctypes.byref(h))
    if st == lr.LR_OK:                      # a GPU is present after all
        assert lib.lr_server_stop(h) == lr.LR_OK
    else:
        assert st == lr.LR_ERR_CUDA
    bad = lr.ServerConfig(device=0, hbm_fraction=2.0)
    assert lib.lr_server_start(ctypes.byref(bad), ctypes.byref(h)) == lr.LR_ERR_ARG
    null = ctypes.c_void_p(0)
    jid = ctypes.c_int64()
    assert lib.lr_server_submit(null, None, ctypes.byref(jid)) == lr.LR_ERR_ARG
    assert lib.lr_server_cancel(null, 1) == lr.LR_ERR_ARG
    assert lib.lr_server_stop(null) == lr.LR_ERR_ARG
    assert lib.lr_plan_launch(null, null) == lr.LR_ERR_ARG
