"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/*.h (no compute calls)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mego_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2109_13504_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for required in ("mego_resample", "mego_resample_gather", "mego_compute_B",
                     "mego_likelihood_B", "mego_resample_host", "mego_sync_status",
                     "mego_workspace_bytes", "mego_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.mego_abi_version.restype = ctypes.c_int
    assert lib.mego_abi_version() == 4
    lib.mego_status_string.restype = ctypes.c_char_p
    lib.mego_status_string.argtypes = [ctypes.c_int]
    assert lib.mego_status_string(5).decode().startswith("invalid weights")
    lib.mego_workspace_bytes.restype = ctypes.c_size_t
    lib.mego_workspace_bytes.argtypes = [ctypes.c_int32]
    assert lib.mego_workspace_bytes(1 << 20) >= 16 * 1024


def test_argument_errors_need_no_gpu(lib):
    # Validation happens on the host before any CUDA call.
    f = lib.mego_resample
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                  ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    fake = ctypes.c_void_p(0x10000)
    out = ctypes.c_void_p(0x20000)
    assert f(None, 10, 4, 1, 0, 0, out, None) == 1            # null weights
    assert f(fake, 0, 4, 1, 0, 0, out, None) == 1             # n = 0
    assert f(fake, 10, -1, 1, 0, 0, out, None) == 1           # B < 0
    assert f(fake, 10, (1 << 24) + 1, 1, 0, 0, out, None) == 1
    assert f(fake, 10, 4, 1, 0, 7, out, None) == 1            # unknown variant
    assert f(fake, 10, 4, 1, 0, 0, ctypes.c_void_p(0x10010), None) == 1  # overlap


def test_binding_structs_match_the_header(lib):
    # The ctypes mirrors in the binding must have the C structs' sizes
    # (a field added on one side only shifts every later field).
    mego = pytest.importorskip("paper_2109_13504_gb300")
    lib.mego_struct_size.restype = ctypes.c_size_t
    lib.mego_struct_size.argtypes = [ctypes.c_int32]
    mirrors = [mego.LaunchCfg, mego.Filter, mego.BatchHandle, mego.Request, mego.Completion,
               mego.ServerCfg, mego.ServerStats]
    for which, cls in enumerate(mirrors):
        assert lib.mego_struct_size(which) == ctypes.sizeof(cls), cls.__name__
    assert lib.mego_struct_size(99) == 0


def test_batch_plan_size_is_host_only(lib):
    # mego_batch_plan_bytes validates the filters and sizes the plan on the
    # host: header, per-filter descriptors and prefix entries, the bound's
    # per-filter outputs and one 16-byte partial per 4096-weight chunk.
    mego = pytest.importorskip("paper_2109_13504_gb300")
    lib.mego_batch_plan_bytes.restype = ctypes.c_size_t
    lib.mego_batch_plan_bytes.argtypes = [ctypes.POINTER(mego.Filter), ctypes.c_int32]

    def plan(sizes):
        arr = (mego.Filter * len(sizes))()
        for k, n in enumerate(sizes):
            arr[k].w = 0x1000
            arr[k].anc = 0x2000
            arr[k].n = n
            arr[k].B = -1
        return lib.mego_batch_plan_bytes(arr, len(sizes))

    one = plan([4096])
    assert one > 0 and one % 256 == 0
    assert plan([4096 * 100]) >= one + 99 * 16      # one partial per 4096-weight chunk
    assert plan([100] * 64) > plan([100] * 8)       # descriptors grow with the count
    assert plan([0]) == 0 and plan([(1 << 30) + 1]) == 0   # invalid sizes
    assert lib.mego_batch_plan_bytes(None, 1) == 0
