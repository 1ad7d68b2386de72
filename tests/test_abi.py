"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/ddrw.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1211_1214_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ddrw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ddrw_[a-z_A-Z0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding_exports():
    assert sorted(binding.EXPORTS) == declared_symbols()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_loads(lib):
    L = binding.load()
    for name in binding.EXPORTS:
        assert getattr(L, name).argtypes is not None or name == "ddrw_destroy"


def test_create_rejects_bad_geometry_without_touching_the_gpu(lib):
    L = binding.load()
    h = ctypes.c_void_p()
    bad = [((4, 4, 4, 4), (3, 3, 3, 3)),   # l not in {2,4,6,8}
           ((4, 4, 4, 6), (2, 2, 2, 2)),   # 3 blocks in z: odd
           ((8, 8, 8, 8), (4, 4, 4, 2)),   # not hypercubic
           ((4, 4, 4, 4), (4, 4, 4, 4))]   # one block per direction
    for dims, blk in bad:
        st = L.ddrw_create(ctypes.byref(h), (ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*blk), 0, None)
        assert st == 1, (dims, blk)


@pytest.mark.parametrize("dims,block", [
    ((256, 256, 256, 16), 8),   # 2^28 sites: above the 2^27 limit of the kernels' 32-bit in-field offsets
    ((8, 8, 8, 8), 8),          # one block per direction (blocks must alternate in colour: >= 2, even)
    ((12, 12, 12, 12), 4),      # three blocks per direction (odd)
    ((6, 6, 6, 6), 3),          # block length 3 (2, 4, 6, 8 are built)
    ((8, 8, 8, 8), (4, 4, 2, 2)),  # non-hypercubic blocks
    ((8, 8, 0, 8), 2),          # empty lattice
])
def test_geometry_is_validated_before_any_device_call(lib, dims, block):
    """ddrw_create rejects a geometry the kernels do not support with DDRW_EINVAL before it touches
    the device (so this runs without a GPU)."""
    with pytest.raises(binding.DDRWError) as ei:
        binding.Context(dims, block)
    assert ei.value.status == 1
