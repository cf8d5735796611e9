"""Argument checks of the C ABI that run on the host before any device work (no GPU needed): bad
lattice extents, time boundary, a lattice too large for 32-bit site indexing, null lattices and
empty or out-of-range sizes all return LQCD_EBADARG with a message in lqcd_last_error, and
nothing is allocated."""
import ctypes

import pytest

from paper_1612_06424_gb300 import build

EBADARG = -1


@pytest.fixture(scope="module")
def lib():
    L = ctypes.CDLL(build.build())
    L.lqcd_last_error.restype = ctypes.c_char_p
    return L


def _dims(*d):
    return (ctypes.c_int * 4)(*d)


@pytest.mark.parametrize("dims,bc,why", [
    ((8, 4, 4, 3), 0, "even"),        # odd extent
    ((8, 0, 4, 4), 0, "even"),        # empty extent
    ((8, 4, 4, 4), 3, "boundary"),    # no such time boundary
    ((256, 256, 256, 256), 0, "too large"),
])
def test_create_lattice_rejects(lib, dims, bc, why):
    out = ctypes.c_void_p(None)
    assert lib.lqcd_create_lattice(_dims(*dims), bc, ctypes.byref(out)) == EBADARG
    assert out.value is None
    assert why in lib.lqcd_last_error().decode()


def test_null_lattice_and_empty_sizes(lib):
    vp = ctypes.c_void_p
    assert lib.lqcd_solve_block(vp(None), 1, vp(None), vp(None), vp(None), vp(None), vp(None), vp(None),
                                vp(None)) == EBADARG
    assert "null lattice" in lib.lqcd_last_error().decode()
    assert lib.lqcd_solve_full(vp(None), 1, vp(None), vp(None), vp(None), vp(None), vp(None), vp(None)) == EBADARG
    assert lib.lqcd_nucleon_contract(0, 1, vp(1), 1, vp(1), vp(1), vp(None)) == EBADARG
    assert lib.lqcd_nucleon_contract(1025, 1, vp(1), 1, vp(1), vp(1), vp(None)) == EBADARG
    assert lib.lqcd_level_mean(ctypes.c_longlong(0), 1, vp(1), vp(1), vp(None)) == EBADARG
    assert lib.lqcd_level_mean(ctypes.c_longlong(8), 0, vp(1), vp(1), vp(None)) == EBADARG
    assert "level_mean" in lib.lqcd_last_error().decode()
