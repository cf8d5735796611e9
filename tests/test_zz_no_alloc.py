"""lqcd_dslash_noalloc, called through the C ABI, agrees with lqcd_dslash.

The allocation-free entry point serves callers that cannot allocate device
memory while they run (an application whose allocator owns the GPU's memory,
or a latency-critical path); its scratch is a fixed device array inside the
library.  Two calls in a row on different inputs (the second must not see the
first's leftovers), both parities of a slab and the whole lattice, the whole
lattice with periodic and antiperiodic time boundaries (the hop across
x0 = T-1 -> 0 and its sign), plus the size limit.  Tolerance: the FP64
operator tolerance of the parity tests (1e-13 relative to the largest
element).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1612_06424_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    L = lqcd.lib()
    L.lqcd_dslash_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(lqcd.Slab), ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return lqcd, L


def test_noalloc_dslash_matches_dslash_twice():
    lqcd, L = _lib()
    dims = (8, 6, 6, 4)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(inputs.random_su3_field(dims, 0.4, 81), 0.13, 1.0)
    stream = torch.cuda.current_stream()
    for call, (dom, dag, seed) in enumerate([((1, 6), 0, 82), (None, 1, 83), ((0, 3), 0, 84)]):
        t0, t1 = dom if dom else (0, dims[0] - 1)
        psi = torch.from_numpy(inputs.gaussian_spinor(dims, seed)[0][inputs.slab_sites(dims, t0, t1)]).cuda()
        ref = lat.dslash(psi, 0, dom, bool(dag), 64)
        out = torch.full_like(psi, float("nan"))
        sl = ctypes.byref(lqcd.Slab(*dom)) if dom else None
        rc = L.lqcd_dslash_noalloc(lat._h, 0, sl, dag, ctypes.c_void_p(psi.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.lqcd_last_error()
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 1e-13 * scale, call
    lat.close()


@pytest.mark.parametrize("bc", ["periodic", "antiperiodic"])
def test_noalloc_dslash_wrapped_time_boundary(bc):
    lqcd, L = _lib()
    dims = (8, 6, 6, 4)
    lat = lqcd.Lattice(dims, bc)
    lat.set_gauge(inputs.random_su3_field(dims, 0.4, 86), 0.13, 1.0)
    stream = torch.cuda.current_stream()
    for dag, seed in ((0, 87), (1, 88)):
        psi = torch.from_numpy(inputs.gaussian_spinor(dims, seed)[0]).cuda()
        ref = lat.dslash(psi, 0, None, bool(dag), 64)
        out = torch.full_like(psi, float("nan"))
        rc = L.lqcd_dslash_noalloc(lat._h, 0, None, dag, ctypes.c_void_p(psi.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.lqcd_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 1e-13 * ref.abs().max().item(), (bc, dag)
    lat.close()


def test_noalloc_dslash_rejects_oversize_slab():
    lqcd, L = _lib()
    dims = (16, 16, 16, 16)  # whole lattice: 65536 sites > limit
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(inputs.unit_field(dims), 0.13, 0.0)
    psi = torch.zeros((lat.V, 4, 3), dtype=torch.complex128, device="cuda")
    rc = L.lqcd_dslash_noalloc(lat._h, 0, None, 0, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(psi.data_ptr()),
                               None)
    assert rc == -1
    assert b"scratch" in L.lqcd_last_error()
    # a slab within the limit works on the same lattice
    sl = lqcd.Slab(0, 9)
    n = lat.slab_len(0, 9)
    x = torch.from_numpy(inputs.gaussian_spinor(dims, 85)[0][:n]).cuda()
    out = torch.empty_like(x)
    rc = L.lqcd_dslash_noalloc(lat._h, 0, ctypes.byref(sl), 0, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0, L.lqcd_last_error()
    torch.cuda.synchronize()
    ref = lat.dslash(x, 0, (0, 9), False, 64)
    assert (out - ref).abs().max().item() <= 1e-13 * ref.abs().max().item()
    lat.close()
