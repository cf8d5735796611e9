"""Every stencil variant the autotuner can pick, checked against the FP64 oracle.

The variant is forced per process through LQCD_HOP_VARIANT (read once by the
library), so each case runs in a child process:
  1: one thread per site, 128 sites of one system per block, default launch
     configuration (FP32: 4 blocks per SM, hop pipeline depth 2);
  2: two threads per site (FP32 only; FP16 falls back to 1);
  3, 4: one thread per site in the alternative launch configurations of the
     forward operator (FP32: 3 blocks / depth 3 and 5 blocks / depth 1; FP16:
     4 / 3 and 6 / 1); dagger launches keep the default.
Each child applies the FP32 / FP16 operator on the whole lattice and on
Dirichlet slabs (D and D^dag; tolerances of tests/test_gpu_parity.py) and
solves a batch of five systems on mixed slabs in FP32, FP16 and FP64 to true
residual 1e-10, checked with the oracle's operator.  8x6x6x4: 576 sites per
parity, several blocks and a ragged tail for every variant.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_1612_06424_gb300 import build, inputs
build.build()
from paper_1612_06424_gb300 import lqcd

dims = (8, 6, 6, 4)
U = inputs.random_su3_field(dims, 0.4, 5)
lat = lqcd.Lattice(dims, "open")
lat.set_gauge(U, 0.13, 1.0)
op = oracle.Operator(dims, U, 0.13, 1.0)
psi = inputs.gaussian_spinor(dims, 6)[0]
for prec, tol in ((32, 2e-6), (16, 3e-3)):
    for dom in (None, (0, 2), (3, 7), (2, 5)):
        for dag in (False, True):
            t0, t1 = dom if dom else (0, 7)
            sl = inputs.slab_sites(dims, t0, t1)
            ref = op.apply(op.masked(psi, t0, t1), t0, t1, dagger=dag)[sl]
            got = lat.dslash(torch.from_numpy(np.ascontiguousarray(psi[sl])).cuda(), 0, dom, dag, prec).cpu().numpy()
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= tol, (prec, dom, dag, err)
doms = [(0, 3), (2, 7), (0, 7), (4, 7), (1, 5)]
srcs = inputs.gaussian_spinor(dims, 8, len(doms))
packed = np.concatenate([srcs[k][inputs.slab_sites(dims, *d)] for k, d in enumerate(doms)])
for prec in (32, 16, 64):
    sol, stats = lat.solve_block(torch.from_numpy(packed).cuda(), doms, [0] * len(doms),
                                 lqcd.SolverParams(tol=1e-10, precision=prec))
    sol = sol.cpu().numpy()
    off = 0
    for k, d in enumerate(doms):
        sl = inputs.slab_sites(dims, *d)
        n = sl.stop - sl.start
        got = np.zeros((op.V, 4, 3), complex)
        got[sl] = sol[off:off + n]
        off += n
        b = op.masked(srcs[k], *d)
        res = np.linalg.norm(b - op.apply(got, *d)) / np.linalg.norm(b)
        assert res <= 1.5e-10 and stats[k]["status"] == 0, (prec, d, res, stats[k])
print("variant ok")
"""


@pytest.mark.parametrize("variant", ["1", "2", "3", "4"])
def test_stencil_variant_parity(variant):
    env = dict(os.environ, LQCD_HOP_VARIANT=variant)
    env.pop("LQCD_HOP_SPLIT", None)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "variant ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_cgnr_fallback_parity():
    """The Krylov fallback (CG on the normal equations, which the solver switches a system to
    once BiCGStab has stalled for six defect-correction cycles), forced for every system with
    LQCD_KRYLOV=cgnr: FP32, FP16 and FP64 solves of five systems on mixed slabs reach the true
    residual 1e-10, checked with the oracle's operator (same child as the stencil variants)."""
    env = dict(os.environ, LQCD_KRYLOV="cgnr")
    env.pop("LQCD_HOP_SPLIT", None)
    env.pop("LQCD_HOP_VARIANT", None)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "variant ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


TUNE_CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_1612_06424_gb300 import build, inputs
build.build()
from paper_1612_06424_gb300 import lqcd

dims = (8, 6, 6, 4)
lat = lqcd.Lattice(dims, "open")
lat.set_gauge(inputs.random_su3_field(dims, 0.4, 5), 0.13, 1.0)
doms = [(0, 3), (2, 7), (0, 7)]
srcs = inputs.gaussian_spinor(dims, 8, len(doms))
packed = np.concatenate([srcs[k][inputs.slab_sites(dims, *d)] for k, d in enumerate(doms)])
sol, st = lat.solve_block(torch.from_numpy(packed).cuda(), doms, [0] * 3, lqcd.SolverParams(tol=1e-10, precision=32))
assert all(x["status"] == 0 for x in st)
print("tune ok")
"""


def test_tuner_decisions_cached(tmp_path):
    """The autotuner times every candidate on the solver's own batch shape, writes its decision to
    LQCD_TUNE_CACHE ("P systems sites variant"), and a later process takes the decision from the
    file instead of timing again (the decision it uses is the one written there)."""
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache), LQCD_VERBOSE="1")
    env.pop("LQCD_HOP_SPLIT", None)
    env.pop("LQCD_HOP_VARIANT", None)
    code = TUNE_CHILD.replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "tune ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    lines = [l.split() for l in cache.read_text().splitlines() if l.strip()]
    mine = [l for l in lines if l[0] == "32" and l[1] == "3"]
    assert mine and all(int(l[3]) in (1, 2, 3, 4) for l in mine), lines
    n_sites = mine[0][2]
    # plant a different decision for that shape: the next process must use it
    planted = 4 if int(mine[0][3]) != 4 else 3
    cache.write_text(f"32 3 {n_sites} {planted}\n")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "tune ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    assert f"stencil variant {planted} for P=32 nsys=3 max_n={n_sites}" in r.stderr, r.stderr[-3000:]
    assert cache.read_text().strip() == f"32 3 {n_sites} {planted}"  # read, not re-timed


TBLK_CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_1612_06424_gb300 import build, inputs
build.build()
from paper_1612_06424_gb300 import lqcd

dims = (12, 8, 4, 4)
for bc in ("open", "antiperiodic"):
    U = inputs.random_su3_field(dims, 0.4, 15)
    lat = lqcd.Lattice(dims, bc)
    lat.set_gauge(U, 0.13, 1.0)
    op = oracle.Operator(dims, U, 0.13, 1.0, oracle.BC_OPEN if bc == "open" else oracle.BC_ANTIPERIODIC)
    psi = inputs.gaussian_spinor(dims, 16)[0]
    for prec, tol in ((32, 2e-6), (16, 3e-3)):
        for dom in (None, (0, 3), (4, 11), (8, 11)):
            for dag in (False, True):
                t0, t1 = dom if dom else (0, 11)
                sl = inputs.slab_sites(dims, t0, t1)
                ref = op.apply(op.masked(psi, t0, t1), t0, t1, dagger=dag)[sl] if dom else op.apply(psi, dagger=dag)
                got = lat.dslash(torch.from_numpy(np.ascontiguousarray(psi[sl])).cuda(), 0, dom, dag, prec).cpu().numpy()
                err = np.abs(got - ref).max() / np.abs(ref).max()
                assert err <= tol, (bc, prec, dom, dag, err)
    doms = [(0, 3), (4, 11), (0, 11), (8, 11)]
    srcs = inputs.gaussian_spinor(dims, 18, len(doms))
    packed = np.concatenate([srcs[k][inputs.slab_sites(dims, *d)] for k, d in enumerate(doms)])
    for prec in (32, 16, 64):
        sol, stats = lat.solve_block(torch.from_numpy(packed).cuda(), doms, [0] * len(doms),
                                     lqcd.SolverParams(tol=1e-10, precision=prec))
        sol = sol.cpu().numpy()
        off = 0
        for k, d in enumerate(doms):
            sl = inputs.slab_sites(dims, *d)
            n = sl.stop - sl.start
            got = np.zeros((op.V, 4, 3), complex)
            got[sl] = sol[off:off + n]
            off += n
            if d == (0, 11):
                b = srcs[k]
                res = np.linalg.norm(b - op.apply(got)) / np.linalg.norm(b)
            else:
                b = op.masked(srcs[k], *d)
                res = np.linalg.norm(b - op.apply(got, *d)) / np.linalg.norm(b)
            assert res <= 1.5e-10 and stats[k]["status"] == 0, (bc, prec, d, res, stats[k])
    lat.close()
print("tblk ok")
"""


@pytest.mark.parametrize("variant,tblk", [("1", "1"), ("3", "1"), ("4", "1"), ("1", "0")])
def test_time_blocked_sites_parity(variant, tblk):
    """LQCD_HOP_TBLK=1 (the default where allowed): each 128-thread block of the one-thread
    stencils covers 32 sites of four consecutive time slices; LQCD_HOP_TBLK=0: 128 consecutive
    sites.  12x8x4x4 (64 sites per slice and parity: two 32-site chunks), slabs of 4, 8 and 12
    slices, open and antiperiodic (wrapping) time boundary; operator and solves against the
    oracle as above."""
    env = dict(os.environ, LQCD_HOP_VARIANT=variant, LQCD_HOP_TBLK=tblk)
    env.pop("LQCD_HOP_SPLIT", None)
    r = subprocess.run([sys.executable, "-c", TBLK_CHILD.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "tblk ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
