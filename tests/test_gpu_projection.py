"""Parity of the quark-line projection on the GPU (Sec. 3.3 eqs. projection, quark_prop_II_proj;
Sec. 6 inverse-iteration vectors) with the FP64 oracle, through the C ABI.

Tolerances: the GPU solves to relative residual 1e-12 (FP32 inner solves, FP64 defect
correction), the oracle to 1e-13.
  projection vectors: unit vectors whose R factor is fixed (upper triangular, positive
    diagonal), so they are unique; an error e in the solves moves them by about
    cond(D_L) * e per iteration, with cond(D_L) < 100 here and 3 iterations: 1e-8 absolute;
  factors: relative 1e-9 of the largest entry (cond * 1e-12 with margin);
  contraction alone (identical factors in): 1e-13 relative (FP64, summation order only);
  complete basis (N_m = 6 L^3): projected = unprojected case-II propagator to 1e-9 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_06424_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
SPLIT = dict(gamma=(0, 3), delta=(4, 4), gamma_star=(4, 7))   # Gammabar = 0..4, g1 = 3
OSPLIT = oracle.Split(gamma=(0, 3), gamma_star=(4, 7), delta=(4, 4))
X_SRC = (1, 2, 0, 3)


def _lq():
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    return lqcd


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _setup(csw, dims=DIMS, seed=5):
    lqcd = _lq()
    U = inputs.random_su3_field(dims, 0.4, seed)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.12, csw)
    return lqcd, lat, oracle.Operator(dims, U, 0.12, csw)


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_boundary_modes_match_oracle(csw):
    lqcd, lat, op = _setup(csw)
    n_m, dom, g1 = 20, (2, 5), 3
    v0 = inputs.gaussian_spinor(DIMS, 60, n_m)
    sl = inputs.slab_sites(DIMS, *dom)
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    phi, st = lat.boundary_modes(_cuda(v0[:, sl]), dom, g1, 0, 3, prm)
    assert st["status"] == 0, st
    phi = phi.cpu().numpy()
    ref = oracle.boundary_modes(op, v0, *dom, g1, 3)
    F = phi.reshape(n_m, -1)
    assert np.abs(F.conj() @ F.T - np.eye(n_m)).max() < 1e-12
    assert np.abs(phi - ref).max() < 1e-8


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_projected_factors_and_propagator_match_oracle(csw):
    lqcd, lat, op = _setup(csw, seed=6)
    n_m = 20
    phi = oracle.boundary_modes(op, inputs.gaussian_spinor(DIMS, 61, n_m), 2, 5, 3, 2)
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    xi, eta, st = lat.projected_factors(_cuda(phi), SPLIT["gamma"], SPLIT["gamma_star"], SPLIT["delta"], 0, prm)
    assert all(s["status"] == 0 for s in st.values()), st
    xr, er = oracle.projected_factors(op, OSPLIT, phi)
    gb = inputs.slab_sites(DIMS, 0, 4)
    gs = inputs.slab_sites(DIMS, 4, 7)
    xg, eg = xi.cpu().numpy(), eta.cpu().numpy()
    assert np.abs(xg - xr[:, gb]).max() <= 1e-9 * np.abs(xr).max()
    assert np.abs(eg - er[:, gs]).max() <= 1e-9 * np.abs(er).max()
    # the contraction kernel alone, on the oracle's factors
    xin = _cuda(xr[:, gb])
    ein = _cuda(er[:, gs])
    fact = lat.projected_propagator(xin, ein, SPLIT["gamma"], SPLIT["gamma_star"], X_SRC, SPLIT["delta"]).cpu().numpy()
    want = oracle.projected_propagator(op, OSPLIT, xr, er, X_SRC)
    assert np.abs(fact - want).max() <= 1e-13 * np.abs(want).max()


def test_complete_basis_gives_the_unprojected_propagator():
    """GPU end to end (modes, factors, contraction) with N_m = 6 L^3 = 48 on 8x2x2x2: the cut
    is exact, so case II equals the oracle's unprojected factorized propagator."""
    dims = (8, 2, 2, 2)
    lqcd, lat, op = _setup(1.0, dims=dims, seed=7)
    n_m = 48
    dom = (1, 6)
    v0 = inputs.gaussian_spinor(dims, 62, n_m)
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    phi, _ = lat.boundary_modes(_cuda(v0[:, inputs.slab_sites(dims, *dom)]), dom, 3, 0, 2, prm)
    xi, eta, _ = lat.projected_factors(phi, (0, 3), (4, 7), (4, 4), 0, prm)
    fact = lat.projected_propagator(xi, eta, (0, 3), (4, 7), X_SRC[:1] + (1, 0, 1), (4, 4)).cpu().numpy()
    ref = oracle.factorized_propagator(op, OSPLIT, inputs.point_sources(dims, X_SRC[:1] + (1, 0, 1)))
    m = op.slab(4, 7)
    assert np.abs(fact[:, m] - ref[:, m]).max() <= 1e-9 * np.abs(ref[:, m]).max()
    assert np.all(fact[:, ~m] == 0)


def test_projection_errors():
    lqcd = _lq()
    U = inputs.random_su3_field(DIMS, 0.4, 8)
    lat = lqcd.Lattice(DIMS, "open")
    lat.set_gauge(U, 0.12, 0.0)
    sl = inputs.slab_sites(DIMS, 2, 5)
    v = inputs.gaussian_spinor(DIMS, 63, 4)[:, sl]
    v[3] = v[1]                                   # linearly dependent start
    with pytest.raises(lqcd.LQCDError) as e:
        lat.boundary_modes(_cuda(v), (2, 5), 3, 0, 1)
    assert e.value.code == -9
    with pytest.raises(lqcd.LQCDError):           # g1 outside the slab
        lat.boundary_modes(_cuda(v[:3]), (2, 5), 6, 0, 1)
    too_many = np.zeros((6 * 64 + 1, 4 * 64, 4, 3), complex)
    with pytest.raises(lqcd.LQCDError):
        lat.boundary_modes(_cuda(too_many), (2, 5), 3, 0, 1)
    latp = lqcd.Lattice(DIMS, "periodic")
    latp.set_gauge(U, 0.12, 0.0)
    phi = _cuda(np.zeros((2, 64, 4, 3), complex))
    with pytest.raises(lqcd.LQCDError):           # open time boundary only
        latp.projected_factors(phi, (0, 3), (4, 7))
