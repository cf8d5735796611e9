"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative to the largest element of the reference):
  FP64 operator: 1e-13 (same arithmetic up to summation order);
  FP32 operator: 2e-6, FP16 operator (FP16 spinors with FP32 norm, FP16 links): 3e-3;
  FP64 solves / propagators: 1e-9 (solver tolerance 1e-12);
  mixed-precision solves: true FP64 residual <= 1e-10, checked with the oracle's D.
Lattices span several thread blocks with a ragged tail (V/2 = 576 sites for
8x6x6x4 with 128-thread blocks).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_06424_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lq():
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    return lqcd


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


BCS = {"open": oracle.BC_OPEN, "periodic": oracle.BC_PERIODIC, "antiperiodic": oracle.BC_ANTIPERIODIC}


@pytest.mark.parametrize("dims", [(8, 6, 6, 4), (4, 4, 4, 4)])
@pytest.mark.parametrize("bc", ["open", "periodic", "antiperiodic"])
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_dslash_fp64_matches_oracle(dims, bc, csw):
    lqcd = _lq()
    U = inputs.random_su3_field(dims, 0.4, 3)
    lat = lqcd.Lattice(dims, bc)
    lat.set_gauge(U, 0.13, csw)
    op = oracle.Operator(dims, U, 0.13, csw, BCS[bc])
    psi = inputs.gaussian_spinor(dims, 4)[0]
    T = dims[0]
    for dom in [None, (1, T - 2), (0, T // 2 - 1)]:
        for dag in (False, True):
            t0, t1 = dom if dom else (0, T - 1)
            sl = inputs.slab_sites(dims, t0, t1)
            ref = op.apply(op.masked(psi, t0, t1), t0, t1, dagger=dag)[sl]
            got = lat.dslash(_cuda(psi[sl]), 0, dom, dag, 64).cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (dom, dag)


@pytest.mark.parametrize("prec,tol", [(32, 2e-6), (16, 3e-3)])
@pytest.mark.parametrize("bc", ["open", "antiperiodic"])
def test_dslash_reduced_precision(prec, tol, bc):
    """FP32 / FP16 stencil on the whole lattice (wrapping time hops for the
    antiperiodic case) and on Dirichlet slabs touching either end, both D and
    D^dag: every dropped or sign-carrying hop of the stencil is exercised."""
    lqcd = _lq()
    dims = (8, 6, 6, 4)
    U = inputs.random_su3_field(dims, 0.4, 5)
    lat = lqcd.Lattice(dims, bc)
    lat.set_gauge(U, 0.13, 1.0)
    op = oracle.Operator(dims, U, 0.13, 1.0, BCS[bc])
    psi = inputs.gaussian_spinor(dims, 6)[0]
    T = dims[0]
    for dom in [None, (0, 2), (3, T - 1), (2, 5)]:
        for dag in (False, True):
            t0, t1 = dom if dom else (0, T - 1)
            sl = inputs.slab_sites(dims, t0, t1)
            ref = op.apply(op.masked(psi, t0, t1), t0, t1, dagger=dag)[sl]
            got = lat.dslash(_cuda(psi[sl]), 0, dom, dag, prec).cpu().numpy()
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (dom, dag)


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_solve_block_matches_oracle(prec):
    lqcd = _lq()
    dims = (8, 6, 6, 4)
    U = inputs.random_su3_field(dims, 0.4, 7)
    kappa, csw = 0.13, 1.0
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, csw)
    op = oracle.Operator(dims, U, kappa, csw)
    doms = [(0, 3), (2, 7), (0, 7)]
    srcs = inputs.gaussian_spinor(dims, 8, len(doms))
    packed = np.concatenate([srcs[k][inputs.slab_sites(dims, *d)] for k, d in enumerate(doms)])
    tol = 1e-12 if prec == 64 else 1e-10
    sol, stats = lat.solve_block(_cuda(packed), doms, [0] * len(doms), lqcd.SolverParams(tol=tol, precision=prec))
    sol = sol.cpu().numpy()
    off = 0
    for k, d in enumerate(doms):
        sl = inputs.slab_sites(dims, *d)
        n = sl.stop - sl.start
        got = np.zeros((op.V, 4, 3), complex)
        got[sl] = sol[off:off + n]
        off += n
        b = op.masked(srcs[k], *d)
        # true residual with the oracle's operator
        res = np.linalg.norm(b - op.apply(got, *d)) / np.linalg.norm(b)
        assert res <= 1.5 * tol, (prec, d, res, stats[k])
        assert stats[k]["true_residual"] <= tol
        if prec == 64:
            ref, _, _ = op.solve(b, *d, tol=1e-13)
            assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [64, 32])
def test_factorized_propagator_4x4_dense(prec):
    """Config 1: 4^4, Wilson kappa = 0.12, eps = 0.3, Gamma = {0,1}, Gamma* = {2,3}."""
    lqcd = _lq()
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.3, 1)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.12, 0.0)
    op = oracle.Operator(dims, U, 0.12, 0.0)
    x_src = (0, 0, 0, 0)
    tol = 1e-12 if prec == 64 else 1e-10
    fact, corr, st = lat.factorized_propagator((0, 1), (2, 3), x_src, params=lqcd.SolverParams(tol=tol, precision=prec))
    eta = inputs.point_sources(dims, x_src)
    f_ref = oracle.factorized_propagator(op, oracle.Split((0, 1), (2, 3)), eta)
    full = oracle.full_propagator(op, eta)
    scale = np.abs(full).max()
    bound = 1e-9 if prec == 64 else 2e-9
    assert np.abs(fact.cpu().numpy() - f_ref).max() <= bound * scale
    assert np.abs(corr.cpu().numpy() - (full - f_ref)).max() <= bound * scale


@pytest.mark.parametrize("bc", ["open", "periodic"])
def test_factorized_propagator_with_overlap_clover(bc):
    lqcd = _lq()
    dims = (8, 4, 4, 6)
    U = inputs.random_su3_field(dims, 0.4, 9)
    kappa, csw = 0.13, 1.0
    lat = lqcd.Lattice(dims, bc)
    lat.set_gauge(U, kappa, csw)
    op = oracle.Operator(dims, U, kappa, csw, BCS[bc])
    x_src = (1, 2, 0, 3)
    split = oracle.Split((0, 3), (4, 7), delta=(4, 5))
    fact, corr, st = lat.factorized_propagator((0, 3), (4, 7), x_src, delta=(4, 5),
                                               params=lqcd.SolverParams(tol=1e-12, precision=64))
    eta = inputs.point_sources(dims, x_src)
    f_ref = oracle.factorized_propagator(op, split, eta)
    full = oracle.full_propagator(op, eta)
    scale = np.abs(full).max()
    assert np.abs(fact.cpu().numpy() - f_ref).max() <= 1e-9 * scale
    assert np.abs(corr.cpu().numpy() - (full - f_ref)).max() <= 1e-9 * scale
    for k in ("gamma", "gamma_bar", "gamma_star", "full"):
        assert st[k]["status"] == 0 and st[k]["true_residual"] <= 1e-12


@pytest.mark.parametrize("prec", [64, 32])
def test_factorized_propagators_batched_over_fields(prec):
    """Two gauge fields (the level-0 field and an inner-level field with Gamma's and
    Gamma*'s own links redrawn) in one batched call, fields passed in reverse order:
    each field's fact and corr match its single-field call and the oracle's
    factorization and full propagator (eqs. quark_prop_I/II, observable_factorization)."""
    lqcd = _lq()
    dims = (8, 4, 4, 6)
    kappa, csw = 0.13, 1.0
    U0 = inputs.random_su3_field(dims, 0.4, 91)
    U1 = inputs.inner_level_fields(U0, dims, [(0, 3), (6, 7)], 2, 0.4, 92, frozen=(4, 5))[1]
    Us = np.stack([U0, U1])
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(Us, kappa, csw)
    x_src = (1, 2, 0, 3)
    tol = 1e-12 if prec == 64 else 1e-10
    params = lqcd.SolverParams(tol=tol, precision=prec)
    fact, corr, st = lat.factorized_propagators((0, 3), (4, 7), x_src, [1, 0], delta=(4, 5), params=params)
    eta = inputs.point_sources(dims, x_src)
    split = oracle.Split((0, 3), (4, 7), delta=(4, 5))
    bound = 1e-9 if prec == 64 else 2e-9
    for j, fid in enumerate([1, 0]):
        for k in ("gamma", "gamma_bar", "gamma_star", "full"):
            assert st[j][k]["status"] == 0 and st[j][k]["true_residual"] <= tol, (j, k, st[j][k])
        f1, c1, _ = lat.factorized_propagator((0, 3), (4, 7), x_src, fid, delta=(4, 5), params=params)
        op = oracle.Operator(dims, Us[fid], kappa, csw)
        f_ref = oracle.factorized_propagator(op, split, eta)
        full = oracle.full_propagator(op, eta)
        scale = np.abs(full).max()
        assert np.abs(fact[j].cpu().numpy() - f_ref).max() <= bound * scale, j
        assert np.abs(corr[j].cpu().numpy() - (full - f_ref)).max() <= bound * scale, j
        assert (fact[j] - f1).abs().max().item() <= bound * scale
        assert (corr[j] - c1).abs().max().item() <= bound * scale
    lat.close()


@pytest.mark.parametrize("csw,dom", [(0.0, (0, 3)), (1.0, (1, 2)), (1.0, (0, 3))])
def test_link_force_matches_oracle(csw, dom):
    lqcd = _lq()
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.4, 51)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.13, csw)
    op = oracle.Operator(dims, U, 0.13, csw)
    phi = inputs.gaussian_spinor(dims, 52)[0]
    F_ref, S_ref, _, _ = oracle.link_force(op, phi, *dom)
    sl = inputs.slab_sites(dims, *dom)
    F, S, st = lat.link_force(_cuda(phi[sl]), dom, 0, lqcd.SolverParams(tol=1e-13, precision=64))
    F = F.cpu().numpy()
    assert abs(S - S_ref) <= 1e-10 * abs(S_ref)
    assert np.abs(F - F_ref).max() <= 1e-9 * np.abs(F_ref).max()


@pytest.mark.parametrize("store", [None, True, False])
def test_autograd_function_returns_force(store):
    """Both ways of the autograd Function (force kept from forward, or X and Y
    recomputed in backward) give the link force of the C ABI."""
    lqcd = _lq()
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.4, 61)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.13, 1.0)
    phi = _cuda(inputs.gaussian_spinor(dims, 62)[0][inputs.slab_sites(dims, 0, 2)])
    omega = torch.zeros((lat.V, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    params = lqcd.SolverParams(tol=1e-13)
    S = lqcd.DomainPseudofermionAction.apply(omega, lat, (0, 2), 0, phi, params, store)
    S.backward()
    F, S2, _ = lat.link_force(phi, (0, 2), 0, params)
    assert abs(S.item() - S2) <= 1e-12 * abs(S2)
    assert torch.allclose(omega.grad, F, rtol=0, atol=1e-12 * F.abs().max().item())


def test_error_paths():
    lqcd = _lq()
    dims = (4, 4, 4, 4)
    lat = lqcd.Lattice(dims, "open")
    U = inputs.random_su3_field(dims, 0.4, 71)
    bad = U.copy()
    bad[5, 2] *= 1.001
    with pytest.raises(lqcd.LQCDError) as e:
        lat.set_gauge(bad, 0.13, 1.0)
    assert e.value.code == -3
    lat.set_gauge(U, 0.13, 1.0)
    src = _cuda(inputs.gaussian_spinor(dims, 72)[0])
    with pytest.raises(lqcd.LQCDError) as e:
        lat.solve_block(src, [(0, 4)], [0])
    assert e.value.code == -1
    with pytest.raises(lqcd.LQCDError) as e:
        lat.solve_block(src, [(0, 3)], [3])
    assert e.value.code == -8
    with pytest.raises(lqcd.LQCDError) as e:
        lat.solve_full(src, [0], lqcd.SolverParams(tol=1e-10, max_iter=2))
    assert e.value.code == -4
    with pytest.raises(lqcd.LQCDError) as e:
        lat.factorized_propagator((0, 1), (2, 3), (2, 0, 0, 0))
    assert e.value.code == -1
    # zero source: zero solution, no error
    sol, st = lat.solve_full(torch.zeros_like(src), [0])
    assert sol.abs().max().item() == 0.0
