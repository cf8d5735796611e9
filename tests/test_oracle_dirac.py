"""Pins of the oracle's Dirac operator against what the paper and the mathematics fix.

- gamma algebra: Clifford relations, gamma_5 = g0 g1 g2 g3 = diag(1,1,-1,-1);
- free field (U = 1): D acts on plane waves as
  D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu, m0 = 1/(2 kappa) - 4
  (normalisation 2 kappa D = 1 - kappa D_hop, Sec. 5), and the propagator
  equals the closed form V^{-1} sum_p e^{ipx} (M - i gamma.sin p)/(M^2 + sin^2 p);
- gamma_5-hermiticity gamma_5 D gamma_5 = D^dag (open BC, clover, slabs);
- gauge covariance D[U^g] = G D[U] G^dag;
- Neumann (hopping) series D^{-1} = 2 kappa sum_n (kappa D_hop)^n at small kappa.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs


def test_gamma_algebra():
    g = [oracle.gamma(mu) for mu in range(5)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * np.eye(4), atol=1e-15)
        assert np.allclose(g[4] @ g[a] + g[a] @ g[4], 0)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))


def _momenta(dims, bc):
    axes = []
    for mu, n in enumerate(dims):
        k = np.arange(n)
        if mu == 0 and bc == oracle.BC_ANTIPERIODIC:
            axes.append((2 * k + 1) * np.pi / n)
        else:
            axes.append(2 * np.pi * k / n)
    return axes


def _coords(dims):
    T, L1, L2, L3 = dims
    return np.stack(np.meshgrid(np.arange(T), np.arange(L1), np.arange(L2), np.arange(L3),
                                indexing="ij"), -1).reshape(-1, 4)


@pytest.mark.parametrize("bc", [oracle.BC_PERIODIC, oracle.BC_ANTIPERIODIC])
def test_free_field_plane_waves(bc):
    dims = (8, 4, 4, 4)
    kappa = 0.12
    m0 = 1 / (2 * kappa) - 4
    op = oracle.Operator(dims, inputs.unit_field(dims), kappa, 0.0, bc)
    g = [oracle.gamma(mu) for mu in range(4)]
    x = _coords(dims)
    rng = np.random.default_rng(5)
    pax = _momenta(dims, bc)
    for trial in range(6):
        p = np.array([pax[mu][rng.integers(dims[mu])] for mu in range(4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (x @ p))
        psi = phase[:, None, None] * u[None]
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (Dp @ u)[None]
        assert np.abs(op.apply(psi) - expect).max() < 1e-13


@pytest.mark.parametrize("dims,bc", [((4, 4, 4, 4), oracle.BC_PERIODIC),
                                     ((8, 4, 4, 4), oracle.BC_ANTIPERIODIC)])
def test_free_field_propagator_closed_form(dims, bc):
    kappa = 0.12
    m0 = 1 / (2 * kappa) - 4
    V = int(np.prod(dims))
    op = oracle.Operator(dims, inputs.unit_field(dims), kappa, 0.0, bc)
    g = [oracle.gamma(mu) for mu in range(4)]
    pax = _momenta(dims, bc)
    P = np.stack(np.meshgrid(*pax, indexing="ij"), -1).reshape(-1, 4)
    x = _coords(dims)
    M = m0 + np.sum(1 - np.cos(P), axis=1)
    s = np.sin(P)
    den = M ** 2 + np.sum(s ** 2, axis=1)
    # S(p) = (M - i gamma.s) / (M^2 + s^2), per momentum a 4x4 spin matrix
    Sp = (M[:, None, None] * np.eye(4)[None] - 1j * np.einsum("pm,mab->pab", s, np.array(g))) / den[:, None, None]
    Sx = np.einsum("xp,pab->xab", np.exp(1j * x @ P.T), Sp) / V       # S(x, 0)
    eta = inputs.point_sources(dims, (0, 0, 0, 0))
    for col in (0, 4, 11):
        sol, _, res = op.solve(eta[col], tol=1e-14)
        s0, c0 = divmod(col, 3)
        expect = np.zeros((V, 4, 3), dtype=np.complex128)
        expect[:, :, c0] = Sx[:, :, s0]
        assert res < 1e-13
        assert np.abs(sol - expect).max() < 1e-13


@pytest.mark.parametrize("csw,slab", [(0.0, (0, 3)), (1.0, (0, 3)), (1.0, (1, 2))])
def test_gamma5_hermiticity(csw, slab):
    dims = (4, 4, 4, 4)
    op = oracle.Operator(dims, inputs.random_su3_field(dims, 0.4, 11), 0.13, csw)
    g5 = oracle.gamma(4)
    v, w = inputs.gaussian_spinor(dims, 12, 2)
    g5w = np.einsum("st,xtc->xsc", g5, w)
    lhs = np.einsum("st,xtc->xsc", g5, op.apply(g5w, *slab))
    rhs = op.apply(w, *slab, dagger=True)
    assert np.abs(lhs - rhs).max() < 1e-13
    # the adjoint is an adjoint: <v, D w> = <D^dag v, w> on the slab
    vm, wm = op.masked(v, *slab), op.masked(w, *slab)
    a = np.vdot(vm, op.apply(wm, *slab))
    b = np.vdot(op.apply(vm, *slab, dagger=True), wm)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("bc", [oracle.BC_OPEN, oracle.BC_PERIODIC])
def test_gauge_covariance(bc):
    dims = (4, 4, 4, 6)
    U = inputs.random_su3_field(dims, 0.4, 21)
    g = inputs.random_gauge_transform(dims, 22)
    T, L1, L2, L3 = dims
    x = _coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % dims[mu]
        yi = ((y[:, 0] * L1 + y[:, 1]) * L2 + y[:, 2]) * L3 + y[:, 3]
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[yi], -1, -2))
    op = oracle.Operator(dims, U, 0.13, 1.0, bc)
    opg = oracle.Operator(dims, Ug, 0.13, 1.0, bc)
    psi = inputs.gaussian_spinor(dims, 23)[0]
    Gpsi = np.einsum("xab,xsb->xsa", g, psi)
    for slab in [(0, T - 1), (1, 2)]:
        lhs = opg.apply(Gpsi, *slab)
        rhs = np.einsum("xab,xsb->xsa", g, op.apply(psi, *slab))
        assert np.abs(lhs - rhs).max() < 1e-13


def test_neumann_series_small_kappa():
    dims = (4, 4, 4, 4)
    kappa = 0.05
    op = oracle.Operator(dims, inputs.random_su3_field(dims, 0.4, 31), kappa, 0.0)
    b = inputs.gaussian_spinor(dims, 32)[0]
    # D_hop psi = (psi - 2 kappa D psi) / kappa ;  D^{-1} = 2 kappa sum_n (kappa D_hop)^n
    term = b.copy()
    acc = b.copy()
    for _ in range(60):
        term = term - 2 * kappa * op.apply(term)          # (kappa D_hop) term
        acc = acc + term
    series = 2 * kappa * acc
    sol, _, _ = op.solve(b, tol=1e-14)
    assert np.abs(sol - series).max() < 1e-13 * np.abs(sol).max()


@pytest.mark.parametrize("csw,slab,bc", [(1.0, (0, 7), oracle.BC_OPEN), (1.0, (2, 5), oracle.BC_OPEN),
                                         (0.0, (0, 7), oracle.BC_ANTIPERIODIC)])
def test_dirac_at_sites_matches_full_operator(csw, slab, bc):
    dims = (8, 4, 4, 6)
    U = inputs.random_su3_field(dims, 0.4, 91)
    op = oracle.Operator(dims, U, 0.13, csw, bc)
    psi = op.masked(inputs.gaussian_spinor(dims, 92)[0], *slab)
    full = op.apply(psi, *slab)
    rng = np.random.default_rng(93)
    sites = rng.choice(op.V, 40, replace=False)
    got = oracle.dirac_at_sites(dims, U, 0.13, csw, bc, slab, sites, psi)
    assert np.abs(got - full[sites]).max() < 1e-14 * np.abs(full).max()
