"""Pins of the oracle's link force F^a_mu(x) = dS/domega for
U_mu(x) -> exp(i omega T_a) U_mu(x), S = phi^dag (D_L^dag D_L)^{-1} phi.

- central finite differences with step h = 1e-5, the difference S(+h) - S(-h)
  taken without cancellation as X+^dag (M- - M+) X-  (M = D_L^dag D_L,
  X+- = M+-^{-1} phi): S+ - S- = phi^dag M+^{-1} (M- - M+) M-^{-1} phi;
- gauge covariance: sum_a F^a T_a transforms as g(x) (.) g(x)^dag.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs

DIMS = (4, 4, 4, 4)


def _expm_herm(H):
    w, v = np.linalg.eigh(H)
    return v @ np.diag(np.exp(1j * w)) @ v.conj().T


def _fd(op_args, U, phi, slab, site, mu, a, h):
    T_a = inputs.gell_mann()[a] / 2
    Up, Um = U.copy(), U.copy()
    Up[site, mu] = _expm_herm(h * T_a) @ U[site, mu]
    Um[site, mu] = _expm_herm(-h * T_a) @ U[site, mu]
    opp = oracle.Operator(DIMS, Up, *op_args)
    opm = oracle.Operator(DIMS, Um, *op_args)
    _, _, Xp, _ = oracle.link_force(opp, phi, *slab)
    _, _, Xm, _ = oracle.link_force(opm, phi, *slab)
    dm = opm.apply(opm.apply(Xm, *slab), *slab, dagger=True) - opp.apply(opp.apply(Xm, *slab), *slab, dagger=True)
    return np.real(np.vdot(Xp, dm)) / (2 * h)


@pytest.mark.parametrize("csw,bc,slab", [(0.0, oracle.BC_OPEN, (0, 3)), (1.0, oracle.BC_OPEN, (1, 2)),
                                         (1.0, oracle.BC_PERIODIC, (0, 3))])
def test_force_matches_finite_differences(csw, bc, slab):
    U = inputs.random_su3_field(DIMS, 0.4, 51)
    op_args = (0.13, csw, bc)
    op = oracle.Operator(DIMS, U, *op_args)
    phi = inputs.gaussian_spinor(DIMS, 52)[0]
    F, S, X, Y = oracle.link_force(op, phi, *slab)
    assert S > 0
    rng = np.random.default_rng(53)
    # links inside the slab, on its boundary, and outside it (clover leaves reach them)
    t_pick = [slab[0], slab[1], max(slab[0] - 1, 0), (slab[1] + 1) % 4, slab[0]]
    checked = 0
    for t in t_pick:
        site = t * 64 + int(rng.integers(64))
        mu = int(rng.integers(4))
        a = int(rng.integers(8))
        fd = _fd(op_args, U, phi, slab, site, mu, a, 1e-5)
        assert abs(F[site, mu, a] - fd) <= 1e-6 * abs(fd) + 1e-10, (site, mu, a, F[site, mu, a], fd)
        checked += abs(fd) > 1e-4
    # some picks may be links D_L does not depend on (e.g. the absent open-BC link)
    assert checked >= 3
    if csw:
        # the clover term reaches links outside the slab
        outside = op.slab(*slab) == False  # noqa: E712
        if outside.any():
            assert np.abs(F[outside]).max() > 0


def test_force_gauge_covariance():
    U = inputs.random_su3_field(DIMS, 0.4, 61)
    g = inputs.random_gauge_transform(DIMS, 62)
    V = 256
    x = np.stack(np.unravel_index(np.arange(V), DIMS), -1)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % DIMS[mu]
        yi = np.ravel_multi_index(y.T, DIMS)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[yi], -1, -2))
    phi = inputs.gaussian_spinor(DIMS, 63)[0]
    phig = np.einsum("xab,xsb->xsa", g, phi)
    slab = (0, 2)
    F, S, _, _ = oracle.link_force(oracle.Operator(DIMS, U, 0.13, 1.0), phi, *slab)
    Fg, Sg, _, _ = oracle.link_force(oracle.Operator(DIMS, Ug, 0.13, 1.0), phig, *slab)
    assert abs(S - Sg) < 1e-11 * abs(S)
    lam = inputs.gell_mann() / 2
    Fm = np.einsum("xma,aij->xmij", F, lam)
    Fgm = np.einsum("xma,aij->xmij", Fg, lam)
    rot = np.einsum("xab,xmbc,xdc->xmad", g, Fm, np.conj(g))
    assert np.abs(rot - Fgm).max() < 1e-10 * np.abs(Fm).max()
