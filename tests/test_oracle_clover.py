"""Pins of the oracle's clover term A(x) = 1/(2 kappa) + c_sw (i/4) sum sigma_mu_nu Fhat_mu_nu(x).

- vanishes (A = 1/(2 kappa)) at U = 1;
- Hermitian and block-diagonal in chirality (commutes with gamma_5);
- gauge covariant: A[U^g](x) = g(x) A[U](x) g(x)^dag;
- closed form for abelian U(1) fields embedded as phases times the colour
  identity: each plaquette in the (mu,nu) plane is exp(i Phi(w)) with w its
  lower-left corner, so Fhat_mu_nu(x) = (i/4) sum over the four corners
  w in {x, x-mu, x-nu, x-mu-nu} of sin Phi(w), and
  A(x) = 1/(2 kappa) - (c_sw/8) sum_w sin Phi(w) sigma_mu_nu.
- the brute-force dense assembly of tests/dense_ref.py (rolled arrays) agrees.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs
from tests import dense_ref


def test_clover_vanishes_on_unit_field():
    dims = (4, 4, 4, 4)
    op = oracle.Operator(dims, inputs.unit_field(dims), 0.13, 1.0)
    assert np.abs(op.A - np.eye(12) / (2 * 0.13)).max() < 1e-15


def test_clover_hermitian_and_chiral():
    dims = (4, 4, 4, 6)
    op = oracle.Operator(dims, inputs.random_su3_field(dims, 0.4, 41), 0.13, 1.0)
    A = op.A
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-15
    # chirality blocks: spin {0,1} x colour and spin {2,3} x colour do not mix
    assert np.abs(A[:, :6, 6:]).max() < 1e-15 and np.abs(A[:, 6:, :6]).max() < 1e-15
    assert np.abs(A - np.eye(12) / 0.26).max() > 0.05


def test_clover_gauge_covariance():
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.4, 42)
    g = inputs.random_gauge_transform(dims, 43)
    T, L1, L2, L3 = dims
    V = T * L1 * L2 * L3
    x = np.stack(np.unravel_index(np.arange(V), dims), -1)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % dims[mu]
        yi = np.ravel_multi_index(y.T, dims)
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[yi], -1, -2))
    A = oracle.Operator(dims, U, 0.13, 1.0).A.reshape(V, 4, 3, 4, 3)
    Ag = oracle.Operator(dims, Ug, 0.13, 1.0).A.reshape(V, 4, 3, 4, 3)
    rot = np.einsum("xab,xsbtc,xdc->xsatd", g, A, np.conj(g))
    assert np.abs(rot - Ag).max() < 1e-13


@pytest.mark.parametrize("mu,nu", [(1, 2), (0, 3), (2, 0)])
def test_clover_abelian_closed_form(mu, nu):
    dims = (6, 4, 6, 4)
    V = int(np.prod(dims))
    x = np.stack(np.unravel_index(np.arange(V), dims), -1)
    rng = np.random.default_rng(7)
    f = rng.uniform(-1, 1, dims[mu])      # U_nu(x) = exp(i f(x_mu))
    h = rng.uniform(-1, 1, dims[nu])      # U_mu(x) = exp(-i h(x_nu))
    U = inputs.unit_field(dims)
    U[:, nu] *= np.exp(1j * f[x[:, mu]])[:, None, None]
    U[:, mu] *= np.exp(-1j * h[x[:, nu]])[:, None, None]
    kappa, csw = 0.125, 1.0
    op = oracle.Operator(dims, U, kappa, csw, oracle.BC_PERIODIC)

    def phi(w):
        # plaquette U_mu(w) U_nu(w+mu) U_mu(w+nu)^dag U_nu(w)^dag = exp(i Phi)
        return (f[(w[:, mu] + 1) % dims[mu]] - f[w[:, mu]]) + (h[(w[:, nu] + 1) % dims[nu]] - h[w[:, nu]])

    def shifted(d_mu, d_nu):
        w = x.copy()
        w[:, mu] = (w[:, mu] + d_mu) % dims[mu]
        w[:, nu] = (w[:, nu] + d_nu) % dims[nu]
        return w

    ssum = sum(np.sin(phi(shifted(a, b))) for a, b in [(0, 0), (-1, 0), (0, -1), (-1, -1)])
    sig = dense_ref.sigma(mu, nu)
    expect = np.eye(12)[None] / (2 * kappa) - (csw / 8) * ssum[:, None, None] * np.kron(sig, np.eye(3))[None]
    assert np.abs(op.A - expect).max() < 1e-14


@pytest.mark.parametrize("bc_name,bc", [("open", oracle.BC_OPEN), ("periodic", oracle.BC_PERIODIC)])
def test_clover_matches_rolled_array_assembly(bc_name, bc):
    dims = (4, 4, 4, 4)
    V = 256
    U = inputs.random_su3_field(dims, 0.4, 44)
    F = dense_ref.clover_fhat(U, dims, bc_name == "open").reshape(4, 4, V, 3, 3)
    expect = np.tile(np.eye(12, dtype=complex) / 0.26, (V, 1, 1))
    for m in range(4):
        for n in range(4):
            if m != n:
                expect += 0.25j * np.einsum("st,xab->xsatb", dense_ref.sigma(m, n), F[m, n]).reshape(V, 12, 12)
    A = oracle.Operator(dims, U, 0.13, 1.0, bc).A
    assert np.abs(A - expect).max() < 1e-14
