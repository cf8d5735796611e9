"""Pins of the oracle's quark-line projection (Sec. 3.3 eqs. projection, quark_prop_II_proj) and
of its inverse-iteration projection vectors (Sec. 6).

- orthonormalize: Q^dag Q = 1 and R = Q^dag W upper triangular with a positive real diagonal;
- P_+ is the half of a spinor the boundary block reads: D_dGamma* (1 - P_+) = 0, checked with the
  independent dense operator;
- boundary_modes spans the same space as P_+ (D_L^{-n} V0)|_{g1} computed by dense solves with no
  intermediate orthonormalisation, and its basis is the unique one whose R is upper triangular
  with positive diagonal (inverse iteration with QR steps equals one QR of D_L^{-n} V0);
- a complete basis (N_m = 6 L^3) makes the projected case-II propagator equal to the unprojected
  one; a partial basis equals the dense expression -D_Gamma*^{-1} D_dGamma* Phi Phi^dag D_Gammabar^{-1}.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs
from tests import dense_ref

DIMS = (4, 2, 2, 2)
S3 = 8
KAPPA = 0.12
SPLIT = oracle.Split(gamma=(0, 1), gamma_star=(2, 3), delta=(2, 2))   # Gammabar = 0..2, g1 = 1
X_SRC = (0, 1, 0, 1)


@pytest.fixture(scope="module")
def setup():
    U = inputs.random_su3_field(DIMS, 0.3, 31)
    op = oracle.Operator(DIMS, U, KAPPA, 0.0)
    M = dense_ref.dense_D(U, DIMS, KAPPA, 0.0, "open")
    return U, op, M


def test_orthonormalize_unique_factor():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((50, 7)) + 1j * rng.standard_normal((50, 7))
    Q = oracle.orthonormalize(W)
    assert np.abs(Q.conj().T @ Q - np.eye(7)).max() < 1e-13
    R = Q.conj().T @ W
    assert np.abs(np.tril(R, -1)).max() < 1e-12
    assert np.all(np.abs(np.diag(R).imag) < 1e-12) and np.all(np.diag(R).real > 0)
    assert np.abs(Q @ R - W).max() < 1e-12


def test_plus_projector_is_what_the_boundary_block_reads(setup):
    _, _, M = setup
    P = oracle.spin_project_plus(np.eye(12).reshape(12, 4, 3)).reshape(12, 12).T   # P[:, k] = P_+ e_k
    assert np.abs(P @ P - P).max() < 1e-14 and abs(np.trace(P).real - 6) < 1e-12
    ig = dense_ref.slab_index(DIMS, 1, 1)                    # last slice of Gamma
    igs = dense_ref.slab_index(DIMS, 2, 3)
    Db = M[np.ix_(igs, ig)]                                  # D_dGamma* restricted to its source slice
    comp = np.kron(np.eye(S3), np.eye(12) - P)
    assert np.abs(Db @ comp).max() < 1e-14
    assert np.abs(Db @ np.kron(np.eye(S3), P)).max() > 0.1


def _brute_modes(M, v0, t0, t1, g1, n_iter):
    idx = dense_ref.slab_index(DIMS, t0, t1)
    ML = M[np.ix_(idx, idx)]
    W = np.stack([v0[i].reshape(-1)[idx] for i in range(v0.shape[0])], axis=1)
    for _ in range(n_iter):
        W = np.linalg.solve(ML, W)
    lo = (g1 - t0) * S3 * 12
    B = W[lo:lo + S3 * 12]                                   # (S3*12, N)
    Pp = oracle.spin_project_plus(B.T.reshape(-1, S3, 4, 3)).reshape(-1, S3 * 12).T
    return Pp


@pytest.mark.parametrize("n_m,n_iter", [(5, 3), (12, 4)])
def test_boundary_modes_match_dense_inverse_powers(setup, n_m, n_iter):
    U, op, M = setup
    v0 = inputs.gaussian_spinor(DIMS, 40 + n_m, n_m)
    phi = oracle.boundary_modes(op, v0, 0, 2, 1, n_iter)
    assert phi.shape == (n_m, S3, 4, 3)
    F = phi.reshape(n_m, -1).T                               # (S3*12, N)
    assert np.abs(F.conj().T @ F - np.eye(n_m)).max() < 1e-12
    assert np.abs(oracle.spin_project_plus(phi) - phi).max() < 1e-14
    B = _brute_modes(M, v0, 0, 2, 1, n_iter)
    R = F.conj().T @ B                                       # B = F R, R upper triangular, diag > 0
    assert np.abs(F @ R - B).max() < 1e-10 * np.abs(B).max()
    assert np.abs(np.tril(R, -1)).max() < 1e-10 * np.abs(R).max()
    assert np.all(np.diag(R).real > 0) and np.abs(np.diag(R).imag).max() < 1e-10 * np.abs(R).max()


def test_complete_basis_reproduces_the_unprojected_propagator(setup):
    U, op, M = setup
    n_m = 6 * S3
    v0 = inputs.gaussian_spinor(DIMS, 77, n_m)
    phi = oracle.boundary_modes(op, v0, 0, 2, 1, 2)
    xi, eta = oracle.projected_factors(op, SPLIT, phi)
    proj = oracle.projected_propagator(op, SPLIT, xi, eta, X_SRC)
    fact = oracle.factorized_propagator(op, SPLIT, inputs.point_sources(DIMS, X_SRC))
    m = op.slab(*SPLIT.gamma_star)
    assert np.abs(proj[:, m] - fact[:, m]).max() < 1e-11 * np.abs(fact[:, m]).max()
    assert np.all(proj[:, ~m] == 0)


def test_partial_basis_matches_dense_expression(setup):
    U, op, M = setup
    n_m = 10
    v0 = inputs.gaussian_spinor(DIMS, 91, n_m)
    phi = oracle.boundary_modes(op, v0, 0, 2, 1, 3)
    xi, eta = oracle.projected_factors(op, SPLIT, phi)
    proj = oracle.projected_propagator(op, SPLIT, xi, eta, X_SRC)
    igb = dense_ref.slab_index(DIMS, 0, 2)
    ig = dense_ref.slab_index(DIMS, 0, 1)
    igs = dense_ref.slab_index(DIMS, 2, 3)
    # Phi on the lattice (columns), restricted to Gamma, and the point-source columns
    Phi = np.zeros((12 * 32, n_m), complex)
    for i in range(n_m):
        Phi[12 * S3:24 * S3, i] = phi[i].reshape(-1)
    E = inputs.point_sources(DIMS, X_SRC).reshape(12, -1).T  # (12V, 12)
    DgbInv_E = np.zeros((12 * 32, 12), complex)
    DgbInv_E[igb] = np.linalg.solve(M[np.ix_(igb, igb)], E[igb])
    chi = M[np.ix_(igs, ig)] @ (Phi[ig] @ (Phi.conj().T @ DgbInv_E))
    want = np.zeros((12 * 32, 12), complex)
    want[igs] = -np.linalg.solve(M[np.ix_(igs, igs)], chi)
    got = proj.reshape(12, -1).T
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    assert np.abs(want[igs]).max() > 1e-6
