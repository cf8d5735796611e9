"""Brute-force pin on 4^4: the oracle's operator, solves, factorized propagator and
correction against a dense matrix assembled independently (tests/dense_ref.py)
and LAPACK LU (numpy.linalg.solve).

Sec. 3: D^{-1} restricted to blocks (eq. block_inverse), fact on Gamma =
D_Gamma^{-1} (eq. quark_prop_I), fact on Gamma* = -D_Gamma*^{-1} D_dGamma*
D_Gammabar^{-1} (eq. quark_prop_II), corr = D^{-1} - fact (eq.
observable_factorization).  Also the exact identity fact + corr_Schur = full,
with corr_Schur computed from the Schur complements only.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs
from tests import dense_ref

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module", params=[(0.12, 0.0, 0.3), (0.13, 1.0, 0.4)], ids=["wilson", "clover"])
def setup(request):
    kappa, csw, eps = request.param
    U = inputs.random_su3_field(DIMS, eps, 1)
    op = oracle.Operator(DIMS, U, kappa, csw)
    M = dense_ref.dense_D(U, DIMS, kappa, csw, "open")
    return op, M


def test_operator_matches_dense(setup):
    op, M = setup
    v = inputs.gaussian_spinor(DIMS, 3)[0]
    assert np.abs(op.apply(v).reshape(-1) - M @ v.reshape(-1)).max() < 1e-13
    assert np.abs(op.apply(v, dagger=True).reshape(-1) - M.conj().T @ v.reshape(-1)).max() < 1e-13
    idx = dense_ref.slab_index(DIMS, 1, 2)
    vm = op.masked(v, 1, 2)
    got = op.apply(vm, 1, 2).reshape(-1)
    assert np.abs(got[idx] - M[np.ix_(idx, idx)] @ vm.reshape(-1)[idx]).max() < 1e-13
    mask = np.ones(got.size, bool)
    mask[idx] = False
    assert np.abs(got[mask]).max() == 0.0


@pytest.mark.parametrize("split", [oracle.Split((0, 1), (2, 3)),
                                   oracle.Split((0, 1), (2, 3), delta=(2, 2)),
                                   oracle.Split((0, 0), (1, 3), delta=(1, 2))],
                         ids=["no_overlap", "delta1", "delta2"])
def test_factorized_propagator_matches_dense_lu(setup, split):
    op, M = setup
    eta = inputs.point_sources(DIMS, (split.gamma[0], 1, 2, 3))[[0, 5, 7, 11]]
    V12 = M.shape[0]
    ig = dense_ref.slab_index(DIMS, *split.gamma)
    igs = dense_ref.slab_index(DIMS, *split.gamma_star)
    igb = dense_ref.slab_index(DIMS, *split.gamma_bar)
    E = eta.reshape(eta.shape[0], -1).T
    full = np.linalg.solve(M, E)
    fact = np.zeros_like(full)
    fact[ig] = np.linalg.solve(M[np.ix_(ig, ig)], E[ig])
    psi_gb = np.zeros_like(full)
    psi_gb[igb] = np.linalg.solve(M[np.ix_(igb, igb)], E[igb])
    chi = M[np.ix_(igs, ig)] @ psi_gb[ig]
    fact[igs] = -np.linalg.solve(M[np.ix_(igs, igs)], chi)
    got_fact = oracle.factorized_propagator(op, split, eta).reshape(eta.shape[0], -1).T
    got_full = oracle.full_propagator(op, eta).reshape(eta.shape[0], -1).T
    scale = np.abs(full).max()
    assert np.abs(got_full - full).max() < 1e-12 * scale
    assert np.abs(got_fact - fact).max() < 1e-12 * scale
    # Schur identity: fact + corr (from block inverses only) = full
    corr = oracle.schur_correction(op, split, eta).reshape(eta.shape[0], -1).T
    assert np.abs(fact + corr - full).max() < 1e-11 * scale
    # Sec. 3.1: with no overlap the case-I block of D^{-1} is S_Gamma^{-1} = (D^{-1})_{Gamma Gamma}
    Sg = np.linalg.inv(M[np.ix_(ig, ig)] - M[np.ix_(ig, igs)] @ np.linalg.solve(M[np.ix_(igs, igs)], M[np.ix_(igs, ig)]))
    assert np.abs(Sg @ E[ig] - full[ig]).max() < 1e-11 * scale
    assert V12 == 3072
