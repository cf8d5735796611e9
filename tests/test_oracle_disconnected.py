"""Pins of the oracle's disconnected-trace estimator (Sec. 5, eq. stochastic_estimator).

- exact identity per site, checked by dense LU: with K = kappa D_hop,
  D^{-1} = 2 kappa sum_{n<8} K^n + K^8 D^{-1} and tr{gamma_5 K^n(x,x)} = 0 for n < 8
  (the spin trace of a closed path with gamma_5 survives only when the path uses all
  four directions, i.e. at least 8 hops), so tr{g5 D^{-1}(x,x)} = tr{g5 K^8 D^{-1}(x,x)};
- with the 12 V unit vectors as sources (the 1/n_src normalisation undone) the
  estimator is the exact slice sum of tr{g5 D_L^{-1}(x,x)} from the dense LU inverse;
- per Gaussian source, the value equals the dense-matrix expression (a wrong power,
  sign or gamma_5 placement fails it), and nine hops break the unit-source equality.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06424_gb300 import inputs
from tests import dense_ref

G5 = np.repeat([1.0, 1.0, -1.0, -1.0], 3)


def _site_traces(M, nsite):
    """tr{g5 M(x,x)} for every site x of a (12 nsite)^2 matrix."""
    g5 = np.tile(G5, nsite)
    return (g5 * M.diagonal()).reshape(nsite, 12).sum(axis=1)


def test_hopping_identity_dense():
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.3, 1)
    kappa = 0.12
    M = dense_ref.dense_D(U, dims, kappa, 0.0, "open")
    Minv = np.linalg.inv(M)
    K = np.eye(M.shape[0]) - 2 * kappa * M
    Kn = np.eye(M.shape[0], dtype=complex)
    for n in range(8):
        assert np.abs(_site_traces(Kn, 256)).max() < 1e-12, n
        Kn = K @ Kn
    lhs = _site_traces(Minv, 256)
    rhs = _site_traces(Kn @ Minv, 256)
    assert np.abs(lhs).max() > 1e-6  # non-trivial
    assert np.abs(lhs - rhs).max() < 1e-12


def _unit_sources(dims, t0, t1):
    s3 = dims[1] * dims[2] * dims[3]
    V = dims[0] * s3
    n = (t1 - t0 + 1) * s3 * 12
    etas = np.zeros((n, V, 4, 3), complex)
    k = 0
    for x in range(t0 * s3, (t1 + 1) * s3):
        for s in range(4):
            for c in range(3):
                etas[k, x, s, c] = 1.0
                k += 1
    return etas


@pytest.mark.parametrize("slab", [(0, 3), (1, 2)])
def test_estimator_with_unit_sources_is_exact(slab):
    dims = (4, 2, 2, 2)
    U = inputs.random_su3_field(dims, 0.3, 2)
    kappa = 0.12
    op = oracle.Operator(dims, U, kappa, 0.0)
    M = dense_ref.dense_D(U, dims, kappa, 0.0, "open")
    idx = dense_ref.slab_index(dims, *slab)
    Minv = np.linalg.inv(M[np.ix_(idx, idx)])
    s3 = 8
    exact = np.zeros(4, complex)
    exact[slab[0]:slab[1] + 1] = _site_traces(Minv, idx.size // 12).reshape(-1, s3).sum(axis=1)
    etas = _unit_sources(dims, *slab)
    est = oracle.disconnected_trace(op, etas, *slab) * len(etas)
    assert np.abs(est[slab[0]:slab[1] + 1]).min() > 1e-6
    assert np.abs(est - exact).max() < 1e-10 * np.abs(exact).max()


def test_estimator_per_source_matches_dense():
    """Per Gaussian source, eta^dag (1 - 2 kappa D_L)^8 D_L^{-1} g5 eta from dense matrices
    built by the independent test-side operator; catches a wrong power, sign or g5 side."""
    dims = (4, 2, 2, 2)
    U = inputs.random_su3_field(dims, 0.3, 3)
    kappa = 0.12
    op = oracle.Operator(dims, U, kappa, 0.0)
    M = dense_ref.dense_D(U, dims, kappa, 0.0, "open")
    rng = np.random.default_rng(7)
    for slab in [(0, 3), (1, 3)]:
        idx = dense_ref.slab_index(dims, *slab)
        ML = M[np.ix_(idx, idx)]
        K8 = np.linalg.matrix_power(np.eye(idx.size) - 2 * kappa * ML, 8)
        g5 = np.tile(G5, idx.size // 12)
        for _ in range(2):
            eta = (rng.standard_normal((32, 4, 3)) + 1j * rng.standard_normal((32, 4, 3))) / np.sqrt(2)
            e = eta.reshape(-1)[idx]
            v = np.conj(e) * (K8 @ np.linalg.solve(ML, g5 * e))
            want = np.zeros(4, complex)
            want[slab[0]:slab[1] + 1] = v.reshape(-1, 8 * 12).sum(axis=1)
            got = oracle.disconnected_trace(op, eta[None], *slab)
            assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
            # a different power gives a different per-source value
            got7 = oracle.disconnected_trace(op, eta[None], *slab, hops=7)
            assert np.abs(got7 - want).max() > 1e-4 * np.abs(want).max()


def test_ninth_power_breaks_exactness():
    """n = 9 hops is one too many: K^9 D^{-1} = K^8 D^{-1} - 2 kappa K^8 and tr{g5 K^8(x,x)} != 0."""
    dims = (4, 2, 2, 2)
    U = inputs.random_su3_field(dims, 0.3, 5)
    op = oracle.Operator(dims, U, 0.12, 0.0)
    etas = _unit_sources(dims, 0, 3)
    est8 = oracle.disconnected_trace(op, etas, 0, 3)
    est9 = oracle.disconnected_trace(op, etas, 0, 3, hops=9)
    assert np.abs(est8 - est9).max() > 1e-6 * np.abs(est8).max()


def test_estimator_rejects_clover():
    dims = (4, 2, 2, 2)
    U = inputs.random_su3_field(dims, 0.3, 4)
    op = oracle.Operator(dims, U, 0.12, 1.0)
    with pytest.raises(ValueError):
        oracle.disconnected_trace(op, np.zeros((1, 32, 4, 3), complex), 0, 3)
