"""Parity of the disconnected-trace estimator (Sec. 5, eq. stochastic_estimator) on the
GPU with the FP64 oracle, through the C ABI.

Tolerance: the GPU solves D_L psi = g5 eta to relative residual 1e-12 (FP32 inner
solves inside FP64 defect correction), the oracle to 1e-13.  The solution error is
at most cond(D_L) * 1e-12 * |eta_L|, the eight hops have norm <= (8 kappa)^8 < 1, so
per slice |t_gpu - t_oracle| <= cond * 1e-12 * |eta_L|^2; with cond(D_L) < 100 for
these fields the test allows 1e-9 * |eta_L|^2 (|eta_L|^2 summed over the slab).
The hops and the contraction are FP64 on both sides.
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


@pytest.mark.parametrize("dims,doms", [
    ((16, 8, 8, 8), [(0, 7), (8, 15), (0, 15)]),           # the two Dirichlet domains and the full lattice
    ((10, 6, 6, 4), [(0, 4), (5, 9), (3, 3), (0, 9)]),     # ragged tail (72 sites per slice and parity), one-slice slab
])
def test_disconnected_trace_matches_oracle(dims, doms):
    lqcd = _lq()
    kappa = 0.12
    U = inputs.random_su3_field(dims, 0.4, 11)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, 0.0)
    n_src = 3
    eta = inputs.gaussian_spinor(dims, 12, n_src)
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    tr, mean, stats = lat.disconnected_trace(_cuda(eta), doms, 0, prm)
    tr = tr.cpu().numpy()
    mean = mean.cpu().numpy()
    assert all(s["status"] == 0 and s["true_residual"] <= 1e-12 for s in stats), stats
    op = oracle.Operator(dims, U, kappa, 0.0)
    s3 = int(np.prod(dims[1:]))
    for d, (t0, t1) in enumerate(doms):
        for i in range(n_src):
            ref = oracle.disconnected_trace(op, eta[i:i + 1], t0, t1)
            eta2 = np.sum(np.abs(eta[i, t0 * s3:(t1 + 1) * s3]) ** 2)
            assert np.abs(tr[i, d] - ref).max() <= 1e-9 * eta2, (d, i)
            assert np.all(tr[i, d, :t0] == 0) and np.all(tr[i, d, t1 + 1:] == 0)
            assert np.abs(ref[t0:t1 + 1]).min() > 1e-6  # non-trivial values compared
        # the mean is the source average of the per-source values
        assert np.abs(mean[d] - tr[:, d].mean(axis=0)).max() <= 1e-14 * np.abs(tr[:, d]).max()


def test_disconnected_trace_unit_sources_exact():
    """All 12 V unit vectors as sources on a 4x2x2x2 lattice: n_src * mean equals the exact
    slice sums of tr{g5 D_L^{-1}(x,x)} from the oracle's dense per-column solves."""
    lqcd = _lq()
    dims = (4, 2, 2, 2)
    kappa = 0.12
    U = inputs.random_su3_field(dims, 0.3, 2)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, 0.0)
    V = 32
    etas = np.zeros((12 * V, V, 4, 3), complex)
    for k in range(12 * V):
        etas[k, k // 12, (k % 12) // 3, k % 3] = 1.0
    prm = lqcd.SolverParams(tol=1e-13, precision=64)
    _, mean, _ = lat.disconnected_trace(_cuda(etas), [(0, 3), (1, 2)], 0, prm)
    got = mean.cpu().numpy() * (12 * V)
    op = oracle.Operator(dims, U, kappa, 0.0)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    for d, (t0, t1) in enumerate([(0, 3), (1, 2)]):
        exact = np.zeros(4, complex)
        for x in range(t0 * 8, (t1 + 1) * 8):
            for s in range(4):
                for c in range(3):
                    e = np.zeros((V, 4, 3), complex)
                    e[x, s, c] = 1.0
                    col, _, _ = op.solve(np.einsum("st,xtc->xsc", g5, e), t0, t1, tol=1e-14)
                    exact[x // 8] += col[x, s, c]  # [D_L^{-1} g5](x s c, x s c)
        assert np.abs(got[d] - exact).max() <= 1e-10 * np.abs(exact).max(), d


def test_disconnected_trace_rejects_clover_and_bad_slabs():
    lqcd = _lq()
    dims = (4, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.3, 3)
    lat = lqcd.Lattice(dims, "open")
    eta = _cuda(inputs.gaussian_spinor(dims, 1, 1))
    lat.set_gauge(U, 0.12, 1.0)
    with pytest.raises(lqcd.LQCDError):
        lat.disconnected_trace(eta, [(0, 3)])
    lat.set_gauge(U, 0.12, 0.0)
    for bad in [(2, 1), (0, 4), (-1, 2)]:
        with pytest.raises(lqcd.LQCDError):
            lat.disconnected_trace(eta, [bad])
    with pytest.raises(lqcd.LQCDError):
        lat.disconnected_trace(eta, [(0, 3)], field=1)
