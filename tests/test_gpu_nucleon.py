"""Parity of the nucleon blocks and contractions on the GPU (Sec. 4.2 eq. nucleon_prop_factorized)
with the FP64 oracle, through the C ABI.

Tolerance of the blocks: the GPU forms the diquark and the (x, c) sum in FP32 (inputs rounded from
FP64), summing in two levels: per-thread partial sums over 64 sites (192 terms), added into running
sums (one per 64 sites).  Each term carries a relative error of a few u32 = 2^-24, so
  |B_gpu - B| <= (3 + 192 + S3/64) u32 * sum_{x,c} |D| |s_k|,
i.e. 1.2e-5 * bound here and 2.4e-5 * bound for a 24^3 slice.  The tensor-core kernel (the default)
sums 64 sites per TMEM accumulation with one rounding of the partial sum per MMA (3 passes per 8 real
K values: 144 per 64 sites, at most 2 u32 each if the tensor core truncates) and takes TF32 hi/lo
splits that lose at most 2^-21 per product (16 u32), so its bound, (16 + 2 * 144 + S3/64) u32, is
1.8e-5 * bound here (below the same tolerance) and 3.1e-5 * bound for a 24^3 slice (the full-size
test in tests/test_gpu_fullsize.py allows 3.5e-5 there); with
bound = sum_{x,c} sum_{ab} |eps| sum_{mn} |s_i| |C g5| |s_j| |s_k| computed here from |s|;
the test allows 3e-5 * bound.  Because |B| is of order bound / sqrt(#terms), a wrong index or sign
moves B by far more than that.  The contraction kernel is FP64: 1e-12 on identical blocks.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_06424_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
S3 = 64


def _lq():
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    return lqcd


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bound(s, t, s3=S3):
    a = np.abs(s[:, t * s3:(t + 1) * s3])                              # (N, S3, 4, 3)
    cg5 = np.abs(oracle.charge_conjugation() @ oracle.gamma(4))
    eps = np.abs(oracle.EPS3)
    d = np.einsum("abc,ixma,mn,jxnb->ijxc", eps, a, cg5, a)
    return np.einsum("ijxc,kxdc->ijkd", d, a)


@pytest.mark.parametrize("kernel", ["fma", "tc"])
@pytest.mark.parametrize("n,conj", [(10, False), (17, True)])
def test_blocks_match_oracle(n, conj, kernel, monkeypatch):
    """Both block kernels: FP32 FMA (k_nucleon_block) and tensor cores (k_nucleon_block_tc,
    TF32 three-pass split, accumulated per 64 sites in TMEM); LQCD_NUCLEON_TC selects."""
    monkeypatch.setenv("LQCD_NUCLEON_TC", "1" if kernel == "tc" else "0")
    lqcd = _lq()
    U = inputs.random_su3_field(DIMS, 0.4, 9)
    lat = lqcd.Lattice(DIMS, "open")
    lat.set_gauge(U, 0.12, 0.0)
    op = oracle.Operator(DIMS, U, 0.12, 0.0)
    rng = np.random.default_rng(n)
    s = rng.standard_normal((n, 512, 4, 3)) + 1j * rng.standard_normal((n, 512, 4, 3))
    slab = (2, 7)
    sl = inputs.slab_sites(DIMS, *slab)
    full = np.zeros_like(s)
    full[:, sl] = s[:, sl]
    B = lat.nucleon_blocks(_cuda(s[:, sl]), slab, 3, 3, conj=conj).cpu().numpy()   # slices 3, 4, 5
    src = np.conj(full) if conj else full
    for q, t in enumerate((3, 4, 5)):
        ref = oracle.nucleon_block(op, src, t)
        bnd = _bound(src, t)
        assert np.all(np.abs(B[q] - ref) <= 3e-5 * bnd + 1e-300), t
        assert np.abs(ref).max() > 1e-3 * bnd.max()       # values far above the tolerance


@pytest.mark.parametrize("conj", [False, True])
def test_tensor_core_blocks_many_tiles(conj, monkeypatch):
    """The tensor-core kernel on 4 x 8^3 (512 sites per slice: 128 chunks of 4 sites, 8 inner
    accumulations of 64 sites folded into the running sums) with N = 40 fields (5 x 3 row tiles
    of 8 x 16 (i, j), 3 column tiles of 16 k, ragged in j and k), two slices: against the
    oracle within the bound above, and against the FP32-FMA kernel."""
    lqcd = _lq()
    dims = (4, 8, 8, 8)
    s3 = 512
    n = 40
    U = inputs.random_su3_field(dims, 0.4, 3)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.12, 0.0)
    op = oracle.Operator(dims, U, 0.12, 0.0)
    rng = np.random.default_rng(40 + conj)
    s = rng.standard_normal((n, 4 * s3, 4, 3)) + 1j * rng.standard_normal((n, 4 * s3, 4, 3))
    got = {}
    for kernel in ("1", "0"):
        monkeypatch.setenv("LQCD_NUCLEON_TC", kernel)
        got[kernel] = lat.nucleon_blocks(_cuda(s), (0, 3), 1, 2, conj=conj).cpu().numpy()   # slices 1, 2
    src = np.conj(s) if conj else s
    for q, t in enumerate((1, 2)):
        ref = oracle.nucleon_block(op, src, t)
        bnd = _bound(src, t, s3)
        assert np.all(np.abs(got["1"][q] - ref) <= 3e-5 * bnd + 1e-300), t
        assert np.all(np.abs(got["1"][q] - got["0"][q]) <= 6e-5 * bnd + 1e-300), t
        assert np.abs(ref).max() > 1e-3 * bnd.max()


def test_contract_matches_oracle_sums():
    lqcd = _lq()
    rng = np.random.default_rng(2)
    n = 6
    bx = rng.standard_normal((2, n, n, n, 4)) + 1j * rng.standard_normal((2, n, n, n, 4))
    by = rng.standard_normal((3, n, n, n, 4)) + 1j * rng.standard_normal((3, n, n, n, 4))
    W = lqcd.nucleon_contract(_cuda(bx), _cuda(by)).cpu().numpy()
    g5pm = oracle.gamma(4) @ (0.5 * (np.eye(4) - oracle.gamma(0)))
    for ix in range(2):
        for iy in range(3):
            w1 = -np.einsum("jikg,gd,ijkd->", bx[ix], g5pm, by[iy])
            w2 = -np.einsum("kijg,gd,ijkd->", bx[ix], g5pm, by[iy])
            assert abs(W[ix, iy, 0] - w1) <= 1e-12 * abs(w1)
            assert abs(W[ix, iy, 1] - w2) <= 1e-12 * abs(w2)


def test_factorized_nucleon_end_to_end():
    """Oracle projection vectors -> GPU factors -> GPU blocks and contraction, against the oracle's
    nucleon_factorized on the oracle's own factors (relative 1e-4: FP32 blocks, see above)."""
    lqcd = _lq()
    U = inputs.random_su3_field(DIMS, 0.4, 10)
    lat = lqcd.Lattice(DIMS, "open")
    lat.set_gauge(U, 0.12, 0.0)
    op = oracle.Operator(DIMS, U, 0.12, 0.0)
    n_m = 12
    phi = oracle.boundary_modes(op, inputs.gaussian_spinor(DIMS, 70, n_m), 2, 5, 3, 2)
    split = oracle.Split(gamma=(0, 3), gamma_star=(4, 7), delta=(4, 4))
    xr, er = oracle.projected_factors(op, split, phi)
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    xi, eta, _ = lat.projected_factors(_cuda(phi), (0, 3), (4, 7), (4, 4), 0, prm)
    Bx = lat.nucleon_blocks(xi, (0, 4), 1, 1, conj=True)
    By = lat.nucleon_blocks(eta, (4, 7), 5, 3)
    W = lqcd.nucleon_contract(Bx, By).cpu().numpy()
    for q, y0 in enumerate((5, 6, 7)):
        w1, w2 = oracle.nucleon_factorized(op, xr, er, 1, y0)
        assert abs(W[0, q, 0] - w1) <= 1e-4 * abs(w1) and abs(w1) > 0
        assert abs(W[0, q, 1] - w2) <= 1e-4 * abs(w2) and abs(w2) > 0


def test_nucleon_errors():
    lqcd = _lq()
    lat = lqcd.Lattice(DIMS, "open")
    s = _cuda(np.zeros((3, 2 * S3, 4, 3), complex))
    with pytest.raises(lqcd.LQCDError):
        lat.nucleon_blocks(s, (2, 3), 3, 2)          # slices 3, 4: 4 outside the slab
    with pytest.raises(lqcd.LQCDError):
        lat.nucleon_blocks(s, (2, 3), 1, 1)


def test_multilevel_nucleon_matches_oracle_estimator():
    """The level-1 part of eq. multilevel_estimator on the GPU (level_mean kernel, then the
    contraction) against the oracle's estimator with the W1 / W2 contractions as the product."""
    lqcd = _lq()
    rng = np.random.default_rng(4)
    n, n1 = 5, 3
    bx = rng.standard_normal((n1, 1, n, n, n, 4)) + 1j * rng.standard_normal((n1, 1, n, n, n, 4))
    by = rng.standard_normal((n1, 2, n, n, n, 4)) + 1j * rng.standard_normal((n1, 2, n, n, n, 4))
    m = lqcd.level_mean(_cuda(bx)).cpu().numpy()
    assert np.abs(m - bx.mean(axis=0)).max() < 1e-15
    W = lqcd.multilevel_nucleon(_cuda(bx), _cuda(by)).cpu().numpy()
    g5pm = oracle.gamma(4) @ (0.5 * (np.eye(4) - oracle.gamma(0)))
    for iy in range(2):
        for q, pat in enumerate(("jikg", "kijg")):
            prod = lambda a, b: -np.einsum(pat + ",gd,ijkd->", a, g5pm, b)
            want = oracle.multilevel_estimator([bx[:, 0]], [by[:, iy]], [[0.0]], prod)
            assert abs(W[0, iy, q] - want) <= 1e-12 * abs(want)


def test_nucleon_point_correlator_matches_oracle():
    """lqcd_nucleon_point (FP64, one warp per site) on random 12-column propagators against the
    oracle's two Wick contractions written as definitions, per sink time slice: 1e-12 of the
    largest |W| (the same FP64 products summed in another order)."""
    lqcd = _lq()
    dims = (6, 4, 4, 6)  # 96 sites per slice: 24 blocks of four sites (every extent is even, so a
    # slice always fills whole blocks)
    lat = lqcd.Lattice(dims, "open")
    rng = np.random.default_rng(31)
    V = int(np.prod(dims))
    props = (rng.standard_normal((2, 12, V, 4, 3)) + 1j * rng.standard_normal((2, 12, V, 4, 3))) / np.sqrt(2)
    W = lat.nucleon_point(_cuda(props)).cpu().numpy()
    for p in range(2):
        ref = oracle.nucleon_point_correlator(props[p], dims[0])
        assert np.abs(W[p] - ref).max() <= 1e-12 * np.abs(ref).max(), p
    # a range of slices gives the same per-slice sums
    W2 = lat.nucleon_point(_cuda(props), t0=2, n_t=3).cpu().numpy()
    assert np.abs(W2 - W[:, 2:5]).max() == 0.0
    lat.close()
    dims = (4, 2, 2, 6)
    lat = lqcd.Lattice(dims, "open")
    V = int(np.prod(dims))
    p1 = (rng.standard_normal((12, V, 4, 3)) + 1j * rng.standard_normal((12, V, 4, 3)))
    W = lat.nucleon_point(_cuda(p1)).cpu().numpy()[0]
    ref = oracle.nucleon_point_correlator(p1, dims[0])
    assert np.abs(W - ref).max() <= 1e-12 * np.abs(ref).max()
    lat.close()


def test_nucleon_hierarchy_matches_oracle():
    """Sec. 6 eq. nucleon_prop_hierarchical on 8 x 4^3 (Wilson-clover kappa 0.13): Gamma = t 0..2,
    Gamma* = 3..7, nested overlaps ending at t = 3, 4, 5, source (1,1,0,2).  The GPU's terms and full
    correlator against the oracle's (factorized propagators by oracle solves, contractions as
    definitions); both solve to 1e-12, so the cubic correlators agree to ~1e-10 relative: 1e-8 of
    max |C| allowed.  The terms telescope to C on the GPU as well."""
    lqcd = _lq()
    dims = (8, 4, 4, 4)
    U = inputs.random_su3_field(dims, 0.4, 33)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.13, 1.0)
    x_src = (1, 1, 0, 2)
    terms, full, st = lat.nucleon_hierarchy((0, 2), (3, 7), [3, 4, 5], x_src,
                                            params=lqcd.SolverParams(tol=1e-12, precision=64))
    for k in ("gamma", "gamma_bar", "gamma_star", "full"):
        assert st[k]["status"] == 0 and st[k]["true_residual"] <= 1e-12, (k, st[k])
    op = oracle.Operator(dims, U, 0.13, 1.0)
    eta = inputs.point_sources(dims, x_src)
    t_ref, _, full_ref = oracle.nucleon_hierarchy(op, (0, 2), (3, 7), [3, 4, 5], eta)
    scale = np.abs(full_ref).max()
    assert np.abs(full - full_ref).max() <= 1e-8 * scale
    assert np.abs(terms - t_ref).max() <= 1e-8 * scale
    assert np.abs(terms.sum(axis=0) - full).max() <= 1e-13 * scale
    lat.close()
