"""Parity at the full sizes of the workloads, checked with the oracle's own operator.

Oracle solves at this size take hours, so every GPU result is checked through
properties the exact answer has, each evaluated with the oracle's independent
FP64 D (no oracle input comes from the CUDA path except the vectors under test):
  full = fact + corr solves D full = eta               (eq. observable_factorization)
  fact on Gamma solves D_Gamma fact = eta              (eq. quark_prop_I)
  psi = D_Gammabar^{-1} eta (solve_block) solves D_Gammabar psi = eta
  -fact on Gamma* solves D_Gamma* (-fact) = P_Gamma* D P_Gamma psi   (eq. quark_prop_II)
Tolerance: the solver's residual 1e-10 (x 1.05 for rounding of the check).  The last
property uses the test's own Gammabar solution psi: it and the one inside the
propagator each meet ||eta - D_Gammabar psi|| <= 1e-10 ||eta||, so their boundary hops
agree to the tolerance relative to ||eta|| (not to the much smaller ||chi||), and the
check allows 1.05e-10 (||chi|| + ||eta||).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_06424_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS = (32, 16, 16, 16)
KAPPA, CSW = 0.13, 1.0
G, DL, GS = (0, 13), (14, 17), (14, 31)
GB = (0, 17)
X_SRC = (2, 0, 0, 0)
COLS = tuple(range(12))  # every column of the propagator


@pytest.fixture(scope="module")
def field():
    U = inputs.random_su3_field(DIMS, 0.4, 1)
    return U, oracle.Operator(DIMS, U, KAPPA, CSW)


def _res(op, b, x, slab):
    r = b - op.apply(x, *slab)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [32, 64])
def test_factorized_propagator_16x32_properties(field, prec):
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    U, op = field
    lat = lqcd.Lattice(DIMS, "open")
    lat.set_gauge(U, KAPPA, CSW)
    params = lqcd.SolverParams(tol=1e-10, precision=prec)
    fact, corr, st = lat.factorized_propagator(G, GS, X_SRC, delta=DL, corr=True, params=params)
    eta = inputs.point_sources(DIMS, X_SRC)
    sgb = inputs.slab_sites(DIMS, *GB)
    src = torch.from_numpy(np.ascontiguousarray(eta[:, sgb])).reshape(-1, 4, 3).cuda()
    psi_gb, st_gb = lat.solve_block(src.contiguous(), [GB] * 12, [0] * 12, params)
    fact, corr = fact.cpu().numpy(), corr.cpu().numpy()
    psi_gb = psi_gb.cpu().numpy().reshape(12, -1, 4, 3)
    tol = 1.05e-10
    for k in ("gamma", "gamma_bar", "gamma_star", "full"):
        assert st[k]["status"] == 0 and st[k]["true_residual"] <= 1e-10, (k, st[k])
    m_g, m_gs = op.slab(*G), op.slab(*GS)
    for c in COLS:
        assert _res(op, eta[c], fact[c] + corr[c], (0, DIMS[0] - 1)) <= tol
        b_g = op.masked(eta[c], *G)
        x_g = op.masked(fact[c], *G)
        assert _res(op, b_g, x_g, G) <= tol
        x_gb = np.zeros((op.V, 4, 3), complex)
        x_gb[sgb] = psi_gb[c]
        assert _res(op, op.masked(eta[c], *GB), x_gb, GB) <= tol
        chi = op.boundary_hop(x_gb, G, GS)
        zeta = -op.masked(fact[c], *GS)
        r = np.linalg.norm(chi - op.apply(zeta, *GS))
        assert r <= tol * (np.linalg.norm(chi) + np.linalg.norm(eta[c])), (c, r, np.linalg.norm(chi))
        # fact is supported on Gamma u Gamma* = the whole lattice and splits exactly there
        assert np.all(fact[c][~(m_g | m_gs)] == 0)
    lat.close()


def _sample_sites(dims, slab, x_src, n_random, rng):
    """Natural indices of a fixed site sample of a slab: the source, four sites on each of
    the slab's two boundary slices and n_random sites inside."""
    s3 = dims[1] * dims[2] * dims[3]
    a, b = slab
    src = ((x_src[0] * dims[1] + x_src[1]) * dims[2] + x_src[2]) * dims[3] + x_src[3]
    out = [src] + [a * s3 + int(v) for v in rng.integers(s3, size=4)] + [b * s3 + int(v) for v in rng.integers(s3, size=4)]
    out += [int(v) for v in rng.integers(a * s3, (b + 1) * s3, size=n_random)]
    return np.array(out, dtype=np.int64)


def _neighbours(dims, sites):
    """The sites themselves and their 8 nearest neighbours (periodic wrap; the slab
    operator ignores the ones outside its slab)."""
    T, L1, L2, L3 = dims
    x3 = sites % L3
    x2 = (sites // L3) % L2
    x1 = (sites // (L3 * L2)) % L1
    x0 = sites // (L3 * L2 * L1)
    out = [sites]
    for d, (x, L) in enumerate(((x0, T), (x1, L1), (x2, L2), (x3, L3))):
        for step in (1, -1):
            c = [x0, x1, x2, x3]
            c[d] = (x + step) % L
            out.append(((c[0] * L1 + c[1]) * L2 + c[2]) * L3 + c[3])
    return np.unique(np.concatenate(out))


def test_batched_32x64_domain_propagators_sampled():
    """The 32^3x64 batched workload (8 slabs x 12 sources x 16 inner-level fields,
    1536 systems, FP16 inner solves + FP64 correction).  Every system reports a true
    residual <= 1e-10, and every system's residual eta - D_L psi is evaluated by the
    oracle (one site at a time, clover from the links) on a fixed 24-site sample of
    its slab: the source, both boundary slices and random sites.  On field 0, one
    column of each slab is checked in full with the oracle's operator."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (64, 32, 32, 32)
    slabs = [(8 * d, 8 * d + 7) for d in range(8)]
    nf = 16
    s3 = 32 ** 3
    U0 = inputs.random_su3_field_device(dims, 0.4, 3, device="cuda")
    Uf = inputs.inner_level_fields_device(U0, dims, slabs, nf, 0.4, 4)
    del U0
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(Uf, 0.134, 1.0)
    doms, fields, xs, cols = [], [], [], []
    for j in range(nf):
        for d, (a, b) in enumerate(slabs):
            for c in range(12):
                doms.append((a, b)); fields.append(j); xs.append((a + 4, 0, 0, 0)); cols.append(c)
    sol, st = lat.point_propagators(doms, fields, xs, cols, lqcd.SolverParams(tol=1e-10, precision=16))
    assert all(x["status"] == 0 and x["true_residual"] <= 1e-10 for x in st)
    n_slab = lat.slab_len(0, 7)
    rng = np.random.default_rng(12)
    V = lat.V
    buf = np.zeros((V, 4, 3), complex)  # full-lattice input of the oracle, filled only where read
    for j in range(nf):
        U = Uf[j].cpu().numpy()
        for k in [q for q in range(len(doms)) if fields[q] == j]:
            a, b = doms[k]
            smp = _sample_sites(dims, (a, b), xs[k], 15, rng)
            need = _neighbours(dims, smp)
            need = need[(need >= a * s3) & (need < (b + 1) * s3)]
            idx = torch.from_numpy(k * n_slab + need - a * s3).cuda()
            buf[need] = sol.index_select(0, idx).cpu().numpy()
            eta = np.zeros((len(smp), 4, 3), complex)
            s0, c0 = divmod(cols[k], 3)
            eta[smp == smp[0], s0, c0] = 1.0  # the first sample is the source site
            r = eta - oracle.dirac_at_sites(dims, U, 0.134, 1.0, oracle.BC_OPEN, (a, b), smp, buf)
            buf[need] = 0
            assert np.abs(r).max() <= 1e-10, (k, np.abs(r).max())
    # field 0 in full, one column per slab
    op = oracle.Operator(dims, Uf[0].cpu().numpy(), 0.134, 1.0)
    for d, (a, b) in enumerate(slabs):
        k = 12 * d + (5 * d) % 12
        x = np.zeros((op.V, 4, 3), complex)
        x[inputs.slab_sites(dims, a, b)] = sol[k * n_slab:(k + 1) * n_slab].cpu().numpy()
        eta = np.zeros((op.V, 4, 3), complex)
        s0, c0 = divmod(cols[k], 3)
        eta[((xs[k][0] * 32 + xs[k][1]) * 32 + xs[k][2]) * 32 + xs[k][3], s0, c0] = 1.0
        assert _res(op, eta, x, (a, b)) <= 1.05e-10, k
    lat.close()


def _expm_i(H):
    w, v = np.linalg.eigh(H)
    return v @ np.diag(np.exp(1j * w)) @ v.conj().T


def test_link_force_24x48_finite_differences():
    """Force of phi^dag (D_L^dag D_L)^{-1} phi on the 24^3x48 lattice, domain
    t 12..23, against central finite differences (h = 1e-5) on 64 random links
    inside, on and around the domain.  The difference S(+h) - S(-h) is taken
    without cancellation as X+^dag (M- - M+) X-, M = D_L^dag D_L, with the GPU's
    FP64 solves (D_L^{-dag} = g5 D_L^{-1} g5) and operator."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (48, 24, 24, 24)
    dom = (12, 23)
    Ud = inputs.random_su3_field_device(dims, 0.4, 5, device="cuda")
    U = Ud.cpu().numpy()
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(Ud, 0.132, 1.0)
    sl = inputs.slab_sites(dims, *dom)
    phi = torch.from_numpy(inputs.gaussian_spinor(dims, 51)[0][sl]).cuda()
    params = lqcd.SolverParams(tol=1e-12, precision=64)
    F, S, _ = lat.link_force(phi, dom, 0, params)
    F = F.cpu().numpy()
    g5 = torch.tensor([1, 1, -1, -1], dtype=torch.complex128, device="cuda").view(1, 4, 1)
    rng = np.random.default_rng(7)
    s3 = 24 ** 3
    lam = inputs.gell_mann() / 2
    h = 1e-5
    worst = 0.0
    for t in rng.choice([11, 12, 13, 17, 22, 23, 24], size=64):
        site = int(t) * s3 + int(rng.integers(s3))
        mu, a = int(rng.integers(4)), int(rng.integers(8))
        Up, Um = U[site, mu].copy(), U[site, mu].copy()
        Up = _expm_i(h * lam[a]) @ Up
        Um = _expm_i(-h * lam[a]) @ Um
        two = Ud.unsqueeze(0).repeat(2, 1, 1, 1, 1)
        two[0, site, mu] = torch.from_numpy(Up).cuda()
        two[1, site, mu] = torch.from_numpy(Um).cuda()
        lat.set_gauge(two, 0.132, 1.0)
        X = []
        for f in (0, 1):
            y, _ = lat.solve_block((g5 * phi).contiguous(), [dom], [f], params)   # D^{-1} g5 phi
            y = (g5 * y).contiguous()                                            # Y = D^{-dag} phi
            x, _ = lat.solve_block(y, [dom], [f], params)                        # X = D^{-1} Y
            X.append(x)
        Xp, Xm = X

        def M(f, v):
            return lat.dslash(lat.dslash(v, f, dom, False, 64), f, dom, True, 64)

        dS = torch.vdot(Xp.reshape(-1), (M(1, Xm) - M(0, Xm)).reshape(-1)).real.item()
        fd = dS / (2 * h)
        err = abs(F[site, mu, a] - fd)
        assert err <= 1e-6 * abs(fd) + 1e-9 * np.abs(F).max(), (site, mu, a, F[site, mu, a], fd)
        worst = max(worst, err)
    lat.close()


def test_link_force_24x48_against_oracle_formula():
    """The GPU force kernels at 24^3x48 (domain t 12..23, kappa 0.132, c_sw 1) against the
    oracle's force formula F = -2 Re <Y, dD_L X> evaluated on the GPU's own X and Y.  X and Y
    come from separate FP64 GPU solves (Y = D_L^{-dag} phi via g5 D_L^{-1} g5, X = D_L^{-1} Y,
    residual 1e-12), and the oracle's D first confirms D_L^dag Y = phi and D_L X = Y to
    1.05e-12.  lat.link_force solves for its own X and Y to 1e-12, so the two forces differ
    by cond(D_L) x 1e-12 relative; 1e-9 of max |F| is allowed, element by element on every
    link of the lattice."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (48, 24, 24, 24)
    dom = (12, 23)
    U = inputs.random_su3_field(dims, 0.4, 5)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(torch.from_numpy(U).cuda(), 0.132, 1.0)
    sl = inputs.slab_sites(dims, *dom)
    phi_h = inputs.gaussian_spinor(dims, 52)[0]
    phi = torch.from_numpy(np.ascontiguousarray(phi_h[sl])).cuda()
    params = lqcd.SolverParams(tol=1e-12, precision=64)
    F, S, st = lat.link_force(phi, dom, 0, params)
    assert all(x["status"] == 0 for x in st), st
    g5 = torch.tensor([1, 1, -1, -1], dtype=torch.complex128, device="cuda").view(1, 4, 1)
    y, _ = lat.solve_block((g5 * phi).contiguous(), [dom], [0], params)
    y = (g5 * y).contiguous()
    x, _ = lat.solve_block(y, [dom], [0], params)
    op = oracle.Operator(dims, U, 0.132, 1.0)
    X = np.zeros((op.V, 4, 3), complex)
    Y = np.zeros((op.V, 4, 3), complex)
    X[sl] = x.cpu().numpy()
    Y[sl] = y.cpu().numpy()
    phi_m = op.masked(phi_h, *dom)
    assert np.linalg.norm(phi_m - op.apply(Y, *dom, dagger=True)) <= 1.05e-12 * np.linalg.norm(phi_m)
    assert np.linalg.norm(Y - op.apply(X, *dom)) <= 1.05e-12 * np.linalg.norm(Y)
    F_ref = op.force(X, Y, *dom)
    F = F.cpu().numpy()
    scale = np.abs(F_ref).max()
    assert scale > 0
    assert np.abs(F - F_ref).max() <= 1e-9 * scale
    assert abs(S - np.linalg.norm(Y) ** 2) <= 1e-9 * S
    lat.close()


def test_factorized_48x96_sampled_sites():
    """48^3x96, kappa 0.135, c_sw 1: Gamma 0..43, frozen 44..51, Gamma* 44..95, one
    inner-level field, FP32 inner + FP64 correction.  Sampled sites (all time
    slices near the cuts, and random ones) of the residuals
      eta - D (fact + corr),  eta - D_Gamma fact|_Gamma
    are evaluated by the oracle one site at a time (no oracle clover array over
    10.6 M sites); each must stay below the solver tolerance times |eta|."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (96, 48, 48, 48)
    G, DL, GS = (0, 43), (44, 51), (44, 95)
    U0 = inputs.random_su3_field_device(dims, 0.4, 7, device="cuda")
    Uj = inputs.inner_level_fields_device(U0, dims, [G, (52, 95)], 8, 0.4, 8, frozen=DL, field_ids=[3])
    del U0
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(Uj, 0.135, 1.0)
    fact, corr, st = lat.factorized_propagator(G, GS, (2, 0, 0, 0), delta=DL, corr=True,
                                               params=lqcd.SolverParams(tol=1e-10, precision=32))
    for k in ("gamma", "gamma_bar", "gamma_star", "full"):
        assert st[k]["status"] == 0 and st[k]["true_residual"] <= 1e-10, (k, st[k])
    U = Uj[0].cpu().numpy()
    del Uj
    s3 = 48 ** 3
    rng = np.random.default_rng(11)
    ts = [0, 1, 2, 3, 42, 43, 44, 45, 50, 51, 52, 94, 95] + list(rng.integers(0, 96, 8))
    sites = np.array([t * s3 + int(rng.integers(s3)) for t in ts] + [2 * s3])  # + the source site
    for c in (0, 11):
        full = (fact[c] + corr[c]).cpu().numpy()
        eta = np.zeros_like(full)
        s0, c0 = divmod(c, 3)
        eta[2 * s3, s0, c0] = 1.0
        r = eta[sites] - oracle.dirac_at_sites(dims, U, 0.135, 1.0, oracle.BC_OPEN, (0, 95), sites, full)
        assert np.abs(r).max() <= 1e-10
        fg = fact[c].cpu().numpy()
        fg[(G[1] + 1) * s3:] = 0  # fact restricted to Gamma
        in_g = sites[sites < (G[1] + 1) * s3]
        r = eta[in_g] - oracle.dirac_at_sites(dims, U, 0.135, 1.0, oracle.BC_OPEN, G, in_g, fg)
        assert np.abs(r).max() <= 1e-10
    lat.close()


def test_disconnected_64x24_against_oracle_contraction():
    """The 64x24^3 Wilson disconnected-trace workload (kappa 0.136), one Gaussian source on
    Gamma* = t 33..63 and on the full lattice.  A separate solve psi = D_L^{-1} g5 eta
    (solve_block, residual 1e-12) is checked with the oracle's D; the oracle then applies
    its own eight hops and contraction (eq. stochastic_estimator) to psi.  Both solves
    reach 1e-12, so the traces differ by at most cond(D_L) * 2e-12 * |eta_L|^2; with
    cond(D_L) < 500 the test allows 1e-9 * |eta_L|^2 per slice."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    kappa = 0.136
    U = inputs.random_su3_field(dims, 0.4, 21)
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(torch.from_numpy(U).cuda(), kappa, 0.0)
    eta = inputs.gaussian_spinor(dims, 23, 1)
    doms = [(33, 63), (0, 63)]
    prm = lqcd.SolverParams(tol=1e-12, precision=32)
    tr, _, st = lat.disconnected_trace(torch.from_numpy(eta).cuda(), doms, 0, prm)
    assert all(s["status"] == 0 for s in st), st
    tr = tr.cpu().numpy()
    op = oracle.Operator(dims, U, kappa, 0.0)
    s3 = 24 ** 3
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None]
    for d, (t0, t1) in enumerate(doms):
        sl = inputs.slab_sites(dims, t0, t1)
        b = np.zeros_like(eta[0])
        b[sl] = g5 * eta[0][sl]
        x, _ = lat.solve_block(torch.from_numpy(np.ascontiguousarray(b[sl])).cuda(), [(t0, t1)], [0], prm)
        psi = np.zeros_like(b)
        psi[sl] = x.cpu().numpy()
        assert _res(op, b, psi, (t0, t1)) <= 1.05e-12
        ref = oracle.disconnected_contract(op, eta, psi[None], t0, t1)
        eta2 = np.sum(np.abs(eta[0][sl]) ** 2)
        assert np.abs(tr[0, d] - ref).max() <= 1e-9 * eta2, d
        assert np.abs(ref[t0:t1 + 1]).min() > 0
    lat.close()


def test_nucleon_blocks_120_modes_24cube_sampled():
    """The block kernel (tensor cores by default) in the launch configuration of the 64x24^3
    projection workload (N_m = 120, a 24^3 slice, ragged k tile): sampled (i, j) rows of B against
    the oracle's definition written for those rows, within the bound of tests/test_gpu_nucleon.py
    for a 24^3 slice ((16 + 288 + 216) u32 = 3.1e-5 of the bound built from |s| for the tensor-core
    kernel, (3 + 192 + 216) u32 = 2.4e-5 for the FP32-FMA one; 3.5e-5 allowed)."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    s3 = 24 ** 3
    n = 120
    lat = lqcd.Lattice(dims, "open")
    rng = np.random.default_rng(17)
    s = (rng.standard_normal((n, s3, 4, 3)) + 1j * rng.standard_normal((n, s3, 4, 3))) / np.sqrt(2)
    B = lat.nucleon_blocks(torch.from_numpy(s).cuda(), (4, 4), 4, 1, conj=True)[0]
    f = np.conj(s)
    cg5 = oracle.charge_conjugation() @ oracle.gamma(4)
    for i, j in [(0, 5), (61, 77), (119, 118), (8, 8)]:
        d = np.einsum("abc,xma,mn,xnb->xc", oracle.EPS3, f[i], cg5, f[j])
        want = np.einsum("xc,kxdc->kd", d, f)
        db = np.einsum("abc,xma,mn,xnb->xc", np.abs(oracle.EPS3), np.abs(f[i]), np.abs(cg5), np.abs(f[j]))
        bound = np.einsum("xc,kxdc->kd", db, np.abs(f))
        got = B[i, j].cpu().numpy()
        assert np.all(np.abs(got - want) <= 3.5e-5 * bound), (i, j)
    lat.close()


def test_nucleon_blocks_120_modes_24cube_symmetries():
    """Properties the definition fixes at any size, on the whole 120^3 x 4 output of one 24^3 slice
    (pinned for the oracle in tests/test_oracle_nucleon.py): B[i][j] = B[j][i] (rows (i, j) and
    (j, i) come from different tiles of the kernel), and a colour rotation s(x) -> g(x) s(x) by a
    random SU(3) matrix per site leaves B unchanged.  The compared results differ by rounding only
    (the tensor-core and FP32-FMA kernels differ by 3e-6 of max |B| on this workload), so 3e-5 of
    max |B| is allowed; an index or sign slip moves entries by O(max |B|)."""
    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    s3 = 24 ** 3
    n = 120
    lat = lqcd.Lattice(dims, "open")
    rng = np.random.default_rng(23)
    s = (rng.standard_normal((n, s3, 4, 3)) + 1j * rng.standard_normal((n, s3, 4, 3))) / np.sqrt(2)
    g = inputs.random_su3(s3, 0.9, 29)                                  # one SU(3) matrix per site
    sg = np.einsum("xab,ixsb->ixsa", g, s)
    B = lat.nucleon_blocks(torch.from_numpy(s).cuda(), (4, 4), 4, 1)[0]
    Bg = lat.nucleon_blocks(torch.from_numpy(sg).cuda(), (4, 4), 4, 1)[0]
    scale = B.abs().max().item()
    assert (B - B.transpose(0, 1)).abs().max().item() <= 3e-5 * scale
    assert (B - Bg).abs().max().item() <= 3e-5 * scale
    assert (B - B.transpose(0, 2)).abs().max().item() > 1e-2 * scale   # not symmetric in (i, k)
    lat.close()
