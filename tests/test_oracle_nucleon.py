"""Pins of the oracle's factorized nucleon contraction (Sec. 4.2 eq. nucleon_prop_factorized).

- C = gamma_0 gamma_2 is a charge-conjugation matrix of this basis: C gamma_mu C^{-1} = -gamma_mu^T;
- the block B is the eps/C-gamma_5 contraction written out site by site and index by index in plain
  loops on a tiny case;
- symmetries that the block's definition fixes, independent of how it is written: invariance under a
  colour rotation s(x) -> g(x) s(x) with g(x) in SU(3) (eps^{abc} g g g = det g eps), symmetry
  under i <-> j (eps and C g5 are both antisymmetric), and covariance under spin rotations
  s -> R s with R^T C g5 R = C g5 (R = exp(theta [g_mu, g_nu] / 4)): B -> R B in its spinor index;
- the factorized W1, W2 equal the propagator form of the two nucleon Wick contractions evaluated with
  the projected propagator S(y,x)[a,b] = -sum_i eta_i(y)[a] xi_i^T(x)[b] for every pair (x, y) of
  the two slices (substituting S into the contraction gives the block form, so any index slip in the
  blocks breaks the equality):
    W1 = sum eps^{abc} eps^{a'b'c'} (Cg5)_{mu nu} (Cg5)_{mu' nu'} (g5 P_-)_{gam del}
             S^{a b'}_{mu nu'} S^{b a'}_{nu mu'} S^{c c'}_{del gam}
    W2 = same with S^{a b'}_{mu nu'} S^{b c'}_{nu gam} S^{c a'}_{del mu'}.
"""
import itertools

import numpy as np

import oracle
from paper_1612_06424_gb300 import inputs

DIMS = (4, 2, 2, 2)
S3 = 8


def _op():
    U = inputs.random_su3_field(DIMS, 0.3, 41)
    return oracle.Operator(DIMS, U, 0.12, 0.0)


def test_charge_conjugation():
    C = oracle.charge_conjugation()
    for mu in range(4):
        g = oracle.gamma(mu)
        assert np.abs(C @ g @ np.linalg.inv(C) + g.T).max() < 1e-14
    assert np.abs(C.conj().T @ C - np.eye(4)).max() < 1e-14


def test_block_matches_explicit_loops():
    op = _op()
    rng = np.random.default_rng(3)
    n = 3
    s = rng.standard_normal((n, 32, 4, 3)) + 1j * rng.standard_normal((n, 32, 4, 3))
    B = oracle.nucleon_block(op, s, 2)
    cg5 = oracle.charge_conjugation() @ oracle.gamma(4)
    want = np.zeros((n, n, n, 4), complex)
    for i, j, k in itertools.product(range(n), repeat=3):
        for x in range(2 * S3, 3 * S3):
            for a, b, c in itertools.permutations(range(3)):
                e = oracle.EPS3[a, b, c]
                d = sum(s[i, x, m, a] * cg5[m, q] * s[j, x, q, b] for m in range(4) for q in range(4))
                want[i, j, k] += e * d * s[k, x, :, c]
    assert np.abs(B - want).max() < 1e-12 * np.abs(want).max()


def test_factorized_equals_propagator_form():
    op = _op()
    rng = np.random.default_rng(5)
    n = 4
    xi = rng.standard_normal((n, 32, 4, 3)) + 1j * rng.standard_normal((n, 32, 4, 3))
    eta = rng.standard_normal((n, 32, 4, 3)) + 1j * rng.standard_normal((n, 32, 4, 3))
    x0, y0 = 1, 3
    w1, w2 = oracle.nucleon_factorized(op, xi, eta, x0, y0)
    C = oracle.charge_conjugation()
    cg5 = C @ oracle.gamma(4)
    g5pm = oracle.gamma(4) @ (0.5 * (np.eye(4) - oracle.gamma(0)))
    E = oracle.EPS3
    r1 = r2 = 0.0
    for x in range(x0 * S3, (x0 + 1) * S3):
        for y in range(y0 * S3, (y0 + 1) * S3):
            # S[mu, a, nu, b] = -sum_i eta_i(y)[mu, a] conj(xi_i(x))[nu, b]
            S = -np.einsum("ima,inb->manb", eta[:, y], np.conj(xi[:, x]))
            r1 += np.einsum("abc,ABC,mn,MN,gd,maNB,nbMA,dcgC->", E, E, cg5, cg5, g5pm, S, S, S)
            r2 += np.einsum("abc,ABC,mn,MN,gd,maNB,nbgC,dcMA->", E, E, cg5, cg5, g5pm, S, S, S)
    assert abs(w1 - r1) < 1e-11 * abs(r1) and abs(r1) > 1e-6
    assert abs(w2 - r2) < 1e-11 * abs(r2) and abs(r2) > 1e-6
    assert abs(w1 - w2) > 1e-6 * abs(w1)        # the two contractions differ


def test_point_correlator_equals_block_form_on_a_projected_propagator():
    """With the projected propagator S(y,x) = -sum_i eta_i(y) xi_i^T(x) and one source site x, the
    point correlator (the two contractions written as definitions) equals the block form of eq.
    nucleon_prop_factorized with the source block taken at that single site."""
    op = _op()
    rng = np.random.default_rng(9)
    n = 4
    xi = rng.standard_normal((n, 32, 4, 3)) + 1j * rng.standard_normal((n, 32, 4, 3))
    eta = rng.standard_normal((n, 32, 4, 3)) + 1j * rng.standard_normal((n, 32, 4, 3))
    x = 1 * S3 + 5
    # S columns: S[(3 nu + b), y, mu, a] = -sum_i eta_i(y)[mu, a] conj(xi_i(x)[nu, b])
    S = -np.einsum("iyma,inb->nbyma", eta, np.conj(xi[:, x])).reshape(12, 32, 4, 3)
    W = oracle.nucleon_point_correlator(S, DIMS[0])
    xi_site = np.zeros_like(xi)  # xi at the source site only
    xi_site[:, x] = xi[:, x]
    for y0 in range(DIMS[0]):
        # the block form sums the source block over slice 1; xi_site vanishes there except at x
        w1, w2 = oracle.nucleon_factorized(op, xi_site, eta, 1, y0)
        assert abs(W[y0, 0] - w1) <= 1e-12 * max(1.0, abs(w1))
        assert abs(W[y0, 1] - w2) <= 1e-12 * max(1.0, abs(w2))
    assert np.abs(W).max() > 1e-3


def test_hierarchy_terms_telescope_and_shrink_with_the_overlap():
    """The terms of eq. nucleon_prop_hierarchical are formed in the printed order and sum to the
    full correlator; and on this field the factorized correlators on Gamma* approach the full
    one as the overlap DeltaGamma grows (the suppression with Delta that Sec. 6 reports)."""
    dims = (8, 2, 2, 2)
    U = inputs.random_su3_field(dims, 0.3, 43)
    op = oracle.Operator(dims, U, 0.12, 0.0)
    eta = inputs.point_sources(dims, (1, 0, 0, 0))
    terms, corr, full = oracle.nucleon_hierarchy(op, (0, 2), (3, 7), [4, 5, 6], eta)
    assert terms.shape == (4, 8)
    assert np.abs(terms.sum(axis=0) - full).max() <= 1e-13 * np.abs(full).max()
    assert np.abs(terms[1] - (corr[1] - corr[0])).max() == 0.0
    # the factorized correlators approach the full one as the overlap grows (Sec. 6 hierarchy)
    far = slice(3, 8)
    errs = [np.abs(c[far] - full[far]).max() for c in corr]
    assert errs[0] > errs[1] > errs[2]


def test_multilevel_estimator_special_cases():
    """n1 = 1 gives the plain estimator mean_i(O_G O_G* + O_corr); for a bilinear product the
    level-1 average equals the mean over all n1^2 (j, k) pairs (the exchange that makes the
    two-level average an n1^2 sample)."""
    rng = np.random.default_rng(8)
    n0, n1 = 3, 4
    og = rng.standard_normal((n0, 1))
    ogs = rng.standard_normal((n0, 1))
    oc = rng.standard_normal((n0, 1))
    assert abs(oracle.multilevel_estimator(og, ogs, oc) - np.mean(og[:, 0] * ogs[:, 0] + oc[:, 0])) < 1e-15
    A = rng.standard_normal((n0, n1, 3, 5))
    Bm = rng.standard_normal((n0, n1, 5))
    C = np.zeros((n0, n1, 3))
    prod = lambda a, b: a @ b
    got = oracle.multilevel_estimator(A, Bm, C, prod)
    want = np.mean([np.mean([A[i, j] @ Bm[i, k] for j in range(n1) for k in range(n1)], axis=0)
                    for i in range(n0)], axis=0)
    assert np.abs(got - want).max() < 1e-13


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 4 * S3, 4, 3)) + 1j * rng.standard_normal((n, 4 * S3, 4, 3))


def test_block_is_colour_gauge_invariant():
    """B(t) is a colour singlet: rotating the colour of every field at each site by the same SU(3)
    matrix g(x) (a different one per site) leaves it unchanged."""
    op = _op()
    s = _fields(3, 5)
    g = inputs.random_su3_field(DIMS, 0.9, 77)[:, 0]                  # one SU(3) matrix per site
    sg = np.einsum("xab,ixsb->ixsa", g, s)
    for t in range(DIMS[0]):
        B, Bg = oracle.nucleon_block(op, s, t), oracle.nucleon_block(op, sg, t)
        assert np.abs(Bg - B).max() < 1e-12 * np.abs(B).max()
    # a colour rotation that is not in SU(3) (det = e^{i phi}) multiplies B by det g
    ph = np.exp(0.7j)
    assert np.abs(oracle.nucleon_block(op, ph ** (1 / 3) * s, 1) - ph * oracle.nucleon_block(op, s, 1)).max() \
        < 1e-12 * np.abs(oracle.nucleon_block(op, s, 1)).max()


def test_block_is_symmetric_in_the_diquark_pair():
    op = _op()
    s = _fields(4, 6)
    for t in (0, 3):
        B = oracle.nucleon_block(op, s, t)
        assert np.abs(B - B.transpose(1, 0, 2, 3)).max() < 1e-12 * np.abs(B).max()
        assert np.abs(B - B.transpose(2, 1, 0, 3)).max() > 1e-3 * np.abs(B).max()   # not symmetric in (i, k)


def test_block_is_covariant_under_spin_rotations():
    from scipy.linalg import expm

    op = _op()
    s = _fields(3, 7)
    cg5 = oracle.charge_conjugation() @ oracle.gamma(4)
    for mu, nu, th in ((0, 1, 0.4), (1, 2, 1.1), (2, 3, -0.8)):
        G = oracle.gamma(mu) @ oracle.gamma(nu) - oracle.gamma(nu) @ oracle.gamma(mu)
        R = expm(0.25 * th * G)
        assert np.abs(R.T @ cg5 @ R - cg5).max() < 1e-13                 # R preserves the diquark form
        sr = np.einsum("st,ixtc->ixsc", R, s)
        B, Br = oracle.nucleon_block(op, s, 2), oracle.nucleon_block(op, sr, 2)
        assert np.abs(Br - np.einsum("st,ijkt->ijks", R, B)).max() < 1e-12 * np.abs(B).max()

