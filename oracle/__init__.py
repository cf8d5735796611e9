"""CPU oracle for the factorized quark propagator (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1612_06424_gb300``) and never imports it.

The arithmetic lives in ``oracle.c`` (plain FP64, natural layout, explicit
12x12 blocks); this module loads it with ctypes and composes the
factorization of Sec. 3 from its primitives, one step per term of the
equations:

  case I   (x, y in Gamma):       fact(y,x) = D_Gamma^{-1}(y,x)                    eq. quark_prop_I
  case II  (x in Gamma, y in Gamma*):
           fact(y,x) = -[D_Gamma*^{-1} D_dGamma* D_Gammabar^{-1}](y,x)             eq. quark_prop_II
  full     D^{-1}(y,x) on the whole lattice;  corr = full - fact                  eq. observable_factorization

and, independently, the exact correction of both cases through the Schur
complements of eq. block_inverse / schur_complement (``schur_correction``),
so that fact + corr = full can be checked without reusing ``full``.

Parity status of every function is pinned by tests/test_oracle_*.py.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_OPEN, BC_PERIODIC, BC_ANTIPERIODIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        c = ctypes.c_int
        d = ctypes.c_double
        _lib.ora_gamma.argtypes = [c, dp]
        _lib.ora_clover.argtypes = [ip, c, dp, d, d, dp]
        _lib.ora_dirac.argtypes = [ip, c, dp, dp, c, c, c, dp, dp]
        _lib.ora_solve.argtypes = [ip, c, dp, dp, c, c, c, dp, dp, d, c, ip, dp]
        _lib.ora_solve.restype = c
        _lib.ora_force.argtypes = [ip, c, dp, d, c, c, dp, dp, dp]
        _lib.ora_dirac_sites.argtypes = [ip, c, dp, d, d, c, c, ctypes.POINTER(ctypes.c_long), c, dp, dp]
    return _lib


def _dp(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def dirac_at_sites(dims, U, kappa: float, csw: float, bc: int, slab, sites, psi) -> np.ndarray:
    """(D_L psi)(x) at the natural site indices `sites` only, shape (len(sites), 4, 3).
    Builds no full-lattice clover array, so it serves very large lattices."""
    Uc = np.ascontiguousarray(U, dtype=np.complex128)
    ps = np.ascontiguousarray(psi, dtype=np.complex128)
    st = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.zeros((st.size, 4, 3), dtype=np.complex128)
    lib().ora_dirac_sites(_dims(dims), int(bc), _dp(Uc), float(kappa), float(csw), int(slab[0]), int(slab[1]),
                          st.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(st.size), _dp(ps), _dp(out))
    return out


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3, 0 = time) and gamma_5 (mu = 4), chiral basis."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().ora_gamma(mu, _dp(out))
    return out


class Operator:
    """The Wilson(-clover) operator D on one gauge field: D = 1/(2 kappa) - D_hop/2 + clover."""

    def __init__(self, dims, U: np.ndarray, kappa: float, csw: float = 0.0, bc: int = BC_OPEN):
        self.dims = tuple(int(v) for v in dims)
        self.V = int(np.prod(self.dims))
        self.bc = int(bc)
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.U = np.ascontiguousarray(U, dtype=np.complex128).reshape(self.V, 4, 3, 3)
        self.A = np.zeros((self.V, 12, 12), dtype=np.complex128)
        lib().ora_clover(_dims(self.dims), self.bc, _dp(self.U), self.kappa, self.csw, _dp(self.A))

    @property
    def T(self) -> int:
        return self.dims[0]

    def slab(self, t0: int, t1: int) -> np.ndarray:
        """Boolean site mask of the time slab t0..t1."""
        s3 = self.V // self.T
        t = np.arange(self.V) // s3
        return (t >= t0) & (t <= t1)

    def apply(self, psi: np.ndarray, t0: int = 0, t1: int | None = None, dagger: bool = False) -> np.ndarray:
        """D_L psi (or D_L^dag psi) for the slab L = t0..t1; psi shape (V,4,3)."""
        t1 = self.T - 1 if t1 is None else t1
        inp = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.V, 4, 3)
        out = np.empty_like(inp)
        lib().ora_dirac(_dims(self.dims), self.bc, _dp(self.U), _dp(self.A), int(t0), int(t1),
                        int(bool(dagger)), _dp(inp), _dp(out))
        return out

    def solve(self, b: np.ndarray, t0: int = 0, t1: int | None = None, dagger: bool = False,
              tol: float = 1e-13, maxit: int = 200000):
        """x = D_L^{-1} b to relative true residual tol; returns (x, iterations, residual)."""
        t1 = self.T - 1 if t1 is None else t1
        bb = np.ascontiguousarray(b, dtype=np.complex128).reshape(self.V, 4, 3)
        x = np.zeros_like(bb)
        its = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        rc = lib().ora_solve(_dims(self.dims), self.bc, _dp(self.U), _dp(self.A), int(t0), int(t1),
                             int(bool(dagger)), _dp(bb), _dp(x), float(tol), int(maxit),
                             ctypes.byref(its), ctypes.byref(res))
        if rc != 0:
            raise RuntimeError(f"oracle solve did not converge: residual {res.value:.3e} after {its.value}")
        return x, its.value, res.value

    def force(self, X: np.ndarray, Y: np.ndarray, t0: int = 0, t1: int | None = None) -> np.ndarray:
        """F[V,4,8] = -2 Re <Y, dD_L/domega^a_mu(x) X> for U_mu(x) -> exp(i omega T_a) U_mu(x)."""
        t1 = self.T - 1 if t1 is None else t1
        F = np.zeros((self.V, 4, 8), dtype=np.float64)
        Xc = np.ascontiguousarray(X, dtype=np.complex128)
        Yc = np.ascontiguousarray(Y, dtype=np.complex128)
        lib().ora_force(_dims(self.dims), self.bc, _dp(self.U), self.csw, int(t0), int(t1),
                        _dp(Xc), _dp(Yc), _dp(F))
        return F

    def masked(self, psi: np.ndarray, t0: int, t1: int) -> np.ndarray:
        out = np.array(psi, dtype=np.complex128, copy=True).reshape(self.V, 4, 3)
        out[~self.slab(t0, t1)] = 0
        return out

    def boundary_hop(self, psi: np.ndarray, src: tuple, dst: tuple) -> np.ndarray:
        """D_dst,src psi = P_dst D P_src psi: the off-diagonal block of eq. block_inverse."""
        return self.masked(self.apply(self.masked(psi, *src)), *dst)


@dataclass
class Split:
    """Two-region decomposition of Sec. 2.1 / 3: Gamma, its overlap DeltaGamma (subset of
    Gamma*, may be None) and Gamma*, each an inclusive time slab.  Gammabar = Gamma u DeltaGamma."""

    gamma: tuple
    gamma_star: tuple
    delta: tuple | None = None

    @property
    def gamma_bar(self) -> tuple:
        return (self.gamma[0], self.delta[1] if self.delta else self.gamma[1])


def factorized_propagator(op: Operator, split: Split, eta: np.ndarray, tol: float = 1e-13):
    """fact[col] for the sources eta[col] (supported in Gamma), following Sec. 3:
    D_Gamma^{-1} eta on Gamma (eq. quark_prop_I, first term) and
    -D_Gamma*^{-1} D_dGamma* (D_Gammabar^{-1} eta)|_Gamma on Gamma* (eq. quark_prop_II)."""
    g, gs, gb = split.gamma, split.gamma_star, split.gamma_bar
    fact = np.zeros_like(eta)
    for c in range(eta.shape[0]):
        psi_g, _, _ = op.solve(eta[c], *g, tol=tol)
        psi_gb, _, _ = op.solve(eta[c], *gb, tol=tol)
        chi = op.boundary_hop(psi_gb, g, gs)
        zeta, _, _ = op.solve(chi, *gs, tol=tol)
        m_g = op.slab(*g)
        m_gs = op.slab(*gs)
        fact[c][m_g] = psi_g[m_g]
        fact[c][m_gs] = -zeta[m_gs]
    return fact


def full_propagator(op: Operator, eta: np.ndarray, tol: float = 1e-13):
    """D^{-1} eta[col] on the whole lattice (the correction solve of Sec. 3.2)."""
    return np.stack([op.solve(eta[c], tol=tol)[0] for c in range(eta.shape[0])])


def schur_correction(op: Operator, split: Split, eta: np.ndarray, tol: float = 1e-13):
    """corr computed from the exact block inverse, eqs. block_inverse / schur_complement:
    y in Gamma:  D_Gamma^{-1} D_dGamma [S_Gamma*^{-1} (D_dGamma* D_Gamma^{-1} eta)]
                 with S_Gamma*^{-1} = (D^{-1})_{Gamma* Gamma*}          (eq. quark_prop_I)
    y in Gamma*: D_Gamma*^{-1} D_dGamma* [(D_Gammabar^{-1} eta) - (D^{-1} eta)]|_Gamma
                 with S_Gamma^{-1} eta = (D^{-1} eta)|_Gamma               (eq. quark_prop_II)."""
    g, gs, gb = split.gamma, split.gamma_star, split.gamma_bar
    corr = np.zeros_like(eta)
    m_g, m_gs = op.slab(*g), op.slab(*gs)
    for c in range(eta.shape[0]):
        psi_g, _, _ = op.solve(eta[c], *g, tol=tol)
        w = op.boundary_hop(psi_g, g, gs)                    # D_dGamma* D_Gamma^{-1} eta
        w_full, _, _ = op.solve(w, tol=tol)                  # D^{-1} w
        w_gs = op.masked(w_full, *gs)                        # S_Gamma*^{-1} w  (w lives on Gamma*)
        u = op.boundary_hop(w_gs, gs, g)                     # D_dGamma (...)
        corr_g, _, _ = op.solve(u, *g, tol=tol)
        psi_gb, _, _ = op.solve(eta[c], *gb, tol=tol)
        full_c, _, _ = op.solve(eta[c], tol=tol)
        diff = op.masked(psi_gb - full_c, *g)
        v = op.boundary_hop(diff, g, gs)
        corr_gs, _, _ = op.solve(v, *gs, tol=tol)
        corr[c][m_g] = corr_g[m_g]
        corr[c][m_gs] = corr_gs[m_gs]
    return corr


def link_force(op: Operator, phi: np.ndarray, t0: int, t1: int, tol: float = 1e-13):
    """Force of S = phi^dag (D_L^dag D_L)^{-1} phi on every link, with
    Y = D_L^{-dag} phi and X = D_L^{-1} Y, so X = (D_L^dag D_L)^{-1} phi and D_L X = Y.
    Returns (F[V,4,8], S, X, Y)."""
    phi_m = op.masked(phi, t0, t1)
    Y, _, _ = op.solve(phi_m, t0, t1, dagger=True, tol=tol)
    X, _, _ = op.solve(Y, t0, t1, dagger=False, tol=tol)
    S = float(np.real(np.vdot(phi_m, X)))
    return op.force(X, Y, t0, t1), S, X, Y


def disconnected_contract(op: Operator, etas: np.ndarray, psis: np.ndarray, t0: int, t1: int,
                          hops: int = 8) -> np.ndarray:
    """The contraction half of eq. stochastic_estimator (Sec. 5), given the solutions
    psi_i = D_L^{-1} gamma_5 eta_i on the slab L = t0..t1 (plain Wilson operator):
        t(x0) = (1/n_src) sum_i sum_{x in slice x0} eta_i^dag(x) [(kappa D_hop)^hops psi_i](x),
    kappa D_hop psi = psi - 2 kappa D_L psi (since 2 kappa D = 1 - kappa D_hop).
    etas, psis: (n_src, V, 4, 3).  Returns complex (T,), zero outside the slab.
    `hops` exists only so that a test can plant a wrong power."""
    if op.csw != 0.0:
        raise ValueError("the (kappa D_hop)^8 subtraction of eq. stochastic_estimator is for the Wilson operator")
    s3 = op.V // op.T
    out = np.zeros(op.T, dtype=np.complex128)
    for eta, psi in zip(etas, psis):
        e = op.masked(eta, t0, t1)
        y = op.masked(psi, t0, t1)
        for _ in range(hops):
            y = y - 2 * op.kappa * op.apply(y, t0, t1)
        prod = np.sum(np.conj(e) * y, axis=(1, 2))
        out += prod.reshape(op.T, s3).sum(axis=1)
    return out / len(etas)


def disconnected_trace(op: Operator, etas: np.ndarray, t0: int, t1: int, tol: float = 1e-13,
                       hops: int = 8) -> np.ndarray:
    """Stochastic estimate of sum_x tr{gamma_5 D_L^{-1}(x,x)} per time slice x0 of the
    slab L = t0..t1 (Sec. 5, eq. stochastic_estimator), plain Wilson operator:
        t(x0) = (1/n_src) sum_i sum_{x in slice x0} eta_i^dag(x) [(kappa D_hop)^8 D_L^{-1} gamma_5 eta_i](x).
    etas: (n_src, V, 4, 3) sources (only their slab part is used).  Returns complex (T,) with
    zeros outside the slab."""
    if op.csw != 0.0:
        raise ValueError("the (kappa D_hop)^8 subtraction of eq. stochastic_estimator is for the Wilson operator")
    g5 = gamma(4)
    psis = []
    for eta in etas:
        e = op.masked(eta, t0, t1)
        psi, _, _ = op.solve(np.einsum("st,xtc->xsc", g5, e), t0, t1, tol=tol)
        psis.append(psi)
    return disconnected_contract(op, etas, np.asarray(psis), t0, t1, hops=hops)


# --------------------------------------------------------------------------
# Quark-line projection (Sec. 3.3 eqs. projection, quark_prop_II_proj; Sec. 6)

def orthonormalize(W: np.ndarray) -> np.ndarray:
    """The orthonormal factor Q of W = Q R (columns of W (n, N) linearly independent), with R
    upper triangular and real positive on its diagonal, which makes Q unique: numpy's
    Householder QR, its column phases fixed."""
    Q, R = np.linalg.qr(W)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def spin_project_plus(v: np.ndarray) -> np.ndarray:
    """P_+ v = (1 + gamma_0)/2 v on the spin index (axis -2 of (..., 4, 3)): the half of a
    spinor on the last slice of Gamma that the boundary block D_dGamma* reads (its backward
    time hop carries (1 + gamma_0))."""
    return np.einsum("st,...tc->...sc", 0.5 * (np.eye(4) + gamma(0)), v)


def boundary_modes(op: Operator, v0: np.ndarray, t0: int, t1: int, g1: int, n_iter: int,
                   tol: float = 1e-13) -> np.ndarray:
    """N_m orthonormal projection vectors on the time slice g1 (the external boundary of Gamma*),
    from n_iter inverse iterations of D on the slab L = t0..t1 (Sec. 6): starting from the slab
    part of v0 (N_m, V, 4, 3), each iteration solves W_i = D_L^{-1} V_i for every column and
    orthonormalises, V = orthonormalize(W); the result is phi = orthonormalize(P_+ V|_{g1})
    (reading: the vectors live in the 6 L^3-dimensional space that D_dGamma* reads, Sec. 3.3).
    Returns phi (N_m, S3, 4, 3)."""
    s3 = op.V // op.T
    m = op.slab(t0, t1)
    n_m = v0.shape[0]
    Vc = np.stack([v0[i].reshape(op.V, 12)[m].reshape(-1) for i in range(n_m)], axis=1)
    for _ in range(n_iter):
        W = np.empty_like(Vc)
        for i in range(n_m):
            full = np.zeros((op.V, 12), dtype=np.complex128)
            full[m] = Vc[:, i].reshape(-1, 12)
            x, _, _ = op.solve(full.reshape(op.V, 4, 3), t0, t1, tol=tol)
            W[:, i] = x.reshape(op.V, 12)[m].reshape(-1)
        Vc = orthonormalize(W)
    lo = (g1 - t0) * s3
    sl = Vc.reshape(-1, 12, n_m)[lo:lo + s3]                     # (S3, 12, N_m)
    sl = np.moveaxis(sl, 2, 0).reshape(n_m, s3, 4, 3)
    P = spin_project_plus(sl).reshape(n_m, s3 * 12).T
    return orthonormalize(P).T.reshape(n_m, s3, 4, 3)


def _on_slice(op: Operator, v: np.ndarray, t: int) -> np.ndarray:
    """Place a slice vector (S3, 4, 3) on time slice t of a zero lattice vector."""
    s3 = op.V // op.T
    out = np.zeros((op.V, 4, 3), dtype=np.complex128)
    out[t * s3:(t + 1) * s3] = v
    return out


def projected_factors(op: Operator, split: Split, phis: np.ndarray, tol: float = 1e-13):
    """The two factors of eq. quark_prop_II_proj for projection vectors phi_i on the last slice
    of Gamma (phis (N_m, S3, 4, 3)):
        xi_i  = D_Gammabar^{-dag} phi_i, so that [phi_i^dag D_Gammabar^{-1}](x) = xi_i(x)^dag,
        eta_i = D_Gamma*^{-1} D_dGamma* phi_i.
    Returns (xi, eta), each (N_m, V, 4, 3)."""
    g, gs, gb = split.gamma, split.gamma_star, split.gamma_bar
    xi = np.zeros((phis.shape[0], op.V, 4, 3), dtype=np.complex128)
    eta = np.zeros_like(xi)
    for i, ph in enumerate(phis):
        p = _on_slice(op, ph, g[1])
        xi[i], _, _ = op.solve(p, *gb, dagger=True, tol=tol)
        eta[i], _, _ = op.solve(op.boundary_hop(p, g, gs), *gs, tol=tol)
    return xi, eta


def projected_propagator(op: Operator, split: Split, xi: np.ndarray, eta: np.ndarray, x_src) -> np.ndarray:
    """Case II of the factorized propagator with the quark line cut by P_L (eq. quark_prop_II_proj),
    12 point sources at x_src: for y in Gamma*,
        fact[b](y)[a] = -sum_i eta_i(y)[a] conj(xi_i(x)[b]),   b = 3 s0 + c0 the source column.
    Returns (12, V, 4, 3), zero outside Gamma*."""
    s3 = op.V // op.T
    L = op.dims
    x = ((x_src[0] * L[1] + x_src[1]) * L[2] + x_src[2]) * L[3] + x_src[3]
    m = op.slab(*split.gamma_star)
    E = eta.reshape(eta.shape[0], op.V, 12)
    Xx = xi.reshape(xi.shape[0], op.V, 12)[:, x, :]             # (N_m, 12): xi_i(x)[b]
    out = -np.einsum("iya,ib->bya", E, np.conj(Xx))
    out[:, ~m] = 0
    return out.reshape(12, op.V, 4, 3)


# --------------------------------------------------------------------------
# Nucleon blocks on projected quark lines (Sec. 4.2 eq. nucleon_prop_factorized)

def charge_conjugation() -> np.ndarray:
    """C = gamma_0 gamma_2 (real, antisymmetric, unitary, C gamma_mu C^{-1} = -gamma_mu^T in this basis)."""
    return gamma(0) @ gamma(2)


EPS3 = np.zeros((3, 3, 3))
EPS3[0, 1, 2] = EPS3[1, 2, 0] = EPS3[2, 0, 1] = 1.0
EPS3[0, 2, 1] = EPS3[2, 1, 0] = EPS3[1, 0, 2] = -1.0


def nucleon_block(op: Operator, s: np.ndarray, t: int) -> np.ndarray:
    """B[i, j, k, alpha] = sum over the sites x of time slice t of
        eps^{abc} {[s_i^T]^a(x) C gamma_5 [s_j]^b(x)} [s_k]^c_alpha(x)
    (the colourless spinor of eq. nucleon_prop_factorized), for the N fields s (N, V, 4, 3)."""
    s3 = op.V // op.T
    cg5 = charge_conjugation() @ gamma(4)
    f = s[:, t * s3:(t + 1) * s3]                                     # (N, S3, 4, 3)
    diq = np.einsum("abc,ixma,mn,jxnb->ijxc", EPS3, f, cg5, f)        # (N, N, S3, 3)
    return np.einsum("ijxc,kxdc->ijkd", diq, f)


def nucleon_factorized(op: Operator, xi: np.ndarray, eta: np.ndarray, x0: int, y0: int):
    """W1, W2 of eq. nucleon_prop_factorized summed over the sites of slices x0 (source, in Gammabar)
    and y0 (sink, in Gamma*):
        W1 = -sum_ijk B_xi[j, i, k](x0)^T g5 P_- B_eta[i, j, k](y0),
        W2 = -sum_ijk B_xi[k, i, j](x0)^T g5 P_- B_eta[i, j, k](y0),
    with the paper's row factor xi_i^T(x) = [phi_i^dag D_Gammabar^{-1}](x) = conj(xi_i(x)) (xi as
    returned by projected_factors), P_- = (1 - gamma_0)/2.  Returns (W1, W2); the factorized
    nucleon correlator is C_N^(f)(y0, x0) = (W1 - W2) / L^3."""
    g5pm = gamma(4) @ (0.5 * (np.eye(4) - gamma(0)))
    bx = nucleon_block(op, np.conj(xi), x0)
    be = nucleon_block(op, eta, y0)
    w1 = -np.einsum("jikg,gd,ijkd->", bx, g5pm, be)
    w2 = -np.einsum("kijg,gd,ijkd->", bx, g5pm, be)
    return w1, w2


def nucleon_point_correlator(S: np.ndarray, T: int) -> np.ndarray:
    """The two nucleon Wick contractions from a point source x to every sink y, summed over the
    sites of each time slice (Sec. 4.2, the contractions whose factorized form is eq.
    nucleon_prop_factorized), for the 12 propagator columns S[(3 nu + b), y, mu, a] = S(y, x)
    [(mu, a), (nu, b)] (sink spin-colour mu, a; source spin-colour nu, b):
        W1(t) = sum_{y in t} eps^{abc} eps^{a'b'c'} (Cg5)_{mu nu} (Cg5)_{mu' nu'} (g5 P_-)_{gam del}
                    S^{a b'}_{mu nu'} S^{b a'}_{nu mu'} S^{c c'}_{del gam}
        W2(t) = the same with S^{a b'}_{mu nu'} S^{b c'}_{nu gam} S^{c a'}_{del mu'}
    with C = gamma_0 gamma_2, P_- = (1 - gamma_0)/2.  Returns W[T, 2] (W1, W2); the correlator
    is W1 - W2.  Written as the definition, one einsum per slice."""
    n_col, V = S.shape[0], S.shape[1]
    assert n_col == 12
    s3 = V // T
    cg5 = charge_conjugation() @ gamma(4)
    g5pm = gamma(4) @ (0.5 * (np.eye(4) - gamma(0)))
    E = EPS3
    # P[y, mu, a, nu, b] = S(y, x)[(mu, a), (nu, b)]
    P = np.asarray(S).reshape(4, 3, V, 4, 3).transpose(2, 3, 4, 0, 1)
    out = np.zeros((T, 2), dtype=np.complex128)
    for t in range(T):
        Pt = P[t * s3:(t + 1) * s3]
        out[t, 0] = np.einsum("abc,ABC,mn,MN,gd,ymaNB,ynbMA,ydcgC->", E, E, cg5, cg5, g5pm, Pt, Pt, Pt,
                              optimize="optimal")
        out[t, 1] = np.einsum("abc,ABC,mn,MN,gd,ymaNB,ynbgC,ydcMA->", E, E, cg5, cg5, g5pm, Pt, Pt, Pt,
                              optimize="optimal")
    return out


def nucleon_hierarchy(op: Operator, gamma_: tuple, gamma_star: tuple, delta_ends, eta: np.ndarray,
                      tol: float = 1e-13):
    """Eq. nucleon_prop_hierarchical (Sec. 6) for the point source of the 12 columns eta:
    C^(i) is the nucleon correlator (W1 - W2 per time slice, nucleon_point_correlator) of the
    factorized propagator with overlap DeltaGamma_i = gamma_[1]+1 .. delta_ends[i] (nested,
    growing), C that of the full propagator, and the terms of the expansion are
        C^(0), C^(1) - C^(0), ..., C^(n-1) - C^(n-2), C^(rest) = C - C^(n-1),
    which sum to C.  Returns (terms [n+1, T] complex, C^(i) [n, T], C [T])."""
    T = op.T
    corr = []
    for d1 in delta_ends:
        split = Split(gamma_, gamma_star, delta=(gamma_[1] + 1, d1))
        w = nucleon_point_correlator(factorized_propagator(op, split, eta, tol=tol), T)
        corr.append(w[:, 0] - w[:, 1])
    w = nucleon_point_correlator(full_propagator(op, eta, tol=tol), T)
    c_full = w[:, 0] - w[:, 1]
    terms = [corr[0]] + [corr[i] - corr[i - 1] for i in range(1, len(corr))] + [c_full - corr[-1]]
    return np.array(terms), np.array(corr), c_full


def multilevel_estimator(o_gamma, o_gamma_star, o_corr, product=np.multiply):
    """Eq. multilevel_estimator (Sec. 2.2): for level-0 fields i and their level-1 fields j, k, l,
        (1/n0) sum_i { [(1/n1) sum_j O_Gamma[i,j]] . [(1/n1) sum_k O_Gamma*[i,k]] + (1/n1) sum_l O_corr[i,l] },
    with `.` the product that joins the two regions' factors (elementwise for scalars; a
    contraction for tensors).  Inputs indexed [i][j] (lists or arrays)."""
    n0 = len(o_gamma)
    total = None
    for i in range(n0):
        g = sum(o_gamma[i]) / len(o_gamma[i])
        gs = sum(o_gamma_star[i]) / len(o_gamma_star[i])
        c = sum(o_corr[i]) / len(o_corr[i])
        term = product(g, gs) + c
        total = term if total is None else total + term
    return total / n0
