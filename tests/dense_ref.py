"""Independent dense assembly of the Wilson(-clover) matrix for tiny lattices.

Test-only code, written separately from the oracle's stencil: the lattice is
handled as numpy arrays of shape (T, L1, L2, L3, ...), neighbours by np.roll,
clover leaves as rolled products of whole link arrays, and D as one dense
(12V x 12V) matrix.  Used as the brute-force pin of the oracle on 4^4.
"""
import numpy as np

G = np.zeros((5, 4, 4), dtype=np.complex128)
G[0, 0, 2] = G[0, 1, 3] = G[0, 2, 0] = G[0, 3, 1] = -1
_s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
for _k in range(3):
    G[_k + 1, :2, 2:] = -1j * _s[_k]
    G[_k + 1, 2:, :2] = 1j * _s[_k]
G[4] = np.diag([1, 1, -1, -1])


def sigma(mu, nu):
    return 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def clover_fhat(U, dims, bc_open):
    """Fhat[mu,nu] of shape (4,4,T,L1,L2,L3,3,3) from rolled link arrays."""
    T, L1, L2, L3 = dims
    u = U.reshape(T, L1, L2, L3, 4, 3, 3).copy()
    if bc_open:
        u[T - 1, :, :, :, 0] = 0
    F = np.zeros((4, 4, T, L1, L2, L3, 3, 3), dtype=np.complex128)
    sh = lambda a, mu, s: np.roll(a, -s, axis=mu)      # sh(a, mu, +1)(x) = a(x + mu)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Um, Un = u[..., mu, :, :], u[..., nu, :, :]
            # plaquette with lower-left corner at w: U_mu(w) U_nu(w+mu) U_mu(w+nu)^dag U_nu(w)^dag
            P = Um @ sh(Un, mu, 1) @ _dag(sh(Um, nu, 1)) @ _dag(Un)
            # transport each corner plaquette back to x (closed loops through x)
            l1 = P
            # corner x-mu: path x -> x+nu -> x+nu-mu -> x-mu -> x
            l2 = Un @ _dag(sh(sh(Um, nu, 1), mu, -1)) @ _dag(sh(Un, mu, -1)) @ sh(Um, mu, -1)
            l3 = _dag(sh(Um, mu, -1)) @ _dag(sh(sh(Un, mu, -1), nu, -1)) @ sh(sh(Um, mu, -1), nu, -1) @ sh(Un, nu, -1)
            l4 = _dag(sh(Un, nu, -1)) @ sh(Um, nu, -1) @ sh(sh(Un, nu, -1), mu, 1) @ _dag(Um)
            Q = l1 + l2 + l3 + l4
            F[mu, nu] = (Q - _dag(Q)) / 8.0
    return F


def dense_D(U, dims, kappa, csw=0.0, bc="open"):
    """Dense D = 1/(2 kappa) - D_hop/2 + c_sw (i/4) sum sigma Fhat as a (12V, 12V) matrix."""
    T, L1, L2, L3 = dims
    V = T * L1 * L2 * L3
    u = U.reshape(V, 4, 3, 3)
    M = np.zeros((V * 12, V * 12), dtype=np.complex128)
    I4 = np.eye(4)
    Fh = clover_fhat(U, dims, bc == "open").reshape(4, 4, V, 3, 3) if csw else None
    for x in range(V):
        c = [x // (L1 * L2 * L3), (x // (L2 * L3)) % L1, (x // L3) % L2, x % L3]
        blk = np.eye(12, dtype=np.complex128) / (2 * kappa)
        if csw:
            for mu in range(4):
                for nu in range(4):
                    if mu != nu:
                        blk += csw * 0.25j * np.kron(sigma(mu, nu), Fh[mu, nu, x])
        M[12 * x:12 * x + 12, 12 * x:12 * x + 12] += blk
        for mu in range(4):
            for step in (1, -1):
                y = list(c)
                y[mu] += step
                f = 1.0
                if not 0 <= y[mu] < dims[mu]:
                    y[mu] %= dims[mu]
                    if mu == 0:
                        f = {"open": 0.0, "periodic": 1.0, "antiperiodic": -1.0}[bc]
                if f == 0.0:
                    continue
                yi = ((y[0] * L1 + y[1]) * L2 + y[2]) * L3 + y[3]
                if step == 1:
                    b = np.kron(I4 - G[mu], u[x, mu])
                else:
                    b = np.kron(I4 + G[mu], _dag(u[yi, mu]))
                M[12 * x:12 * x + 12, 12 * yi:12 * yi + 12] += -0.5 * f * b
    return M


def slab_index(dims, t0, t1):
    s3 = dims[1] * dims[2] * dims[3]
    sites = np.arange(t0 * s3, (t1 + 1) * s3)
    return (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
