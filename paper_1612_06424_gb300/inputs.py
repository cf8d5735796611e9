"""Seeded synthetic inputs: gauge fields, gauge transformations and sources.

This module draws random numbers and shapes them into the inputs both the
CUDA path and the CPU oracle consume.  It holds none of the arithmetic of the
method (no Dirac operator, no solver, no factorization): the same arrays are
handed to both sides.

Layouts (natural site order, time slowest):
  site index  i = ((x0*L1 + x1)*L2 + x2)*L3 + x3,   dims = (T, L1, L2, L3)
  gauge field U[i, mu, a, b]  complex128, mu = 0 is time (the paper's x0)
  spinor      psi[i, s, c]    complex128, spin s = 0..3, colour c = 0..2
  propagator  S[col, i, s, c] with source column col = 3*s0 + c0

Field law (stand-in for the paper's quenched ensembles, Sec. 5): every link
is U = exp(i*eps*H), H = sum_a h_a * lambda_a / 2 with h_a ~ N(0, 1) and
lambda_a the Gell-Mann matrices, then re-unitarised so that the third row is
exactly conj(row0 x row1).  Random numbers come from numpy's Philox
bit generator keyed by (seed, stream), so every draw is reproducible.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_su3",
    "random_su3_field",
    "random_su3_field_device",
    "inner_level_fields_device",
    "unit_field",
    "random_gauge_transform",
    "point_sources",
    "gaussian_spinor",
    "inner_level_fields",
    "slab_sites",
]


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF,
                                                     int(stream) & 0xFFFFFFFFFFFFFFFF]))


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1] = -1j
    l[1, 1, 0] = 1j
    l[2, 0, 0] = 1
    l[2, 1, 1] = -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2] = -1j
    l[4, 2, 0] = 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2] = -1j
    l[6, 2, 1] = 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): exact SU(3)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(n: int, eps: float, seed: int, stream: int = 0) -> np.ndarray:
    """n random SU(3) matrices exp(i*eps*H), H traceless Hermitian Gaussian."""
    rng = _rng(seed, stream)
    h = rng.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, gell_mann() / 2)
    w, v = np.linalg.eigh(H)
    u = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), np.conj(v))
    return _reunitarise(u)


def random_su3_field(dims, eps: float, seed: int, stream: int = 0,
                     chunk: int = 1 << 21) -> np.ndarray:
    """Gauge field U[V, 4, 3, 3] of independent exp(i*eps*H) links."""
    V = int(np.prod(dims))
    n = 4 * V
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for k, lo in enumerate(range(0, n, chunk)):
        hi = min(n, lo + chunk)
        out[lo:hi] = random_su3(hi - lo, eps, seed, stream * 65536 + k)
    return out.reshape(V, 4, 3, 3)


def _normals(n: int, seed: int, stream: int, device, rng: str):
    """(n, 8) standard normals as a float64 tensor on `device`: numpy's Philox keyed by
    (seed, stream) drawn on the host (rng="host", the draws of the numpy path), or torch's
    generator on the device seeded from (seed, stream) (rng="device": the same law, other
    draws, for large lattices where host draws dominate the set-up time)."""
    import torch

    if rng == "host":
        return torch.from_numpy(_rng(seed, stream).standard_normal((n, 8))).to(device)
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 0x9E3779B1 + int(stream) * 0x85EBCA77) & 0x7FFFFFFFFFFFFFFF)
    return torch.randn((n, 8), dtype=torch.float64, device=device, generator=g)


def _su3_torch(h, eps: float, torch_device):
    """exp(i eps H) for H = sum_a h_a lambda_a / 2 (h: numpy or torch (n, 8)), computed on a
    torch device, then re-unitarised; returns a complex128 tensor (n, 3, 3) on that device."""
    import torch

    lam = torch.from_numpy(gell_mann() / 2).to(torch_device)
    ht = (h if isinstance(h, torch.Tensor) else torch.from_numpy(h)).to(torch_device).to(torch.complex128)
    H = torch.einsum("na,aij->nij", ht, lam)
    u = torch.linalg.matrix_exp(1j * eps * H)
    r0 = u[:, 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = u[:, 1, :]
    r1 = r1 - torch.sum(torch.conj(r0) * r1, dim=-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.conj(torch.linalg.cross(r0, r1, dim=-1))
    return torch.stack([r0, r1, r2], dim=-2)


def random_su3_field_device(dims, eps: float, seed: int, device="cuda", stream: int = 0, chunk: int = 1 << 22,
                            rng: str = "host"):
    """The field law of random_su3_field (rng="host": the same Philox draws) with the matrix
    exponential done by torch on `device`; returns a complex128 tensor [V, 4, 3, 3] there.
    For large lattices, where the numpy path is slow."""
    import torch

    V = int(np.prod(dims))
    n = 4 * V
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for k, lo in enumerate(range(0, n, chunk)):
        hi = min(n, lo + chunk)
        out[lo:hi] = _su3_torch(_normals(hi - lo, seed, stream * 65536 + k, out.device, rng), eps, out.device)
    return out.reshape(V, 4, 3, 3)


def inner_level_fields_device(U0, dims, slabs, n_fields: int, eps: float, seed: int, frozen=None,
                              chunk: int = 1 << 22, field_ids=None, rng: str = "host"):
    """inner_level_fields with the redrawn links exponentiated by torch on U0's device (rng as in
    random_su3_field_device).  U0: complex128 tensor [V, 4, 3, 3]; returns [n, V, 4, 3, 3] on the
    same device for the fields field_ids (default: all n_fields)."""
    import torch

    T = dims[0]
    s3 = int(dims[1] * dims[2] * dims[3])
    V = T * s3
    t_of_site = np.arange(V) // s3
    ids = list(range(n_fields)) if field_ids is None else list(field_ids)
    out = U0.unsqueeze(0).repeat(len(ids), 1, 1, 1, 1)
    for d, (t0, t1) in enumerate(slabs):
        in_slab = (t_of_site >= t0) & (t_of_site <= t1)
        own = np.repeat(in_slab[:, None], 4, axis=1)
        own[:, 0] &= t_of_site != t1
        if frozen is not None:
            f0, f1 = frozen
            start_frozen = (t_of_site >= f0) & (t_of_site <= f1)
            end_t = np.minimum(t_of_site + 1, T - 1)
            end_frozen_t = (end_t >= f0) & (end_t <= f1)
            own &= ~start_frozen[:, None]
            own[:, 0] &= ~end_frozen_t
        idx = np.nonzero(own.reshape(-1))[0]
        idx_t = torch.from_numpy(idx).to(U0.device)
        for q, j in enumerate(ids):
            flat = out[q].reshape(-1, 3, 3)
            if rng == "host":
                gen = _rng(seed, (d + 1) * 4096 + j)
            for k, lo in enumerate(range(0, idx.size, chunk)):
                hi = min(idx.size, lo + chunk)
                if rng == "host":
                    h = gen.standard_normal((hi - lo, 8))
                else:
                    h = _normals(hi - lo, seed, ((d + 1) * 4096 + j) * 65536 + k, U0.device, rng)
                flat[idx_t[lo:hi]] = _su3_torch(h, eps, U0.device)
    return out


def unit_field(dims) -> np.ndarray:
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def random_gauge_transform(dims, seed: int, eps: float = 2.0) -> np.ndarray:
    """One random SU(3) matrix g(x) per site, shape (V, 3, 3)."""
    V = int(np.prod(dims))
    return random_su3(V, eps, seed, stream=0x6A)


def point_sources(dims, x_src) -> np.ndarray:
    """The 12 spin-colour point sources eta_col(y) = delta_{y,x} delta_{s,s0} delta_{c,c0}."""
    T, L1, L2, L3 = dims
    V = T * L1 * L2 * L3
    i = ((x_src[0] * L1 + x_src[1]) * L2 + x_src[2]) * L3 + x_src[3]
    eta = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            eta[3 * s + c, i, s, c] = 1.0
    return eta


def gaussian_spinor(dims, seed: int, n: int = 1, stream: int = 0) -> np.ndarray:
    """n complex Gaussian spinor fields, Re and Im ~ N(0, 1/2), shape (n, V, 4, 3)."""
    V = int(np.prod(dims))
    rng = _rng(seed, 0x5EED + stream)
    z = rng.standard_normal((n, V, 4, 3, 2)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def gaussian_spinor_device(dims, seed: int, n: int = 1, device="cuda"):
    """n complex Gaussian spinor fields with the law of gaussian_spinor (Re, Im ~ N(0, 1/2)),
    drawn by torch's seeded generator on `device` (different draws from the numpy path);
    complex128 tensor (n, V, 4, 3).  For many sources on large lattices."""
    import torch

    V = int(np.prod(dims))
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((n, V, 4, 3), dtype=torch.complex128, device=device)
    for i in range(n):
        out[i] = torch.randn((V, 4, 3), dtype=torch.complex128, device=device, generator=g)
    return out


def slab_sites(dims, t0: int, t1: int) -> slice:
    """Natural-order site range of the time slab t0..t1 (time is slowest)."""
    s3 = int(dims[1] * dims[2] * dims[3])
    return slice(t0 * s3, (t1 + 1) * s3)


def inner_level_fields(U0: np.ndarray, dims, slabs, n_fields: int, eps: float,
                       seed: int, frozen=None) -> np.ndarray:
    """Synthetic inner-level gauge fields (stand-in for level-1 updates).

    Field j equals the level-0 field U0 except that every link owned by a
    domain slab is redrawn from (seed, slab, j).  Ownership: a link whose
    start or end site lies in the frozen slab (if any) stays at level 0;
    otherwise a link belongs to the slab of its start site, except the
    forward temporal link leaving a slab, which stays at level 0.
    """
    T = dims[0]
    s3 = int(dims[1] * dims[2] * dims[3])
    V = T * s3
    t_of_site = np.arange(V) // s3
    out = np.repeat(U0[None], n_fields, axis=0)
    for d, (t0, t1) in enumerate(slabs):
        in_slab = (t_of_site >= t0) & (t_of_site <= t1)
        own = np.repeat(in_slab[:, None], 4, axis=1)
        own[:, 0] &= t_of_site != t1
        if frozen is not None:
            f0, f1 = frozen
            start_frozen = (t_of_site >= f0) & (t_of_site <= f1)
            end_t = np.minimum(t_of_site + 1, T - 1)
            end_frozen_t = (end_t >= f0) & (end_t <= f1)
            own &= ~start_frozen[:, None]
            own[:, 0] &= ~end_frozen_t
        idx = np.nonzero(own.reshape(-1))[0]
        for j in range(n_fields):
            new = random_su3(idx.size, eps, seed, stream=(d + 1) * 4096 + j)
            flat = out[j].reshape(-1, 3, 3)
            flat[idx] = new
    return out
