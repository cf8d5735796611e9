"""The systems of factorized propagators split between processes (one GPU each).

A unit is one point-source column of one gauge field: u = 12 * field_index + column.
Its factorized propagator (Sec. 3) needs, in order,
  stage A   D_Gamma^{-1} eta and D_Gammabar^{-1} eta          (eqs. quark_prop_I, quark_prop_II)
            and the boundary source chi = D_dGamma* (D_Gammabar^{-1} eta)|_Gamma,
  stage B   -D_Gamma*^{-1} chi                                 (eq. quark_prop_II),
and its correction the full-lattice solve D^{-1} eta (eq. observable_factorization).
Stage B depends on stage A only through chi, a vector on one time slice (two with a
wrapping time boundary): L1 L2 L3 x 12 complex numbers per unit and slot.  So the plan
puts the Gamma side and the Gamma* side of a unit on different ranks and ships chi
between them, point to point; the full-lattice solves are spread over all ranks whole
(every rank holds the whole gauge field; no halo exchange).

For world = 1 everything runs on rank 0 and nothing is sent.  For world >= 2 the first
n_a = world // 2 ranks take stage A (unit u on rank u mod n_a), the others stage B
(unit u on rank n_a + u mod n_b), and the full solve of u runs on rank u mod world.

The compute is a `stages` object with four calls on lists of units (the GPU one is
LatticeStages below; the tests also drive the same plan with a CPU implementation):
  gamma_and_gbar(units) -> (fact on Gamma [n, ...], psi on Gammabar [n, ...])
  boundary(psi_gbar, units) -> chi [n, 2, L1 L2 L3, 4, 3]
  gamma_star(chi, units) -> fact on Gamma* [n, ...]
  full(units) -> D^{-1} eta [n, V, 4, 3]
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch


@dataclass
class Plan:
    world: int
    n_units: int

    @property
    def n_a(self) -> int:
        return 1 if self.world == 1 else self.world // 2

    @property
    def n_b(self) -> int:
        return 1 if self.world == 1 else self.world - self.n_a

    def a_rank(self, u: int) -> int:
        return u % self.n_a

    def b_rank(self, u: int) -> int:
        return 0 if self.world == 1 else self.n_a + u % self.n_b

    def c_rank(self, u: int) -> int:
        return u % self.world

    def units(self, rank: int, stage: str) -> list[int]:
        f = {"a": self.a_rank, "b": self.b_rank, "c": self.c_rank}[stage]
        return [u for u in range(self.n_units) if f(u) == rank]


@dataclass
class RankResult:
    """What one rank computed: per unit, fact on Gamma, fact on Gamma*, the full solve."""

    gamma: dict = field(default_factory=dict)
    gamma_star: dict = field(default_factory=dict)
    full: dict = field(default_factory=dict)
    sent: list = field(default_factory=list)  # (unit, src, dst, bytes) of every chi shipped


def run(stages, plan: Plan, rank: int, dist=None, with_full: bool = True) -> RankResult:
    """This rank's share of the plan: stage A, the chi exchange, stage B, the full solves."""
    res = RankResult()
    ua = plan.units(rank, "a")
    ub = plan.units(rank, "b")
    chi_local = {}
    if ua:
        fact_g, psi_gb = stages.gamma_and_gbar(ua)
        chi = stages.boundary(psi_gb, ua)
        for i, u in enumerate(ua):
            res.gamma[u] = fact_g[i]
            chi_local[u] = chi[i].contiguous()
    # point-to-point hand-off of chi from the Gamma-side rank to the Gamma*-side rank; both
    # sides walk the units in increasing order, so the messages of a rank pair match in order
    reqs, recv = [], {}
    if plan.world > 1:
        for u in ua:
            dst = plan.b_rank(u)
            reqs.append(dist.isend(chi_local[u], dst=dst))
            res.sent.append((u, rank, dst, chi_local[u].numel() * chi_local[u].element_size()))
        for u in ub:
            buf = torch.empty(stages.chi_shape, dtype=torch.complex128, device=stages.device)
            reqs.append(dist.irecv(buf, src=plan.a_rank(u)))
            recv[u] = buf
        for r in reqs:
            r.wait()
    else:
        recv = chi_local
    if ub:
        chi_b = torch.stack([recv[u] for u in ub])
        fact_gs = stages.gamma_star(chi_b, ub)
        for i, u in enumerate(ub):
            res.gamma_star[u] = fact_gs[i]
    if with_full:
        uc = plan.units(rank, "c")
        if uc:
            full = stages.full(uc)
            for i, u in enumerate(uc):
                res.full[u] = full[i]
    return res


def assemble(results, plan: Plan, stages):
    """fact [n_units, V, 4, 3] and full (or None) from the ranks' results (rank 0 after a gather)."""
    n = plan.n_units
    V = stages.V
    fact = torch.zeros((n, V, 4, 3), dtype=torch.complex128)
    full = torch.zeros((n, V, 4, 3), dtype=torch.complex128) if any(r.full for r in results) else None
    g0, g1 = stages.gamma_sites
    s0, s1 = stages.gamma_star_sites
    for r in results:
        for u, v in r.gamma.items():
            fact[u, g0:g1] = v.cpu()
        for u, v in r.gamma_star.items():
            fact[u, s0:s1] = v.cpu()
        if full is not None:
            for u, v in r.full.items():
                full[u] = v.cpu()
    return fact, full


class LatticeStages:
    """The stages of the plan on this process's GPU through the C ABI (lqcd.Lattice): point-source
    solves on Gamma and Gammabar (lqcd_point_propagators), chi (lqcd_schur_boundary), the Gamma*
    solves (lqcd_schur_solve) and the full-lattice solves.  Unit u is column u % 12 of the loaded
    field field_ids[u // 12]."""

    def __init__(self, lat, gamma, gamma_star, x_src, field_ids, delta=None, params=None):
        self.lat = lat
        self.G, self.GS, self.delta = tuple(gamma), tuple(gamma_star), delta
        self.gbar = (0, delta[1] if delta is not None and delta[1] >= delta[0] else gamma[1])
        self.x_src = tuple(x_src)
        self.field_ids = list(field_ids)
        self.params = params
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.chi_shape = (2, lat.S3, 4, 3)
        self.V = lat.V
        self.gamma_sites = (gamma[0] * lat.S3, (gamma[1] + 1) * lat.S3)
        self.gamma_star_sites = (gamma_star[0] * lat.S3, (gamma_star[1] + 1) * lat.S3)

    def _fields(self, units):
        return [self.field_ids[u // 12] for u in units]

    def _points(self, units, dom):
        n = len(units)
        sol, _ = self.lat.point_propagators([dom] * n, self._fields(units), [self.x_src] * n,
                                            [u % 12 for u in units], self.params)
        return sol.view(n, -1, 4, 3)

    def gamma_and_gbar(self, units):
        return self._points(units, self.G), self._points(units, self.gbar)

    def boundary(self, psi_gbar, units):
        return self.lat.schur_boundary(psi_gbar.contiguous(), self.G, self.GS, self._fields(units), self.delta)

    def gamma_star(self, chi, units):
        out, _ = self.lat.schur_solve(chi, self.G, self.GS, self._fields(units), self.delta, self.params)
        return out

    def full(self, units):
        return self._points(units, (0, self.lat.T - 1))
