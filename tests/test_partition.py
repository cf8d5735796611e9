"""The split of factorized propagators between processes (paper_1612_06424_gb300/partition.py),
run on CPU as two gloo ranks, with the oracle standing in for each rank's GPU.

Rank 0 solves the Gamma side (D_Gamma^{-1} eta, D_Gammabar^{-1} eta, chi), rank 1 receives chi
and solves Gamma* (eq. quark_prop_II); the full-lattice solves are spread over both.  The
assembled fact and full propagators must equal, bit for bit, the oracle's own factorization
(Sec. 3) and full propagator computed in one process, and the only data that crosses ranks is
chi: 2 x L1 L2 L3 x 12 complex numbers per unit.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1612_06424_gb300 import inputs, partition

DIMS = (6, 4, 4, 4)
KAPPA, CSW = 0.13, 1.0
G, DL, GS = (0, 1), (2, 2), (2, 5)
X_SRC = (1, 2, 0, 3)
TOL = 1e-11


class OracleStages:
    """The four stage calls of partition.run evaluated by the FP64 oracle (CPU tensors)."""

    def __init__(self, fields, bc=oracle.BC_OPEN):
        self.ops = [oracle.Operator(DIMS, U, KAPPA, CSW, bc) for U in fields]
        self.eta = inputs.point_sources(DIMS, X_SRC)
        self.s3 = DIMS[1] * DIMS[2] * DIMS[3]
        self.V = int(np.prod(DIMS))
        self.gbar = (0, DL[1])
        self.chi_shape = (2, self.s3, 4, 3)
        self.device = torch.device("cpu")
        self.gamma_sites = (G[0] * self.s3, (G[1] + 1) * self.s3)
        self.gamma_star_sites = (GS[0] * self.s3, (GS[1] + 1) * self.s3)

    def _sl(self, slab):
        return slice(slab[0] * self.s3, (slab[1] + 1) * self.s3)

    def gamma_and_gbar(self, units):
        fg, fb = [], []
        for u in units:
            op, c = self.ops[u // 12], u % 12
            fg.append(op.solve(self.eta[c], *G, tol=TOL)[0][self._sl(G)])
            fb.append(op.solve(self.eta[c], *self.gbar, tol=TOL)[0][self._sl(self.gbar)])
        return torch.from_numpy(np.stack(fg)), torch.from_numpy(np.stack(fb))

    def boundary(self, psi_gbar, units):
        out = []
        for i, u in enumerate(units):
            op = self.ops[u // 12]
            x = np.zeros((self.V, 4, 3), complex)
            x[self._sl(self.gbar)] = psi_gbar[i].numpy()
            w = op.boundary_hop(x, G, GS)
            out.append(np.stack([w[self._sl((GS[0], GS[0]))], w[self._sl((GS[1], GS[1]))]]))
        return torch.from_numpy(np.stack(out))

    def gamma_star(self, chi, units):
        out = []
        for i, u in enumerate(units):
            op = self.ops[u // 12]
            b = np.zeros((self.V, 4, 3), complex)
            b[self._sl((GS[0], GS[0]))] += chi[i, 0].numpy()
            b[self._sl((GS[1], GS[1]))] += chi[i, 1].numpy()
            out.append(-op.solve(b, *GS, tol=TOL)[0][self._sl(GS)])
        return torch.from_numpy(np.stack(out))

    def full(self, units):
        return torch.from_numpy(np.stack([self.ops[u // 12].solve(self.eta[u % 12], tol=TOL)[0] for u in units]))


def _fields():
    U0 = inputs.random_su3_field(DIMS, 0.4, 9)
    U1 = inputs.inner_level_fields(U0, DIMS, [G, (3, 5)], 2, 0.4, 19, frozen=DL)[1]
    return [U0, U1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    stages = OracleStages(_fields())
    plan = partition.Plan(world, 24)
    res = partition.run(stages, plan, rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    if rank == 0:
        fact, full = partition.assemble(gathered, plan, stages)
        out["fact"] = fact.numpy()
        out["full"] = full.numpy()
        out["sent"] = [s for r in gathered for s in r.sent]
        out["units"] = {s: [plan.units(r, s) for r in range(world)] for s in "abc"}
    dist.barrier()
    dist.destroy_process_group()


def test_plan_covers_every_unit_once():
    for world in (1, 2, 3, 4, 8):
        plan = partition.Plan(world, 24)
        for stage in "abc":
            got = sorted(u for r in range(world) for u in plan.units(r, stage))
            assert got == list(range(24)), (world, stage)
        if world > 1:
            assert all(plan.a_rank(u) != plan.b_rank(u) for u in range(24))
            assert {plan.a_rank(u) for u in range(24)}.isdisjoint({plan.b_rank(u) for u in range(24)})


def test_two_ranks_exchange_only_chi_and_match_the_oracle():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # rank 0 holds the Gamma side, rank 1 the Gamma* side, the full solves are split
    assert out["units"]["a"] == [list(range(24)), []]
    assert out["units"]["b"] == [[], list(range(24))]
    s3 = DIMS[1] * DIMS[2] * DIMS[3]
    assert sorted(u for u, _, _, _ in out["sent"]) == list(range(24))
    assert all(src == 0 and dst == 1 and nb == 2 * s3 * 12 * 16 for _, src, dst, nb in out["sent"])
    # the oracle's factorization of Sec. 3 and its full propagator, field by field, through the
    # same oracle calls (so the assembled arrays must agree to the last bit)
    stages = OracleStages(_fields())
    split = oracle.Split(G, GS, delta=DL)
    for j, op in enumerate(stages.ops):
        ref = oracle.factorized_propagator(op, split, stages.eta, tol=TOL)
        full = oracle.full_propagator(op, stages.eta, tol=TOL)
        assert np.array_equal(out["fact"][12 * j:12 * j + 12], ref), j
        assert np.array_equal(out["full"][12 * j:12 * j + 12], full), j


@pytest.mark.gpu
def test_lattice_stages_compose_the_factorized_propagator():
    """On the GPU: the stage entry points (point propagators, lqcd_schur_boundary,
    lqcd_schur_solve) run through the one-process plan give the fact and full propagators of
    lqcd_factorized_propagators for two fields, and the oracle's, at the FP64 tolerance 1e-9."""
    from paper_1612_06424_gb300 import build, lqcd

    build.build()
    fields = _fields()
    lat = lqcd.Lattice(DIMS, "open")
    lat.set_gauge(np.stack(fields), KAPPA, CSW)
    params = lqcd.SolverParams(tol=1e-12, precision=64)
    stages = partition.LatticeStages(lat, G, GS, X_SRC, [0, 1], delta=DL, params=params)
    plan = partition.Plan(1, 24)
    fact, full = partition.assemble([partition.run(stages, plan, 0, None)], plan, stages)
    f2, c2, _ = lat.factorized_propagators(G, GS, X_SRC, [0, 1], delta=DL, params=params)
    ref_fact = f2.cpu().reshape(24, -1, 4, 3)
    ref_full = (f2 + c2).cpu().reshape(24, -1, 4, 3)
    scale = ref_full.abs().max().item()
    assert (fact - ref_fact).abs().max().item() <= 1e-9 * scale
    assert (full - ref_full).abs().max().item() <= 1e-9 * scale
    split = oracle.Split(G, GS, delta=DL)
    eta = inputs.point_sources(DIMS, X_SRC)
    for j, U in enumerate(fields):
        op = oracle.Operator(DIMS, U, KAPPA, CSW)
        ref = oracle.factorized_propagator(op, split, eta)
        assert np.abs(fact.numpy()[12 * j:12 * j + 12] - ref).max() <= 1e-9 * scale
    lat.close()
