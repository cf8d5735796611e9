#!/usr/bin/env python
"""Benchmark of the factorized quark propagator on one GB300.

Metric: seconds per 12-source factorized propagator (factorized part of
Sec. 3 plus the full-lattice correction) at true FP64 residual 1e-10, and
the Wilson-clover Dslash's achieved HBM bandwidth against the measured peak.

Workload (one "step"): the 16^3x32 lattice, random SU(3) links
U = exp(i 0.4 H) (a stand-in for the paper's quenched ensembles), Wilson-clover
kappa = 0.1300, c_sw = 1.0, open time boundary; Gamma = t 0..13,
DeltaGamma = 14..17 (frozen), Gamma* = 14..31; 12 point sources at
x = (2,0,0,0).  A step loads the gauge field (even-odd packing, compression,
clover blocks and their inverses), solves the Gamma, Gammabar, Gamma* domain
systems and the full lattice for all 12 sources (batched), assembles
fact = D_Gamma^{-1} on Gamma and -D_Gamma*^{-1} D_dGamma* D_Gammabar^{-1} on
Gamma*, and corr = D^{-1} - fact.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 64|32|16]
  python bench.py --impl reference     # the CPU oracle on the host cores
  python bench.py --workload batched_32x64   # 8 slabs x 12 sources x 16 inner-level fields
  python bench.py --workload force_24x48     # domain pseudofermion link force, 4 domains
  python bench.py --workload factorized_48x96  # 8 inner-level fields x 12 sources, 48^3x96

Multi-GPU (torchrun): every rank computes its own propagators (its own
gauge field, independent problems); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WL = {
    "name": "16^3x32 Wilson-clover factorized propagator + correction",
    "dims": (32, 16, 16, 16),
    "kappa": 0.13,
    "csw": 1.0,
    "eps": 0.4,
    "gamma": (0, 13),
    "delta": (14, 17),
    "gamma_star": (14, 31),
    "x_src": (2, 0, 0, 0),
    "tol": 1e-10,
}
METRIC = "s per 12-source factorized propagator @ res 1e-10 (Dslash HBM GB/s vs peak in roofline)"
UNIT = "s/propagator"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[64, 32, 16])
    ap.add_argument("--no-fp64-form", action="store_true", help="skip timing the plain FP64 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="factorized_16x32",
                    choices=["factorized_16x32", "batched_32x64", "force_24x48", "factorized_48x96",
                             "disconnected_64x24", "projection_64x24"])
    ap.add_argument("--fields", type=int, default=8, help="inner-level fields of factorized_48x96")
    ap.add_argument("--sources", type=int, default=100, help="Gaussian sources of disconnected_64x24")
    ap.add_argument("--modes", type=int, default=120, help="projection vectors of projection_64x24")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _strip_comments(src: str) -> str:
    """C++ source without // comments and blank lines (a comment edit does not change the kernel)."""
    out = []
    for line in src.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code.strip():
            out.append(code)
    return "\n".join(out)


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("common.cuh", "dslash.cuh"):
        with open(os.path.join(ROOT, "paper_1612_06424_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic(precision):
    """Per-launch DRAM bytes of the hop kernel from the committed ncu summary,
    or None if absent or taken on a different kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "dslash_traffic.json")) as fh:
            t = json.load(fh)
        e = t.get(str(precision))
        if e and e.get("kernel_hash") == _kernel_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.p = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


_ORACLE_ITERS = {}


def _oracle_iterations(op):
    """Iterations the oracle's own BiCGStab needs on this workload to residual
    1e-10: one column solved on Gamma (t 0..13) to 1e-5, doubled (the residual
    falls geometrically), measured once per process (about 20 s)."""
    from paper_1612_06424_gb300 import inputs

    if "gamma" not in _ORACLE_ITERS:
        eta = inputs.point_sources(WL["dims"], WL["x_src"])[0]
        t0 = time.perf_counter()
        _, its, _ = op.solve(eta, *WL["gamma"], tol=1e-5)
        _ORACLE_ITERS["gamma"] = 2 * its
        _ORACLE_ITERS["seconds"] = time.perf_counter() - t0
    return _ORACLE_ITERS["gamma"]


def _cpu_baseline(U, sample_seconds=8.0):
    """The oracle (plain FP64 C, one thread) on the host cores, for one
    12-source factorized propagator with correction on the 16^3x32 workload,
    from a bounded sample: the time of one oracle D application on each solve
    domain (Gamma, Gammabar, Gamma*, full lattice), measured, times
    2 applications per BiCGStab iteration x the oracle's iteration count
    (measured on Gamma, one column, residual 1e-10) x 12 columns."""
    import oracle
    from paper_1612_06424_gb300 import inputs

    dims = WL["dims"]
    op = oracle.Operator(dims, U, WL["kappa"], WL["csw"])
    its = _oracle_iterations(op)
    psi = inputs.gaussian_spinor(dims, 99)[0]
    T = dims[0]
    groups = {"gamma": WL["gamma"], "gamma_bar": (0, WL["delta"][1]), "gamma_star": WL["gamma_star"], "full": (0, T - 1)}
    per = sample_seconds / len(groups)
    t_apply = {}
    for k, (a, b) in groups.items():
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < per or n < 2:
            op.apply(psi, a, b)
            n += 1
        t_apply[k] = (time.perf_counter() - t0) / n
    total = sum(12 * 2 * its * t for t in t_apply.values())
    return {"value": total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle D applications on each solve domain ({', '.join(f'{k} {v:.3f} s' for k, v in t_apply.items())}) "
                      f"x 2 x {its} oracle BiCGStab iterations to 1e-10 (twice those measured for one column on Gamma "
                      f"to 1e-5, {_ORACLE_ITERS.get('seconds', 0):.0f} s) x 12 columns; extrapolated"}


def run_reference(args):
    """--impl reference: the CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1612_06424_gb300 import inputs

    U = inputs.random_su3_field(WL["dims"], WL["eps"], 1)
    for _ in range(args.warmup):
        _cpu_baseline(U, sample_seconds=2.0)
    vals = [_cpu_baseline(U, sample_seconds=4.0) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WL["name"], "dims": list(WL["dims"]), "kappa": WL["kappa"], "c_sw": WL["csw"]},
        "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0}))


def _max_over_ranks(value, dist, device="cuda"):
    """The largest of the ranks' values (the job's time); the only collective of
    the multi-GPU path besides the barriers around the timed region."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def _rank_seed(rank):
    """Gauge-field seed of a rank: every rank solves its own, independent problem."""
    return 1 + rank


def run_batched(args):
    """32^3x64, kappa 0.1340, c_sw 1.0: 8 time-slab domains of 8 slices x 12 point
    sources (slab centre, spatial origin) x 16 inner-level fields (every slab's own
    links redrawn), 1536 domain systems in one batched call (waves by free memory),
    FP16 vectors with FP32 norm inside, FP64 defect correction to residual 1e-10."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dims = (64, 32, 32, 32)
    slabs = [(8 * d, 8 * d + 7) for d in range(8)]
    nf = 16
    t0 = time.time()
    U0 = inputs.random_su3_field_device(dims, 0.4, 3, device="cuda")
    Uf = inputs.inner_level_fields_device(U0, dims, slabs, nf, 0.4, 4)
    del U0
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(Uf, 0.134, 1.0)
    del Uf
    torch.cuda.empty_cache()
    t_gen = time.time() - t0
    doms, fields, xs, cols = [], [], [], []
    for j in range(nf):
        for d, (a, b) in enumerate(slabs):
            for c in range(12):
                doms.append((a, b)); fields.append(j); xs.append((a + 4, 0, 0, 0)); cols.append(c)
    n = len(doms)
    sol = torch.empty((n * lat.slab_len(0, 7), 4, 3), dtype=torch.complex128, device="cuda")
    params = lqcd.SolverParams(tol=1e-10, precision=args.precision)
    for _ in range(max(0, args.warmup)):
        lat.point_propagators(doms[:96], fields[:96], xs[:96], cols[:96], params)
    torch.cuda.synchronize()
    l0 = lqcd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks() as clk:
        e0.record()
        for _ in range(args.steps):
            _, st = lat.point_propagators(doms, fields, xs, cols, params, sol=sol)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (lqcd.kernel_launches() - l0) // max(1, args.steps)
    d_ms, d_bytes, d_flops = lat.dslash_bench(doms[:192], fields[:192], args.precision, 20)
    peak, peak_kind = _peaks()
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "s per 12-source domain propagator, batched (1536 systems) @ res 1e-10", "value": ms / 1e3 / (n / 12),
        "unit": "s/12-source domain propagator", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": "32^3x64 batched domain propagators", "dims": list(dims), "kappa": 0.134, "c_sw": 1.0,
                   "systems": n, "slabs": 8, "fields": nf, "sources": 12, "residual": 1e-10},
        "seconds_all_systems": ms / 1e3, "setup_s": t_gen,
        "iters_max": max(x["iters"] for x in st), "iters_mean": sum(x["iters"] for x in st) / n,
        "true_residual_max": max(x["true_residual"] for x in st),
        "status_bad": sum(1 for x in st if x["status"] != 0),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                     "kernel": f"k_hop_lin<{args.precision}> on 192 systems (16 slabs x 12 sources)",
                     "ms_per_launch": round(d_ms, 4)},
        "clocks": clk.summary(), "gpu_launches": int(launches)}))
    lat.close()


def run_force(args):
    """24^3x48, kappa 0.1320, c_sw 1.0: link force of phi^dag (D_L^dag D_L)^{-1} phi
    for 4 time-slab domains of 12 slices (Gaussian phi), FP64 and mixed solves."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (48, 24, 24, 24)
    doms = [(12 * d, 12 * d + 11) for d in range(4)]
    U = inputs.random_su3_field_device(dims, 0.4, 5, device="cuda")
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, 0.132, 1.0)
    phis = [torch.from_numpy(inputs.gaussian_spinor(dims, 50 + d)[0][inputs.slab_sites(dims, *dom)]).cuda()
            for d, dom in enumerate(doms)]
    out = {}
    for prec in (64, args.precision):
        params = lqcd.SolverParams(tol=1e-10, precision=prec)
        for _ in range(max(1, args.warmup)):
            lat.link_force(phis[0], doms[0], 0, params)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            for d, dom in enumerate(doms):
                F, S, st = lat.link_force(phis[d], dom, 0, params)
        e1.record()
        torch.cuda.synchronize()
        out[prec] = {"s_per_domain_force": e0.elapsed_time(e1) / 1e3 / (args.steps * len(doms)),
                     "iters": [x["iters"] for x in st], "true_residual": max(x["true_residual"] for x in st)}
    print(json.dumps({
        "metric": "s per domain link force (2 solves + force kernels) @ res 1e-10",
        "value": out[args.precision]["s_per_domain_force"], "unit": "s/force", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": "24^3x48 domain link force", "dims": list(dims), "kappa": 0.132, "c_sw": 1.0,
                   "domains": [list(d) for d in doms]},
        "fp64_form": out[64], "this_precision": out[args.precision]}))
    lat.close()


def run_factorized_48(args):
    """48^3x96, kappa 0.1350, c_sw 1.0: Gamma = t 0..43, frozen DeltaGamma = 44..51,
    Gamma* = 44..95; 12 point sources at (2,0,0,0) on each of `--fields` inner-level
    fields (the level-0 field with the links of Gamma and of t 52..95 redrawn; links
    starting or ending in the frozen slab kept), factorized propagator plus the
    full-lattice correction per field.  The fields run one after another (each
    packed field is 23 GB; fact + corr are 49 GB)."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (96, 48, 48, 48)
    G, DL, GS = (0, 43), (44, 51), (44, 95)
    lat = lqcd.Lattice(dims, "open")
    V = lat.V
    fact = torch.empty((12, V, 4, 3), dtype=torch.complex128, device="cuda")
    corr = torch.empty_like(fact)
    params = lqcd.SolverParams(tol=1e-10, precision=args.precision)
    t_fields, t_solve, stats = 0.0, 0.0, []
    U0 = inputs.random_su3_field_device(dims, 0.4, 7, device="cuda")
    with Clocks() as clk:
        for j in range(args.fields):
            t0 = time.time()
            Uj = inputs.inner_level_fields_device(U0, dims, [G, (52, 95)], args.fields, 0.4, 8, frozen=DL,
                                                  field_ids=[j])
            lat.set_gauge(Uj, 0.135, 1.0)
            del Uj
            torch.cuda.synchronize()
            t1 = time.time()
            _, _, st = lat.factorized_propagator(G, GS, (2, 0, 0, 0), delta=DL, corr=True, params=params,
                                                 out=(fact, corr))
            torch.cuda.synchronize()
            t_fields += t1 - t0
            t_solve += time.time() - t1
            stats.append(st)
    print(json.dumps({
        "metric": "s per 12-source factorized propagator + correction @ res 1e-10 (48^3x96)",
        "value": t_solve / args.fields, "unit": "s/propagator", "n_gpus": 1, "steps": args.fields, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": "48^3x96 factorized propagator, inner-level fields", "dims": list(dims), "kappa": 0.135,
                   "c_sw": 1.0, "gamma": list(G), "delta": list(DL), "gamma_star": list(GS), "fields": args.fields},
        "field_setup_s_per_field": t_fields / args.fields,
        "iters": [{k: v["iters"] for k, v in st.items()} for st in stats],
        "true_residual_max": max(v["true_residual"] for st in stats for v in st.values()),
        "clocks": clk.summary()}))
    lat.close()


def _oracle_disconnected_sample(U, dims, kappa, doms, iters, sample_seconds=12.0):
    """The oracle (plain FP64 C, one thread) on the host cores, for one source of the
    disconnected estimator, from a bounded sample: the measured time of one oracle D
    application on each slab, times (2 per BiCGStab iteration x the GPU solve's iteration
    count on that slab + 8 hops + 1 for the residual), summed over the slabs; extrapolated."""
    import oracle
    from paper_1612_06424_gb300 import inputs

    op = oracle.Operator(dims, U, kappa, 0.0)
    psi = inputs.gaussian_spinor(dims, 98)[0]
    per = sample_seconds / len(doms)
    total, parts = 0.0, []
    for (a, b), its in zip(doms, iters):
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < per or n < 2:
            op.apply(psi, a, b)
            n += 1
        t = (time.perf_counter() - t0) / n
        total += t * (2 * its + 9)
        parts.append(f"slab {a}..{b}: {t:.3f} s x (2 x {its} + 9)")
    return {"value": total, "unit": "s/source", "cores": 1, "kind": "oracle",
            "sample": "oracle D applications per slab (" + "; ".join(parts) + "), iteration counts of the GPU "
                      "solves; per source, extrapolated"}


def run_disconnected(args):
    """64x24^3 Wilson (c_sw = 0), kappa 0.1360, open time boundaries: the stochastic
    disconnected traces of Sec. 4.1 with `--sources` Gaussian sources (100 in the paper) on
    Gamma = t 0..32 and Gamma* = 33..63 (Dirichlet blocks) and on the full lattice, all
    solved together; eight (kappa D_hop) hops and per-slice contractions on the GPU."""
    import numpy as np
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    kappa = 0.136
    doms = [(0, 32), (33, 63), (0, 63)]
    U = inputs.random_su3_field_device(dims, 0.4, 21, device="cuda")
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, 0.0)
    del U
    eta = inputs.gaussian_spinor_device(dims, 22, args.sources, device="cuda")
    params = lqcd.SolverParams(tol=1e-10, precision=args.precision)
    for _ in range(max(1, args.warmup)):
        lat.disconnected_trace(eta[:4], doms, 0, params)
    torch.cuda.synchronize()
    n0 = lqcd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks() as clk:
        e0.record()
        for _ in range(args.steps):
            tr, mean, st = lat.disconnected_trace(eta, doms, 0, params)
        e1.record()
        torch.cuda.synchronize()
    launches = lqcd.kernel_launches() - n0
    sec = e0.elapsed_time(e1) / 1e3 / args.steps
    # roofline of the FP32 hop kernel on the same batch shape
    n_rf = min(args.sources, 24)
    ms, by, fl = lat.dslash_bench([d for _ in range(n_rf) for d in doms], [0] * (3 * n_rf), args.precision, 20)
    hbm, hbm_src = _peaks()
    mean_h = mean.cpu().numpy()
    out = {
        "metric": "s per Gaussian source of the disconnected estimator (Gamma, Gamma*, full) @ res 1e-10 (64x24^3)",
        "value": sec / args.sources, "unit": "s/source", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": "64x24^3 Wilson disconnected traces", "dims": list(dims), "kappa": kappa, "c_sw": 0.0,
                   "domains": [list(d) for d in doms], "sources": args.sources, "l2": "inputs larger than L2"},
        "iters": {n: s["iters"] for n, s in zip(["gamma", "gamma_star", "full"], st)},
        "true_residual_max": max(s["true_residual"] for s in st),
        "sum_over_slices": {n: [float(np.sum(mean_h[d]).real), float(np.sum(mean_h[d]).imag)]
                            for d, n in enumerate(["gamma", "gamma_star", "full"])},
        "roofline": {"bound": "hbm", "achieved": by / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": by / (ms * 1e-3) / 1e9 / hbm, "traffic": None, "peak_source": hbm_src,
                     "kernel": f"FP{args.precision} hop kernel, {3 * n_rf} systems of this workload's slabs"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        Uh = inputs.random_su3_field(dims, 0.4, 21)
        out["cpu_baseline"] = _oracle_disconnected_sample(Uh, dims, kappa, doms, [s["iters"] for s in st])
    print(json.dumps(out))
    lat.close()


def run_projection(args):
    """64x24^3 Wilson (c_sw = 0), kappa 0.1360, open time boundaries: the quark-line cut of
    Sec. 3.3 with the Sec. 5 setup for Delta = 8: Gammabar = t 0..31 (Gamma = 0..23,
    DeltaGamma = 24..31), Gamma* = 24..63; N_m = `--modes` (120 in the paper) projection
    vectors from 10 inverse iterations on t 16..31, cut on slice 23; the factors xi, eta
    (2 N_m solves) and the projected case-II propagator for 12 point sources at (4,0,0,0).
    Then the nucleon blocks of eq. nucleon_prop_factorized on the source slice 4 and the 40
    sink slices of Gamma*, and their two Wick contractions (reported separately; `value` is
    the projected propagator)."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    kappa = 0.136
    G, DL, GS = (0, 23), (24, 31), (24, 63)
    mdom, g1, n_iter = (16, 31), 23, 10
    n_m = args.modes
    U = inputs.random_su3_field_device(dims, 0.4, 31, device="cuda")
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, 0.0)
    del U
    v0 = inputs.gaussian_spinor_device(dims, 32, n_m, device="cuda")
    s3 = 24 ** 3
    v0 = v0[:, mdom[0] * s3:(mdom[1] + 1) * s3].contiguous()
    params = lqcd.SolverParams(tol=1e-10, precision=args.precision)
    # warm-up on a few modes and one iteration
    phi_w, _ = lat.boundary_modes(v0[:8], mdom, g1, 0, 1, params)
    lat.projected_factors(phi_w, G, GS, DL, 0, params)
    torch.cuda.synchronize()
    n0 = lqcd.kernel_launches()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    x0 = 4
    with Clocks() as clk:
        ev[0].record()
        phi, st_m = lat.boundary_modes(v0, mdom, g1, 0, n_iter, params)
        ev[1].record()
        xi, eta, st_f = lat.projected_factors(phi, G, GS, DL, 0, params)
        ev[2].record()
        fact = lat.projected_propagator(xi, eta, G, GS, (x0, 0, 0, 0), DL)
        ev[3].record()
        # nucleon blocks: source slice x0 from xi (conjugated), sink slices of Gamma* from eta
        Bx = lat.nucleon_blocks(xi, (0, DL[1]), x0, 1, conj=True)
        By = lat.nucleon_blocks(eta, GS, GS[0], GS[1] - GS[0] + 1)
        ev[4].record()
        W = lqcd.nucleon_contract(Bx, By)
        ev[5].record()
        torch.cuda.synchronize()
    launches = lqcd.kernel_launches() - n0
    t = [ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(5)]
    n_sl = 1 + GS[1] - GS[0] + 1
    block_flops = 8.0 * 12 * n_m ** 3 * s3 * n_sl                   # (x, c) contraction, complex FMA = 8 flop
    fp32_peak = lqcd.fma_peak(32)
    cn = (W[0, :, 0] - W[0, :, 1]).cpu() / s3
    out = {
        "metric": "s per projected quark line (N_m modes, 10 inverse iterations, factors, 12-source case-II "
                  "propagator) @ res 1e-10 (64x24^3)",
        "value": sum(t[:3]), "unit": "s/projected propagator", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": sum(t[:3]) * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": "64x24^3 Wilson quark-line projection, Delta = 8", "dims": list(dims), "kappa": kappa,
                   "c_sw": 0.0, "gamma": list(G), "delta": list(DL), "gamma_star": list(GS), "modes": n_m,
                   "mode_slab": list(mdom), "cut_slice": g1, "inverse_iterations": n_iter},
        "seconds": {"modes": t[0], "factors": t[1], "contraction": t[2], "nucleon_blocks": t[3],
                    "nucleon_contract": t[4]},
        "nucleon_blocks_roofline": {"bound": "alu", "achieved": block_flops / t[3] / 1e12, "peak": fp32_peak,
                                    "unit": "TFLOP/s", "frac": block_flops / t[3] / 1e12 / fp32_peak,
                                    "peak_source": "measured FP32 FMA (lqcd_fma_peak)",
                                    "kernel": f"k_nucleon_block, N_m = {n_m}, {n_sl} slices of {s3} sites"},
        "nucleon_cf_over_slices": [[float(v.real), float(v.imag)] for v in cn[:4]],
        "iters": {"modes_max": st_m["iters"], "gamma_bar": st_f["gamma_bar"]["iters"],
                  "gamma_star": st_f["gamma_star"]["iters"]},
        "true_residual_max": max(st_m["true_residual"], st_f["gamma_bar"]["true_residual"],
                                 st_f["gamma_star"]["true_residual"]),
        "fact_norm_gamma_star": float(torch.linalg.vector_norm(fact).item()),
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(out))
    lat.close()


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_32x64":
        return run_batched(args)
    if args.workload == "force_24x48":
        return run_force(args)
    if args.workload == "disconnected_64x24":
        return run_disconnected(args)
    if args.workload == "projection_64x24":
        return run_projection(args)
    if args.workload == "factorized_48x96":
        return run_factorized_48(args)
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = WL["dims"]
    U = inputs.random_su3_field(dims, WL["eps"], _rank_seed(rank))
    U_dev = torch.from_numpy(U).cuda()
    lat = lqcd.Lattice(dims, "open")
    V = lat.V
    fact = torch.empty((12, V, 4, 3), dtype=torch.complex128, device="cuda")
    corr = torch.empty_like(fact)

    def step(prec, U_src=None):
        lat.set_gauge(U_dev if U_src is None else U_src, WL["kappa"], WL["csw"])
        _, _, st = lat.factorized_propagator(WL["gamma"], WL["gamma_star"], WL["x_src"], delta=WL["delta"],
                                             corr=True, params=lqcd.SolverParams(tol=WL["tol"], precision=prec),
                                             out=(fact, corr))
        return st

    def timed(prec, K, W):
        for _ in range(W):
            step(prec)
        torch.cuda.synchronize()
        barrier()
        l0 = lqcd.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        stats = None
        for _ in range(K):
            stats = step(prec)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = _max_over_ranks(e0.elapsed_time(e1), dist)
        launches = lqcd.kernel_launches() - l0
        return ms, launches, stats

    # headline: the requested precision
    with Clocks() as clk:
        ms, launches, stats = timed(args.precision, args.steps, args.warmup)
    clocks = clk.summary()
    value = ms / 1e3 / (args.steps * world)
    worst_res = max(s["true_residual"] for s in stats.values())

    # plain FP64 form on the same box (context for the mixed-precision speed-up)
    fp64_form = None
    if not args.no_fp64_form and args.precision != 64:
        ms64, _, st64 = timed(64, max(1, min(args.steps, 2)), 1)
        fp64_form = {"value": ms64 / 1e3 / (max(1, min(args.steps, 2)) * world), "unit": UNIT, "dtype": "f64",
                     "iters": {k: v["iters"] for k, v in st64.items()},
                     "true_residual": max(s["true_residual"] for s in st64.values())}

    # end to end through the public API: host field in, host propagators out
    U_pin = torch.from_numpy(U).pin_memory()
    fact_h = torch.empty(fact.shape, dtype=fact.dtype, pin_memory=True)
    corr_h = torch.empty(corr.shape, dtype=corr.dtype, pin_memory=True)
    Ke = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(Ke):
        step(args.precision, U_src=U_pin.numpy())
        fact_h.copy_(fact, non_blocking=True)
        corr_h.copy_(corr, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1), dist)
    e2e = {"value": e2e_ms / 1e3 / (Ke * world), "unit": UNIT, "h2d_bytes_per_step": int(U.nbytes),
           "d2h_bytes_per_step": int(fact.numel() * 16 * 2)}

    # roofline of the dominant kernel: the hop kernel of the inner solves,
    # on the stage-A batch (12 x Gammabar + 12 x Gamma systems) it runs on
    doms = [(0, WL["delta"][1])] * 12 + [WL["gamma"]] * 12
    lat.set_gauge(U_dev, WL["kappa"], WL["csw"])
    d_ms, d_bytes, d_flops = lat.dslash_bench(doms, [0] * 24, args.precision, 50)
    peak, peak_kind = _peaks()
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    traffic = _traffic(args.precision)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "kernel": f"k_hop_lin<{args.precision}> (Wilson-clover hop + clover + axpy, even-odd)",
                "ms_per_launch": round(d_ms, 5), "alg_bytes_per_launch": d_bytes,
                "tflops": round(d_flops / (d_ms * 1e-3) / 1e12, 3)}
    dslash_other = {}
    fp64_peak = lqcd.fma_peak(64)
    for p in (64, 32, 16):
        if p == args.precision:
            continue
        m, b, f = lat.dslash_bench(doms, [0] * 24, p, 20)
        dslash_other[str(p)] = {"GB/s": round(b / (m * 1e-3) / 1e9, 1), "TFLOP/s": round(f / (m * 1e-3) / 1e12, 3),
                                "ms": round(m, 5)}
        if p == 64:  # FP64 is bound by the FP64 FMA rate on this GPU, not by HBM
            dslash_other["64"].update({"bound": "alu", "fp64_fma_peak_tflops_measured": round(fp64_peak, 3),
                                       "alu_frac": round(f / (m * 1e-3) / 1e12 / fp64_peak, 3)})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(U)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}[args.precision], "data": "synthetic",
            "config": {"workload": WL["name"], "dims": list(dims), "kappa": WL["kappa"], "c_sw": WL["csw"],
                       "eps": WL["eps"], "gamma": list(WL["gamma"]), "delta": list(WL["delta"]),
                       "gamma_star": list(WL["gamma_star"]), "x_src": list(WL["x_src"]), "sources": 12,
                       "precision": {64: "fp64", 32: "fp32 inner BiCGStab + fp64 defect correction",
                                     16: "fp16 vectors/links (fp32 norm) inner + fp64 defect correction"}[args.precision],
                       "residual": WL["tol"], "l2": "working set > L2 (no flush)",
                       "parallelism": f"replicas x{world} (independent propagators)"},
            "true_residual": worst_res,
            "iters": {k: v["iters"] for k, v in stats.items()},
            "cycles": {k: v["cycles"] for k, v in stats.items()},
            "fp64_form": fp64_form,
            "e2e": e2e, "roofline": roofline, "dslash_other_precisions": dslash_other,
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
