#!/usr/bin/env python
"""Benchmark of the factorized quark propagator on one GB300.

Metric: seconds per 12-source factorized propagator (factorized part of
Sec. 3 plus the full-lattice correction) at true FP64 residual 1e-10, and
the Wilson-clover stencil's achieved HBM bandwidth against the measured peak.

Default workload (one "step"): the 48^3x96 lattice, Wilson-clover kappa =
0.1350, c_sw = 1.0, open time boundary; Gamma = t 0..43, DeltaGamma = 44..51
(frozen), Gamma* = 44..95; 12 point sources at x = (2,0,0,0).  Eight
inner-level gauge fields (the level-0 field U = exp(i 0.4 H), a stand-in for
the paper's quenched ensembles, with the links of Gamma and of t 52..95
redrawn; links starting or ending in the frozen slab kept) stay resident in
HBM; step i takes field i mod 8.  A step loads that field (even-odd packing,
compression, clover blocks and their inverses), solves the Gamma, Gammabar,
Gamma* domain systems and the full lattice for all 12 sources (batched),
assembles fact = D_Gamma^{-1} on Gamma and -D_Gamma*^{-1} D_dGamma*
D_Gammabar^{-1} on Gamma*, and corr = D^{-1} - fact.  The propagators of a
field (fact + corr, 49 GB) and its packed copy (23 GB) leave no room for a
second field's, so the fields run one per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 64|32|16]
  python bench.py --impl reference     # the CPU oracle on the host cores
  python bench.py --workload factorized_16x32  # 16^3x32 factorized propagator + correction
  python bench.py --workload batched_32x64   # 8 slabs x 12 sources x 16 inner-level fields
  python bench.py --workload force_24x48     # domain pseudofermion link force, 4 domains
  python bench.py --workload nucleon_hierarchy_64x24  # Sec. 6 Delta = 8/12/16 hierarchy

Multi-GPU (torchrun): every rank computes its own propagators (its own
gauge fields, independent problems); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
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
    "name": "48^3x96 Wilson-clover factorized propagator + correction, 8 inner-level fields",
    "dims": (96, 48, 48, 48),
    "kappa": 0.135,
    "csw": 1.0,
    "eps": 0.4,
    "gamma": (0, 43),
    "delta": (44, 51),
    "gamma_star": (44, 95),
    "x_src": (2, 0, 0, 0),
    "tol": 1e-10,
    "fields": 8,
}
WL16 = {
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
# kernels of one BiCGStab iteration as lqcd_stencil_bench numbers them, with their launches per iteration
HOP_KERNELS = {1: ("k_hop_clinv (A_ee^-1 D_hop, first half of D^)", 2), 2: ("k_hop_lin + <r0,v>", 1),
               3: ("k_hop_lin + <t,s>, |t|^2", 1)}
BLAS_KERNELS = {4: ("k_bicg_s_w (s = r - alpha v)", 1), 5: ("k_bicg_xr_w (x, r update + 2 dots)", 1),
                6: ("k_bicg_p_w (p update)", 1)}
DTYPE = {64: "f64", 32: "f32+f64", 16: "f16+f32+f64"}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[64, 32, 16])
    ap.add_argument("--no-fp64-form", action="store_true", help="skip timing the plain FP64 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 16^3x32 figures of the default line")
    ap.add_argument("--workload", default="factorized_48x96",
                    choices=["factorized_48x96", "factorized_16x32", "batched_32x64", "force_24x48",
                             "disconnected_64x24", "projection_64x24", "nucleon_hierarchy_64x24"])
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


# sources whose code decides the iteration kernels' memory traffic (device code and launch setup)
KERNEL_SOURCES = ("common.cuh", "dslash.cuh", "blas.cuh", "internal.h", "kernels.cu")


def _kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1612_06424_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic(precision, kernel):
    """DRAM bytes per system site of one kernel of the solver's iteration (lqcd_stencil_bench
    numbering) from the committed ncu record, or None if absent or taken on a different
    kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "dslash_traffic.json")) as fh:
            t = json.load(fh)
        e = t.get(f"{precision}:{kernel}")
        if e and e.get("kernel_hash") == _kernel_hash():
            return float(e["dram_bytes_per_launch"]) / float(e["system_sites"])
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


def _stage_sites(wl):
    """Sites of each solve of a factorized propagator (Gamma, Gammabar, Gamma*, full)."""
    s3 = wl["dims"][1] * wl["dims"][2] * wl["dims"][3]
    T = wl["dims"][0]
    slabs = {"gamma": wl["gamma"], "gamma_bar": (0, wl["delta"][1]), "gamma_star": wl["gamma_star"],
             "full": (0, T - 1)}
    return {k: (b - a + 1) * s3 for k, (a, b) in slabs.items()}


class OracleIterations:
    """The oracle's own BiCGStab iteration count to residual 1e-10 for one column of the
    16^3x32 Gamma system (kappa 0.13, c_sw 1, t 0..13, source (2,0,0,0), spin-colour 0),
    counted in a background host thread (the oracle's C code runs without the GIL) so that
    it overlaps the GPU work; about half a minute on one core."""

    def __init__(self):
        self.result = None
        self.seconds = None
        self._ex = cf.ThreadPoolExecutor(1)
        self._fut = self._ex.submit(self._run)

    def _run(self):
        import oracle
        from paper_1612_06424_gb300 import inputs

        U = inputs.random_su3_field(WL16["dims"], WL16["eps"], 1)
        op = oracle.Operator(WL16["dims"], U, WL16["kappa"], WL16["csw"])
        eta = inputs.point_sources(WL16["dims"], WL16["x_src"])[0]
        t0 = time.perf_counter()
        _, its, _ = op.solve(eta, *WL16["gamma"], tol=1e-10)
        self.seconds = time.perf_counter() - t0
        return its

    def get(self):
        its = self._fut.result()
        self._ex.shutdown()
        return its


SAMPLE_SLICES = 2  # time slices of the workload's field in the oracle's timing sample


def _oracle_sample_operator(U_slab, dims, kappa, csw):
    """The oracle's operator on the sample lattice (periodic in time, so that every site does
    all eight hops like the bulk of the workload's lattice); returns (op, clover build seconds)."""
    import oracle

    oracle.gamma(0)  # the oracle's static tables, filled once before any thread starts
    t0 = time.perf_counter()
    op = oracle.Operator(dims, U_slab, kappa, csw, oracle.BC_PERIODIC)
    return op, time.perf_counter() - t0


def _oracle_apply_sample(op, psis, threads, min_seconds=4.0):
    """Wall seconds of the oracle's D (plain FP64 C, as it stands) applied to the 12 distinct spinor
    columns psis at once, one column per host thread (`threads` threads); repeated until
    min_seconds have passed (at least once).  Returns seconds per round of 12 applications."""
    rounds = 0
    with cf.ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        while rounds < 1 or time.perf_counter() - t0 < min_seconds:
            list(ex.map(lambda c: op.apply(psis[c]), range(12)))
            rounds += 1
        return (time.perf_counter() - t0) / rounds


def _cpu_threads():
    n = os.cpu_count() or 1
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        pass
    return max(1, min(12, n))


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def _cpu_cost(wall_round, sample_sites, wl, iters):
    """Extrapolated oracle seconds for one 12-source factorized propagator + correction: every
    column runs on its own thread (12 columns per round), and a column's solves apply D twice per
    BiCGStab iteration plus twice for the initial and final true residuals, on each solve's sites."""
    sites = _stage_sites(wl)
    apps = sum(sites[k] * (2 * iters[k] + 2) for k in sites)
    return wall_round * apps / sample_sites


def _cpu_baseline(U_sample, wl, gpu_iters, ratio, ora_its, ora_secs, gpu16_its):
    """The oracle on the host cores for the default workload, from a bounded sample: its D applied
    to 12 columns at once on U_sample, the first SAMPLE_SLICES time slices of a step's field
    (host array), measured, times the
    site-applications of the propagator's four solves, with the oracle's iteration count taken as
    the GPU's count on each solve times the oracle/GPU iteration ratio measured on the 16^3x32
    Gamma system (one column, residual 1e-10)."""
    from paper_1612_06424_gb300 import inputs

    ns = SAMPLE_SLICES
    dims_s = (ns,) + tuple(wl["dims"][1:])
    s3 = wl["dims"][1] * wl["dims"][2] * wl["dims"][3]
    op, t_cl = _oracle_sample_operator(U_sample, dims_s, wl["kappa"], wl["csw"])
    threads = _cpu_threads()
    wall = _oracle_apply_sample(op, inputs.gaussian_spinor(dims_s, 97, 12), threads)
    iters = {k: int(round(v * ratio)) for k, v in gpu_iters.items()}
    value = _cpu_cost(wall, ns * s3, wl, iters)
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": _cpu_model(),
            "nproc": os.cpu_count(),
            "sample": f"oracle D on 12 columns at once ({threads} threads) over the first {ns} time slices of the "
                      f"48^3x96 field: {wall:.2f} s per round of 12 (clover build {t_cl:.1f} s, not counted); "
                      f"x the site-applications of the four solves per column (2 per iteration + 2) with "
                      f"oracle iteration counts {iters} = GPU counts {gpu_iters} x {ratio:.3f}, the oracle/GPU "
                      f"ratio on the 16^3x32 Gamma system (oracle {ora_its} iterations to 1e-10 in "
                      f"{ora_secs:.0f} s on one core, GPU {gpu16_its}); extrapolated"}


def run_reference(args):
    """--impl reference: the CPU oracle, as it stands, on the host cores.  Each step is the bounded
    sample of _cpu_baseline (the oracle's D on 12 columns at once over a few time slices of a
    48^3x96-shaped field); the iteration count of every solve is the oracle's own, measured once on the
    16^3x32 Gamma system (kappa 0.13): a lower bound for the kappa 0.135 systems of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1612_06424_gb300 import inputs

    wl = WL
    ns = SAMPLE_SLICES
    dims_s = (ns,) + tuple(wl["dims"][1:])
    s3 = wl["dims"][1] * wl["dims"][2] * wl["dims"][3]
    its_job = OracleIterations()
    op, _ = _oracle_sample_operator(inputs.random_su3_field(dims_s, wl["eps"], 7), dims_s, wl["kappa"], wl["csw"])
    threads = _cpu_threads()
    ora_its = its_job.get()
    iters = {k: ora_its for k in ("gamma", "gamma_bar", "gamma_star", "full")}

    psis = inputs.gaussian_spinor(dims_s, 97, 12)

    def one():
        wall = _oracle_apply_sample(op, psis, threads, min_seconds=0.0)
        return _cpu_cost(wall, ns * s3, wl, iters), wall

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    vals = [one() for _ in range(args.steps)]
    elapsed = time.perf_counter() - t0
    v = statistics.median(x[0] for x in vals)
    cb = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": _cpu_model(),
          "nproc": os.cpu_count(),
          "sample": f"per step: oracle D on 12 columns at once ({threads} threads) over {ns} time slices of a "
                    f"48^3x96-shaped field (median {statistics.median(x[1] for x in vals):.2f} s per round), x the "
                    f"site-applications of the four solves with the oracle's iteration count {ora_its} (measured "
                    f"to 1e-10 on the 16^3x32 Gamma system in {its_job.seconds:.0f} s); extrapolated; "
                    f"the {args.steps} sampled steps took {elapsed:.0f} s"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "dims": list(wl["dims"]), "kappa": wl["kappa"], "c_sw": wl["csw"]},
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


def _dist_setup():
    """(world, rank, local rank, torch.distributed or None) of a torchrun launch (NCCL for N > 1)."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local, dist


def _timed(step, prec, K, W, dist):
    """W untimed steps, then K timed steps between a barrier and a synchronize on both sides,
    CUDA events on the current stream; returns (ms of the K steps, max over ranks; kernel
    launches of this rank in the timed region; statistics of the last step)."""
    import torch

    from paper_1612_06424_gb300 import lqcd

    for _ in range(W):
        step(prec)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l0 = lqcd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed launches
    e0.record()
    stats = None
    for _ in range(K):
        stats = step(prec)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = _max_over_ranks(e0.elapsed_time(e1), dist)
    return ms, lqcd.kernel_launches() - l0, stats


def _tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst figure x the nominal TF32 / bf16 ratio
    (1.1 / 2.25 PFLOP/s), or the fallback 1.9 PFLOP/s bf16 x that ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


def _nucleon_roofline(block_flops, seconds, fp32_peak, n_m, n_sl, s3):
    """The block contraction on the tensor cores (default kernel): three TF32 passes per
    product, against the TF32 peak; the contraction's own rate beside it."""
    peak, kind = _tf32_peak()
    tensor = 3.0 * block_flops / seconds / 1e12
    return {"bound": "tensor", "achieved": round(tensor, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(tensor / peak, 4), "peak_kind": kind,
            "contraction_tflops": round(block_flops / seconds / 1e12, 2),
            "fp32_fma_peak_measured": round(fp32_peak, 1),
            "kernel": f"k_nucleon_block_tc (tcgen05 kind::tf32, 3 passes), N_m = {n_m}, {n_sl} slices of {s3} sites"}


def _iteration_roofline(lat, doms, fields, precision, reps=10):
    """The kernels of one BiCGStab iteration, each timed alone on the solver's batch `doms`
    (lqcd_stencil_bench): the hop kernels (2 x k_hop_clinv, k_hop_lin with <r0,v>, k_hop_lin with
    <t,s>, |t|^2) weighted by their launches per iteration give the stencil roofline; the three
    vector updates give the BLAS figures."""
    peak, peak_kind = _peaks()
    sites = float(sum((b - a + 1) * lat.S3 // 2 for a, b in doms))  # system sites per parity

    def group(kernels):
        per, tot_b, tot_t, traffic, have_traffic = {}, 0.0, 0.0, 0.0, True
        for k, (name, n_launch) in kernels.items():
            ms, by, fl = lat.stencil_bench(doms, fields, precision, k, reps)
            t = _traffic(precision, k)
            per[name] = {"ms": round(ms, 4), "alg_bytes": by, "GB/s": round(by / (ms * 1e-3) / 1e9, 1),
                         "frac": round(by / (ms * 1e-3) / 1e9 / peak, 4), "launches_per_iteration": n_launch,
                         "tflops": round(fl / (ms * 1e-3) / 1e12, 3),
                         "dram_bytes": None if t is None else round(t * sites)}
            tot_b += n_launch * by
            tot_t += n_launch * ms
            if t is None:
                have_traffic = False
            else:
                traffic += n_launch * t * sites
        achieved = tot_b / (tot_t * 1e-3) / 1e9
        return per, achieved, tot_b, tot_t, (traffic if have_traffic else None)

    hop, hop_gbs, hop_b, hop_t, hop_traffic = group(HOP_KERNELS)
    blas, blas_gbs, blas_b, blas_t, _ = group(BLAS_KERNELS)
    n_hop = sum(n for _, n in HOP_KERNELS.values())
    roofline = {"bound": "hbm", "achieved": round(hop_gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(hop_gbs / peak, 4),
                "traffic": None if hop_traffic is None else round(hop_traffic / n_hop),
                "peak_kind": peak_kind,
                "kernel": f"FP{precision} stencil as the solver launches it: 2 x k_hop_clinv + 2 x k_hop_lin (fused "
                          f"reductions) per BiCGStab iteration, time-weighted, on {len(doms)} systems of the "
                          f"solver's batch; achieved and traffic per launch (mean of the 4)",
                "alg_bytes_per_launch": round(hop_b / n_hop), "ms_per_launch": round(hop_t / n_hop, 4),
                "per_kernel": hop}
    blas_out = {"GB/s": round(blas_gbs, 1), "frac": round(blas_gbs / peak, 4), "ms_per_iteration": round(blas_t, 4),
                "alg_bytes_per_iteration": blas_b, "per_kernel": blas,
                "iteration_share_of_time": round(blas_t / (blas_t + hop_t), 3)}
    return roofline, blas_out


def _factorized_16x32(args, dist, world, rank, K, W, with_fp64):
    """The 16^3x32 factorized propagator + correction (kappa 0.13, c_sw 1, Gamma 0..13, DeltaGamma
    14..17, Gamma* 14..31, source (2,0,0,0)): a step loads the field and runs the propagator."""
    import torch

    from paper_1612_06424_gb300 import inputs, lqcd

    wl = WL16
    U = inputs.random_su3_field(wl["dims"], wl["eps"], _rank_seed(rank))
    U_dev = torch.from_numpy(U).cuda()
    lat = lqcd.Lattice(wl["dims"], "open")
    fact = torch.empty((1, 12, lat.V, 4, 3), dtype=torch.complex128, device="cuda")
    corr = torch.empty_like(fact)

    def step(prec, U_src=None):
        lat.set_gauge(U_dev if U_src is None else U_src, wl["kappa"], wl["csw"])
        _, _, st = lat.factorized_propagators(wl["gamma"], wl["gamma_star"], wl["x_src"], [0], delta=wl["delta"],
                                              corr=True, params=lqcd.SolverParams(tol=wl["tol"], precision=prec),
                                              out=(fact, corr))
        return st[0]

    out = {"workload": wl["name"]}
    with Clocks() as clk:
        ms, launches, st = _timed(step, args.precision, K, W, dist)
    out.update({"value": ms / 1e3 / (K * world), "unit": UNIT, "steps": K, "warmup": W, "dtype": DTYPE[args.precision],
                "iters": {k: v["iters"] for k, v in st.items()}, "cycles": {k: v["cycles"] for k, v in st.items()},
                "true_residual": max(v["true_residual"] for v in st.values()), "gpu_launches": int(launches),
                "clocks": clk.summary()})
    if with_fp64 and args.precision != 64:
        ms64, _, st64 = _timed(step, 64, 2, 1, dist)
        out["fp64_form"] = {"value": ms64 / 1e3 / (2 * world), "unit": UNIT, "dtype": "f64",
                            "iters": {k: v["iters"] for k, v in st64.items()},
                            "true_residual": max(v["true_residual"] for v in st64.values())}
    doms = [(0, wl["delta"][1])] * 12 + [wl["gamma"]] * 12
    lat.set_gauge(U_dev, wl["kappa"], wl["csw"])
    out["roofline"], out["blas"] = _iteration_roofline(lat, doms, [0] * 24, args.precision, reps=30)
    out["_U"] = U
    out["_lat"], out["_fact"], out["_corr"], out["_step"] = lat, fact, corr, step
    return out


def run_factorized_16x32(args):
    """--workload factorized_16x32: the 16^3x32 figures as their own JSON line."""
    import torch

    from paper_1612_06424_gb300 import build

    world, rank, _, dist = _dist_setup()
    build.build()
    r = _factorized_16x32(args, dist, world, rank, args.steps, args.warmup, not args.no_fp64_form)
    lat = r.pop("_lat")
    for k in ("_U", "_fact", "_corr", "_step"):
        r.pop(k)
    if rank == 0:
        line = {"metric": METRIC, "n_gpus": world, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "data": "synthetic",
                "ms_per_step": r["value"] * 1e3 * world,
                "config": {"workload": WL16["name"], "dims": list(WL16["dims"]), "kappa": WL16["kappa"],
                           "c_sw": WL16["csw"], "residual": WL16["tol"], "l2": "working set > L2 (no flush)"}}
        line.update(r)
        line.pop("workload")
        print(json.dumps(line))
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    del torch


def run_headline(args):
    """The default workload (module docstring): 48^3x96, 12 sources x 8 inner-level fields, one
    field per step, plus the full-lattice correction, residual 1e-10."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    world, rank, _, dist = _dist_setup()
    build.build()
    wl = WL
    dims = wl["dims"]
    T = dims[0]
    G, DL, GS = wl["gamma"], wl["delta"], wl["gamma_star"]
    nf = args.fields
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    ora = OracleIterations() if want_cpu else None  # host thread; overlaps the GPU work
    t0 = time.time()
    seed = _rank_seed(rank)
    U0 = inputs.random_su3_field_device(dims, wl["eps"], 6 + seed, device="cuda", rng="device")
    Uf = inputs.inner_level_fields_device(U0, dims, [G, (DL[1] + 1, T - 1)], nf, wl["eps"], 7 + seed, frozen=DL,
                                          rng="device")
    del U0
    torch.cuda.empty_cache()
    t_gen = time.time() - t0
    lat = lqcd.Lattice(dims, "open")
    V = lat.V
    fact = torch.empty((1, 12, V, 4, 3), dtype=torch.complex128, device="cuda")
    corr = torch.empty_like(fact)
    counter = [0]

    def step(prec, U_src=None):
        j = counter[0] % nf
        counter[0] += 1
        lat.set_gauge(Uf[j] if U_src is None else U_src, wl["kappa"], wl["csw"])
        _, _, st = lat.factorized_propagators(G, GS, wl["x_src"], [0], delta=DL, corr=True,
                                              params=lqcd.SolverParams(tol=wl["tol"], precision=prec),
                                              out=(fact, corr))
        return st[0]

    with Clocks() as clk:
        ms, launches, stats = _timed(step, args.precision, args.steps, args.warmup, dist)
    clocks = clk.summary()
    value = ms / 1e3 / (args.steps * world)
    gpu_iters = {k: v["iters"] for k, v in stats.items()}

    # plain FP64 form on the same box and workload (one field)
    fp64_form = None
    if not args.no_fp64_form and args.precision != 64:
        ms64, _, st64 = _timed(step, 64, 1, 0, dist)
        fp64_form = {"value": ms64 / 1e3 / world, "unit": UNIT, "dtype": "f64", "fields": 1,
                     "iters": {k: v["iters"] for k, v in st64.items()},
                     "true_residual": max(v["true_residual"] for v in st64.values())}

    # end to end through the public API: the step's field from pinned host memory in, both
    # propagators out to host memory (pinned when the host can lock that much)
    U_h = Uf[0].cpu()
    try:
        U_h = U_h.pin_memory()
        fact_h = torch.empty(fact.shape, dtype=fact.dtype, pin_memory=True)
        corr_h = torch.empty(corr.shape, dtype=corr.dtype, pin_memory=True)
        pinned = True
    except RuntimeError:
        fact_h = torch.empty(fact.shape, dtype=fact.dtype)
        corr_h = torch.empty(corr.shape, dtype=corr.dtype)
        pinned = False
    Ke = 1
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(Ke):
        step(args.precision, U_src=U_h.numpy())
        fact_h.copy_(fact, non_blocking=pinned)
        corr_h.copy_(corr, non_blocking=pinned)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1), dist)
    e2e = {"value": e2e_ms / 1e3 / (Ke * world), "unit": UNIT, "h2d_bytes_per_step": int(U_h.numel() * 16),
           "d2h_bytes_per_step": int(fact.numel() * 16 * 2), "steps": Ke, "pinned_host": pinned}
    del fact_h, corr_h

    # roofline of the stencil as the solver launches it, on the Gamma* batch of a step
    lat.set_gauge(Uf[0], wl["kappa"], wl["csw"])
    roofline, blas = _iteration_roofline(lat, [GS] * 12, [0] * 12, args.precision)
    fp64_peak = lqcd.fma_peak(64)
    m64, _, f64 = lat.stencil_bench([GS] * 12, [0] * 12, 64, 0, 3)
    dslash64 = {"TFLOP/s": round(f64 / (m64 * 1e-3) / 1e12, 3), "ms": round(m64, 3), "bound": "alu",
                "fp64_fma_peak_tflops_measured": round(fp64_peak, 3),
                "alu_frac": round(f64 / (m64 * 1e-3) / 1e12 / fp64_peak, 3)}
    s3 = dims[1] * dims[2] * dims[3]
    U_sample = Uf[0][:SAMPLE_SLICES * s3].cpu().numpy() if want_cpu else None
    lat.close()
    del fact, corr
    torch.cuda.empty_cache()

    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        del Uf
        torch.cuda.empty_cache()
        r = _factorized_16x32(args, None, 1, 0, 5, 3, True)
        r.pop("_lat").close()
        for k in ("_U", "_fact", "_corr", "_step"):
            r.pop(k)
        extra = r

    cpu = None
    if want_cpu:
        ora_its = ora.get()
        gpu16 = (extra or {}).get("fp64_form", {}).get("iters", {}).get("gamma") or (extra or {}).get("iters", {}).get(
            "gamma")
        ratio = ora_its / gpu16 if gpu16 else 1.0
        cpu = _cpu_baseline(U_sample, wl, gpu_iters, ratio, ora_its, ora.seconds or 0.0, gpu16)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": wl["name"], "dims": list(dims), "kappa": wl["kappa"], "c_sw": wl["csw"],
                       "eps": wl["eps"], "gamma": list(G), "delta": list(DL), "gamma_star": list(GS),
                       "x_src": list(wl["x_src"]), "sources": 12, "inner_level_fields": nf,
                       "fields_per_step": 1,
                       "precision": {64: "fp64", 32: "fp32 inner BiCGStab + fp64 defect correction",
                                     16: "fp16 vectors/links (fp32 norm) inner + fp64 defect correction"}[
                           args.precision],
                       "residual": wl["tol"], "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{world} (independent propagators)"},
            "true_residual": max(v["true_residual"] for v in stats.values()),
            "iters": gpu_iters, "cycles": {k: v["cycles"] for k, v in stats.items()},
            "fp64_form": fp64_form, "e2e": e2e, "roofline": roofline, "blas": blas,
            "dslash_fp64": dslash64, "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches),
            "setup_s": round(t_gen, 1), "factorized_16x32": extra,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


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
    disconnected traces of Sec. 5 with `--sources` Gaussian sources (100 in the paper) on
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
    Sec. 3.3 with the Sec. 6 setup for Delta = 8: Gammabar = t 0..31 (Gamma = 0..23,
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
        "nucleon_blocks_roofline": _nucleon_roofline(block_flops, t[3], fp32_peak, n_m, n_sl, s3),
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


def run_hierarchy(args):
    """64x24^3 Wilson-clover (kappa 0.1360, c_sw 1.0), open time boundary: the nucleon hierarchy of
    Sec. 6 eq. nucleon_prop_hierarchical with the paper's split, Gamma = t 0..23, Gamma* = 24..63
    and overlaps Delta = 8, 12, 16 (DeltaGamma = 24 .. 23+Delta), 12 point sources at (4,0,0,0): the
    three factorized propagators and the full one in one batched set of solves, then the nucleon
    point correlators.  A step is one hierarchy."""
    import torch

    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    dims = (64, 24, 24, 24)
    kappa, csw = 0.136, 1.0
    G, GS, ends = (0, 23), (24, 63), [31, 35, 39]
    U = inputs.random_su3_field_device(dims, 0.4, 41, device="cuda")
    lat = lqcd.Lattice(dims, "open")
    lat.set_gauge(U, kappa, csw)
    del U
    params = lqcd.SolverParams(tol=1e-10, precision=args.precision)
    for _ in range(max(0, args.warmup)):
        lat.nucleon_hierarchy(G, GS, ends, (4, 0, 0, 0), 0, params)
    torch.cuda.synchronize()
    n0 = lqcd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks() as clk:
        e0.record()
        for _ in range(args.steps):
            terms, full, st = lat.nucleon_hierarchy(G, GS, ends, (4, 0, 0, 0), 0, params)
        e1.record()
        torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / args.steps
    ys = [30, 40, 50]
    print(json.dumps({
        "metric": "s per nucleon hierarchy (3 factorized propagators + full, 12 sources, contractions) @ res 1e-10",
        "value": sec, "unit": "s/hierarchy", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": "64x24^3 nucleon hierarchy, Delta = 8/12/16", "dims": list(dims), "kappa": kappa,
                   "c_sw": csw, "gamma": list(G), "gamma_star": list(GS), "delta_ends": ends, "x_src": [4, 0, 0, 0]},
        "iters": {k: v["iters"] for k, v in st.items()},
        "true_residual_max": max(v["true_residual"] for v in st.values()),
        "terms_over_full": {str(y): [abs(terms[k][y]) / abs(full[y]) for k in range(len(ends) + 1)] for y in ys},
        "gpu_launches": lqcd.kernel_launches() - n0, "clocks": clk.summary()}))
    lat.close()


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    runs = {"batched_32x64": run_batched, "force_24x48": run_force, "disconnected_64x24": run_disconnected,
            "projection_64x24": run_projection, "factorized_16x32": run_factorized_16x32,
            "factorized_48x96": run_headline, "nucleon_hierarchy_64x24": run_hierarchy}
    return runs[args.workload](args)


if __name__ == "__main__":
    main()
