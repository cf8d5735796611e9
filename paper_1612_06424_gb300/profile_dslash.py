"""Run the solver's hop kernel alone on a batch of systems (for ncu / timing).

  python -m paper_1612_06424_gb300.profile_dslash --dims 32 16 16 16 --precision 32 \
      --slabs 0:17x12 0:13x12 --reps 3
  python -m paper_1612_06424_gb300.profile_dslash --factorized --precision 32

Prints ms per launch, algorithmic GB/s and TFLOP/s.  Each launch is one
kernel of the solver's BiCGStab iteration over every system of the batch
(--kernels, numbered as lqcd_stencil_bench: 0 plain second half of D^,
1 clover-inverse first half, 2 / 3 second half with the fused reductions,
4-6 the vector updates); the default is 0 (k_hop_lin, out_o = A_oo y_o -
1/4 D_hop x_e).
With --factorized it instead runs one 12-source factorized propagator with
correction on the 16^3x32 workload (Gamma 0..13, DeltaGamma 14..17, Gamma*
14..31, source (2,0,0,0)), i.e. every kernel of the solver.  With
--nucleon N it runs the nucleon-block kernel for N random fields on
--nucleon-slices time slices of the lattice (e.g. --dims 64 24 24 24
--nucleon 120 --nucleon-slices 1) `--reps` times.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 16, 16, 16])
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--slabs", nargs="+", default=["0:17x12", "0:13x12"],
                    help="t0:t1xN = N systems on slab t0..t1 (all on field 0)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--kernels", type=int, nargs="+", default=[0])
    ap.add_argument("--field-seed", type=int, default=1)
    ap.add_argument("--kappa", type=float, default=0.13)
    ap.add_argument("--csw", type=float, default=1.0)
    ap.add_argument("--factorized", action="store_true")
    ap.add_argument("--nucleon", type=int, default=0)
    ap.add_argument("--nucleon-slices", type=int, default=1)
    a = ap.parse_args()
    from paper_1612_06424_gb300 import build, inputs, lqcd

    build.build()
    doms = []
    for s in a.slabs:
        rng, n = s.split("x")
        t0, t1 = (int(v) for v in rng.split(":"))
        doms += [(t0, t1)] * int(n)
    if a.nucleon:
        import torch

        lat = lqcd.Lattice(tuple(a.dims), "open")
        s3 = a.dims[1] * a.dims[2] * a.dims[3]
        ns = a.nucleon_slices
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        s = torch.randn((a.nucleon, ns * s3, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        lat.nucleon_blocks(s, (0, ns - 1), 0, ns, conj=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            lat.nucleon_blocks(s, (0, ns - 1), 0, ns, conj=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        fl = 8.0 * 12 * a.nucleon ** 3 * s3 * ns
        print(f"nucleon blocks N={a.nucleon} slices={ns} of {s3} sites: {ms:.3f} ms/launch, "
              f"{fl / ms / 1e9:.2f} TFLOP/s (8 flop per complex FMA of the (x, c) contraction)")
        lat.close()
        return
    if a.dims[0] * a.dims[1] * a.dims[2] * a.dims[3] > 2_000_000:
        U = inputs.random_su3_field_device(tuple(a.dims), 0.4, a.field_seed, device="cuda", rng="device")
    else:
        U = inputs.random_su3_field(tuple(a.dims), 0.4, a.field_seed)
    lat = lqcd.Lattice(tuple(a.dims), "open")
    lat.set_gauge(U, a.kappa, a.csw)
    if a.factorized:
        import time

        import torch

        t = time.time()
        _, _, st = lat.factorized_propagator((0, 13), (14, 31), (2, 0, 0, 0), delta=(14, 17),
                                             params=lqcd.SolverParams(precision=a.precision))
        torch.cuda.synchronize()
        print(f"factorized propagator P={a.precision}: {1e3 * (time.time() - t):.1f} ms",
              {k: (v["iters"], v["true_residual"]) for k, v in st.items()})
        lat.close()
        return
    del U
    for k in a.kernels:
        ms, by, fl = lat.stencil_bench(doms, [0] * len(doms), a.precision, k, a.reps)
        print(f"dims={a.dims} P={a.precision} systems={len(doms)} kernel={k}: {ms:.4f} ms/launch, "
              f"{by / ms / 1e6:.1f} GB/s algorithmic ({by / 1e6:.1f} MB/launch), {fl / ms / 1e9:.2f} TFLOP/s")
    lat.close()


if __name__ == "__main__":
    main()
