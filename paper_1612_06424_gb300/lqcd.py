"""Thin Python binding of the C ABI in include/lqcd.h (argument marshalling only).

Every operation runs in the CUDA library ``lib/liblqcd.so``; this module
only converts torch tensors to device pointers, structs and error codes.
There is no CPU fallback: importing the binding without the built library,
or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LQCD_LIB") or os.path.join(_HERE, "lib", "liblqcd.so")

BC = {"open": 0, "periodic": 1, "antiperiodic": 2}

ERRORS = {
    -1: "EBADARG", -2: "ENOMEM", -3: "ENONUNITARY", -4: "ENOTCONVERGED",
    -5: "EBREAKDOWN", -6: "ENAN", -7: "ECUDA", -8: "ENOFIELD", -9: "ERANK",
}


class LQCDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Slab(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int), ("t1", ctypes.c_int)]


class SplitC(ctypes.Structure):
    _fields_ = [("gamma", Slab), ("delta", Slab), ("gamma_star", Slab)]


class ParamsC(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int), ("max_wave", ctypes.c_int)]


class StatsC(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class SolverParams:
    tol: float = 1e-10
    max_iter: int = 100000
    precision: int = 64
    inner_tol: float = 0.0
    check_every: int = 0
    max_wave: int = 0

    def c(self) -> ParamsC:
        return ParamsC(self.tol, self.max_iter, self.precision, self.inner_tol, self.check_every, self.max_wave)


_lib = None


def lib() -> ctypes.CDLL:
    """Load liblqcd.so (built by __graft_entry__.build() / build.py); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    c = ctypes.c_int
    L.lqcd_create_lattice.argtypes = [ip, c, ctypes.POINTER(vp)]
    L.lqcd_destroy_lattice.argtypes = [vp]
    L.lqcd_set_gauge.argtypes = [vp, c, vp, ctypes.c_double, ctypes.c_double, c, vp]
    L.lqcd_dslash.argtypes = [vp, c, ctypes.POINTER(Slab), c, c, vp, vp, vp]
    L.lqcd_solve_block.argtypes = [vp, c, ctypes.POINTER(Slab), ip, vp, vp, ctypes.POINTER(ParamsC),
                                   ctypes.POINTER(StatsC), vp]
    L.lqcd_solve_full.argtypes = [vp, c, ip, vp, vp, ctypes.POINTER(ParamsC), ctypes.POINTER(StatsC), vp]
    L.lqcd_factorized_propagator.argtypes = [vp, ctypes.POINTER(SplitC), ip, c, vp, vp, ctypes.POINTER(ParamsC),
                                             ctypes.POINTER(StatsC), vp]
    L.lqcd_factorized_propagators.argtypes = [vp, ctypes.POINTER(SplitC), ip, c, ip, vp, vp,
                                              ctypes.POINTER(ParamsC), ctypes.POINTER(StatsC), vp]
    L.lqcd_schur_boundary.argtypes = [vp, ctypes.POINTER(SplitC), c, ip, vp, vp, vp]
    L.lqcd_schur_solve.argtypes = [vp, ctypes.POINTER(SplitC), c, ip, vp, vp, ctypes.POINTER(ParamsC),
                                   ctypes.POINTER(StatsC), vp]
    L.lqcd_nucleon_point.argtypes = [vp, c, vp, c, c, vp, vp]
    L.lqcd_nucleon_hierarchy.argtypes = [vp, ctypes.POINTER(SplitC), c, ip, ip, c, vp, ctypes.POINTER(ParamsC),
                                         ctypes.POINTER(StatsC), vp]
    L.lqcd_link_force.argtypes = [vp, ctypes.POINTER(Slab), c, vp, vp, dp, ctypes.POINTER(ParamsC),
                                  ctypes.POINTER(StatsC), vp]
    L.lqcd_point_propagators.argtypes = [vp, c, ctypes.POINTER(Slab), ip, ip, ip, vp, ctypes.POINTER(ParamsC),
                                         ctypes.POINTER(StatsC), vp]
    L.lqcd_dslash_bench.argtypes = [vp, c, ctypes.POINTER(Slab), ip, c, c, dp, dp, dp, vp]
    L.lqcd_stencil_bench.argtypes = [vp, c, ctypes.POINTER(Slab), ip, c, c, c, dp, dp, dp, vp]
    L.lqcd_boundary_modes.argtypes = [vp, ctypes.POINTER(Slab), c, c, c, c, vp, vp, ctypes.POINTER(ParamsC),
                                      ctypes.POINTER(StatsC), vp]
    L.lqcd_projected_factors.argtypes = [vp, ctypes.POINTER(SplitC), c, c, vp, vp, vp, ctypes.POINTER(ParamsC),
                                         ctypes.POINTER(StatsC), vp]
    L.lqcd_projected_propagator.argtypes = [vp, ctypes.POINTER(SplitC), c, vp, vp, ip, vp, vp]
    L.lqcd_nucleon_blocks.argtypes = [vp, ctypes.POINTER(Slab), c, vp, c, c, c, vp, vp]
    L.lqcd_nucleon_contract.argtypes = [c, c, vp, c, vp, vp, vp]
    L.lqcd_level_mean.argtypes = [ctypes.c_longlong, c, vp, vp, vp]
    L.lqcd_disconnected_trace.argtypes = [vp, c, ctypes.POINTER(Slab), c, c, vp, vp, vp, ctypes.POINTER(ParamsC),
                                          ctypes.POINTER(StatsC), vp]
    L.lqcd_last_error.restype = ctypes.c_char_p
    L.lqcd_kernel_launches.restype = ctypes.c_longlong
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise LQCDError(rc, lib().lqcd_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str) -> ctypes.c_void_p:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError(f"{name}: need a contiguous complex128 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def kernel_launches() -> int:
    return int(lib().lqcd_kernel_launches())


def fma_peak(bits: int = 64) -> float:
    """Measured FMA throughput of the current GPU (TFLOP/s) in FP64 or FP32."""
    t = ctypes.c_double(0.0)
    lib().lqcd_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    _check(lib().lqcd_fma_peak(bits, ctypes.byref(t), _stream(None)))
    return t.value


class Lattice:
    """A lattice T x L1 x L2 x L3 (time first) with its gauge fields on the current GPU."""

    def __init__(self, dims, bc: str = "open"):
        if not torch.cuda.is_available():
            raise RuntimeError("lqcd: a CUDA device is required (no CPU fallback)")
        self.dims = tuple(int(d) for d in dims)
        self.T = self.dims[0]
        self.S3 = self.dims[1] * self.dims[2] * self.dims[3]
        self.V = self.T * self.S3
        self.bc = bc
        h = ctypes.c_void_p()
        _check(lib().lqcd_create_lattice((ctypes.c_int * 4)(*self.dims), BC[bc], ctypes.byref(h)))
        self._h = h
        self.n_fields = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().lqcd_destroy_lattice(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- fields
    def set_gauge(self, U, kappa: float, csw: float = 0.0, stream=None):
        """U: complex128 [n_fields, V, 4, 3, 3] (or [V, 4, 3, 3]) as numpy (host) or CUDA tensor."""
        if isinstance(U, np.ndarray):
            arr = np.ascontiguousarray(U, dtype=np.complex128)
            n = arr.size // (self.V * 36)
            _check(lib().lqcd_set_gauge(self._h, n, ctypes.c_void_p(arr.ctypes.data), kappa, csw, 1, _stream(stream)))
        else:
            n = U.numel() // (self.V * 36)
            _check(lib().lqcd_set_gauge(self._h, n, _dev(U.contiguous(), "U"), kappa, csw, 0, _stream(stream)))
        self.n_fields = n
        self.kappa, self.csw = kappa, csw

    # ------------------------------------------------------------- operators
    def slab_len(self, t0: int, t1: int) -> int:
        return (t1 - t0 + 1) * self.S3

    def dslash(self, psi: torch.Tensor, field: int = 0, dom=None, dagger: bool = False, precision: int = 64,
               stream=None) -> torch.Tensor:
        """D_L psi on the slab dom=(t0, t1) (None: whole lattice); psi [sites_of_slab, 4, 3]."""
        out = torch.empty_like(psi)
        sl = ctypes.byref(Slab(*dom)) if dom is not None else None
        _check(lib().lqcd_dslash(self._h, field, sl, int(dagger), precision, _dev(psi, "psi"), _dev(out, "out"),
                                 _stream(stream)))
        return out

    def solve_block(self, src: torch.Tensor, doms, field_ids, params: SolverParams | None = None, stream=None):
        """Batched D_{L_k} psi_k = eta_k; src = slab vectors back to back (complex128, CUDA)."""
        n = len(doms)
        sl = (Slab * n)(*[Slab(*d) for d in doms])
        fi = (ctypes.c_int * n)(*field_ids)
        sol = torch.empty_like(src)
        st = (StatsC * n)()
        p = (params or SolverParams()).c()
        rc = lib().lqcd_solve_block(self._h, n, sl, fi, _dev(src, "src"), _dev(sol, "sol"), ctypes.byref(p), st,
                                    _stream(stream))
        _check(rc)
        return sol, [s.as_dict() for s in st]

    def point_propagators(self, doms, field_ids, x_src, cols, params: SolverParams | None = None, sol=None,
                          stream=None):
        """Batched D_{L_k} psi_k = point source (x_src[k], column cols[k]); returns (sol, stats)."""
        n = len(doms)
        sl = (Slab * n)(*[Slab(*d) for d in doms])
        fi = (ctypes.c_int * n)(*field_ids)
        xs = (ctypes.c_int * (4 * n))(*[int(v) for x in x_src for v in x])
        cs = (ctypes.c_int * n)(*cols)
        total = sum(self.slab_len(*d) for d in doms)
        if sol is None:
            sol = torch.empty((total, 4, 3), dtype=torch.complex128, device=torch.device("cuda", torch.cuda.current_device()))
        st = (StatsC * n)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_point_propagators(self._h, n, sl, fi, xs, cs, _dev(sol, "sol"), ctypes.byref(p), st,
                                            _stream(stream)))
        return sol, [s.as_dict() for s in st]

    def solve_full(self, src: torch.Tensor, field_ids, params: SolverParams | None = None, stream=None):
        n = len(field_ids)
        fi = (ctypes.c_int * n)(*field_ids)
        sol = torch.empty_like(src)
        st = (StatsC * n)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_solve_full(self._h, n, fi, _dev(src, "src"), _dev(sol, "sol"), ctypes.byref(p), st,
                                     _stream(stream)))
        return sol, [s.as_dict() for s in st]

    def factorized_propagator(self, gamma, gamma_star, x_src, field: int = 0, delta=None, corr: bool = True,
                              params: SolverParams | None = None, stream=None, out=None):
        """(fact, corr, stats) for the 12 point sources at x_src (Sec. 3); fact/corr [12, V, 4, 3]."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            fact = torch.empty((12, self.V, 4, 3), dtype=torch.complex128, device=dev)
            cor = torch.empty_like(fact) if corr else None
        else:
            fact, cor = out
        d = delta if delta is not None else (gamma[1] + 1, gamma[1])
        sp = SplitC(Slab(*gamma), Slab(*d), Slab(*gamma_star))
        st = (StatsC * 4)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_factorized_propagator(self._h, ctypes.byref(sp), (ctypes.c_int * 4)(*x_src), field,
                                                _dev(fact, "fact"), _dev(cor, "corr") if cor is not None else None,
                                                ctypes.byref(p), st, _stream(stream)))
        names = ["gamma", "gamma_bar", "gamma_star", "full"]
        return fact, cor, {k: s.as_dict() for k, s in zip(names, st)}

    def factorized_propagators(self, gamma, gamma_star, x_src, fields, delta=None, corr: bool = True,
                               params: SolverParams | None = None, stream=None, out=None):
        """Sec. 3 for several gauge fields in one batched call: (fact, corr, stats) with fact/corr
        [n_fields, 12, V, 4, 3] and stats[j] the four stage statistics of field fields[j]."""
        n = len(fields)
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            fact = torch.empty((n, 12, self.V, 4, 3), dtype=torch.complex128, device=dev)
            cor = torch.empty_like(fact) if corr else None
        else:
            fact, cor = out
        sp = self._split(gamma, gamma_star, delta)
        st = (StatsC * (4 * n))()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_factorized_propagators(self._h, ctypes.byref(sp), (ctypes.c_int * 4)(*x_src), n,
                                                 (ctypes.c_int * n)(*fields), _dev(fact, "fact"),
                                                 _dev(cor, "corr") if cor is not None else None, ctypes.byref(p),
                                                 st, _stream(stream)))
        names = ["gamma", "gamma_bar", "gamma_star", "full"]
        stats = [{k: st[4 * j + i].as_dict() for i, k in enumerate(names)} for j in range(n)]
        return fact, cor, stats

    def schur_boundary(self, psi_gbar: torch.Tensor, gamma, gamma_star, field_ids, delta=None, stream=None):
        """chi_k = D_dGamma* psi_k (eq. quark_prop_II) for slab vectors psi [n, Gammabar sites, 4, 3] on the
        fields field_ids; chi [n, 2, L1 L2 L3, 4, 3] (slot 0: first slice of Gamma*, slot 1: last slice)."""
        n = len(field_ids)
        chi = torch.empty((n, 2, self.S3, 4, 3), dtype=torch.complex128, device=psi_gbar.device)
        sp = self._split(gamma, gamma_star, delta)
        _check(lib().lqcd_schur_boundary(self._h, ctypes.byref(sp), n, (ctypes.c_int * n)(*field_ids),
                                         _dev(psi_gbar, "psi"), _dev(chi, "chi"), _stream(stream)))
        return chi

    def schur_solve(self, chi: torch.Tensor, gamma, gamma_star, field_ids, delta=None,
                    params: SolverParams | None = None, stream=None):
        """fact_k = -D_Gamma*^{-1} chi_k on Gamma* (eq. quark_prop_II); returns (fact [n, Gamma* sites, 4, 3],
        stats)."""
        n = len(field_ids)
        out = torch.empty((n, self.slab_len(*gamma_star), 4, 3), dtype=torch.complex128, device=chi.device)
        sp = self._split(gamma, gamma_star, delta)
        st = (StatsC * n)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_schur_solve(self._h, ctypes.byref(sp), n, (ctypes.c_int * n)(*field_ids),
                                      _dev(chi.contiguous(), "chi"), _dev(out, "fact"), ctypes.byref(p), st,
                                      _stream(stream)))
        return out, [s.as_dict() for s in st]

    def nucleon_point(self, props: torch.Tensor, t0: int = 0, n_t: int | None = None, stream=None):
        """(W1, W2) per sink time slice of point-source propagators props [n, 12, V, 4, 3] (or [12, V, 4, 3]);
        returns complex128 [n, n_t, 2] on the propagators' device.  The correlator is W1 - W2."""
        p = props if props.dim() == 5 else props.unsqueeze(0)
        n_t = self.T - t0 if n_t is None else n_t
        W = torch.empty((p.shape[0], n_t, 2), dtype=torch.complex128, device=p.device)
        _check(lib().lqcd_nucleon_point(self._h, p.shape[0], _dev(p.contiguous(), "props"), t0, n_t, _dev(W, "W"),
                                        _stream(stream)))
        return W

    def nucleon_hierarchy(self, gamma, gamma_star, delta_ends, x_src, field: int = 0,
                          params: SolverParams | None = None, stream=None):
        """Eq. nucleon_prop_hierarchical (Sec. 6): the terms C^(0), C^(1) - C^(0), ..., C^(rest) [n_d + 1, T]
        of the nucleon correlator from the point source x_src, for the nested overlaps DeltaGamma_d =
        gamma[1]+1 .. delta_ends[d]; returns (terms, full C [T], stats) as numpy complex128."""
        n = len(delta_ends)
        C = np.zeros((n + 2, self.T), dtype=np.complex128)
        sp = self._split(gamma, gamma_star, None)
        st = (StatsC * 4)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_nucleon_hierarchy(self._h, ctypes.byref(sp), n, (ctypes.c_int * n)(*delta_ends),
                                            (ctypes.c_int * 4)(*x_src), field, ctypes.c_void_p(C.ctypes.data),
                                            ctypes.byref(p), st, _stream(stream)))
        names = ["gamma", "gamma_bar", "gamma_star", "full"]
        return C[:n + 1], C[n + 1], {k: s.as_dict() for k, s in zip(names, st)}

    def dslash_bench(self, doms, field_ids, precision: int = 32, reps: int = 20, stream=None):
        """(ms per launch, algorithmic bytes per launch, flops per launch) of the solver's hop kernel."""
        n = len(doms)
        sl = (Slab * n)(*[Slab(*d) for d in doms])
        fi = (ctypes.c_int * n)(*field_ids)
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().lqcd_dslash_bench(self._h, n, sl, fi, precision, reps, ctypes.byref(ms), ctypes.byref(by),
                                       ctypes.byref(fl), _stream(stream)))
        return ms.value, by.value, fl.value

    def stencil_bench(self, doms, field_ids, precision: int = 32, kernel: int = 0, reps: int = 20, stream=None):
        """(ms per launch, algorithmic bytes, flops) of one kernel of the solver's iteration
        (0-3: hop kernels, 4-6: vector updates; see lqcd_stencil_bench in include/lqcd.h)."""
        n = len(doms)
        sl = (Slab * n)(*[Slab(*d) for d in doms])
        fi = (ctypes.c_int * n)(*field_ids)
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().lqcd_stencil_bench(self._h, n, sl, fi, precision, kernel, reps, ctypes.byref(ms),
                                        ctypes.byref(by), ctypes.byref(fl), _stream(stream)))
        return ms.value, by.value, fl.value

    def link_force(self, phi: torch.Tensor, dom, field: int = 0, params: SolverParams | None = None,
                   want_force: bool = True, stream=None):
        """(force [V,4,8] float64 or None, S, stats) of S = phi^dag (D_L^dag D_L)^{-1} phi."""
        dev = phi.device
        F = torch.zeros((self.V, 4, 8), dtype=torch.float64, device=dev) if want_force else None
        S = ctypes.c_double(0.0)
        st = (StatsC * 2)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_link_force(self._h, ctypes.byref(Slab(*dom)), field, _dev(phi, "phi"),
                                     ctypes.c_void_p(F.data_ptr()) if F is not None else None, ctypes.byref(S),
                                     ctypes.byref(p), st, _stream(stream)))
        return F, S.value, [s.as_dict() for s in st]

    def disconnected_trace(self, eta: torch.Tensor, doms, field: int = 0, params: SolverParams | None = None,
                           stream=None):
        """Sec. 5 eq. stochastic_estimator on each slab of `doms` (Wilson operator, c_sw = 0).

        eta: device complex128 [n_src, V, 4, 3] sources.  Returns (trace, mean, stats):
        trace [n_src, n_doms, T] per source and time slice, mean [n_doms, T] over the
        sources (both complex128 on eta's device), stats per slab."""
        n_src = eta.shape[0]
        n = len(doms)
        sl = (Slab * n)(*[Slab(*d) for d in doms])
        T = self.dims[0]
        tr = torch.empty((n_src, n, T), dtype=torch.complex128, device=eta.device)
        mean = torch.empty((n, T), dtype=torch.complex128, device=eta.device)
        st = (StatsC * n)()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_disconnected_trace(self._h, n, sl, field, n_src, _dev(eta, "eta"), _dev(tr, "trace"),
                                             _dev(mean, "mean"), ctypes.byref(p), st, _stream(stream)))
        return tr, mean, [s.as_dict() for s in st]

    def boundary_modes(self, v0: torch.Tensor, dom, g1: int, field: int = 0, n_iter: int = 10,
                       params: SolverParams | None = None, stream=None):
        """Sec. 6 projection vectors: n_iter inverse iterations of D on the slab `dom` from the
        starting vectors v0 (complex128 [n_modes, slab sites, 4, 3]), each followed by an
        orthonormalisation; phi = orthonormalised (1 + g0)/2 V on slice g1.
        Returns (phi [n_modes, L1 L2 L3, 4, 3], stats)."""
        n = v0.shape[0]
        phi = torch.empty((n, self.S3, 4, 3), dtype=torch.complex128, device=v0.device)
        st = StatsC()
        p = (params or SolverParams()).c()
        _check(lib().lqcd_boundary_modes(self._h, ctypes.byref(Slab(*dom)), g1, field, n, n_iter, _dev(v0, "v0"),
                                         _dev(phi, "phi"), ctypes.byref(p), ctypes.byref(st), _stream(stream)))
        return phi, st.as_dict()

    def _split(self, gamma, gamma_star, delta):
        d = delta if delta is not None else (gamma[1] + 1, gamma[1])
        return SplitC(Slab(*gamma), Slab(*d), Slab(*gamma_star))

    def projected_factors(self, phi: torch.Tensor, gamma, gamma_star, delta=None, field: int = 0,
                          params: SolverParams | None = None, stream=None):
        """Factors of eq. quark_prop_II_proj for projection vectors phi [N, L1 L2 L3, 4, 3] on the last
        slice of Gamma: xi = D_Gammabar^{-dag} phi (slab vectors on Gammabar) and
        eta = D_Gamma*^{-1} D_dGamma* phi (slab vectors on Gamma*).  Returns (xi, eta, stats)."""
        n = phi.shape[0]
        gb = (0, delta[1] if delta is not None and delta[1] >= delta[0] else gamma[1])
        xi = torch.empty((n, self.slab_len(*gb), 4, 3), dtype=torch.complex128, device=phi.device)
        eta = torch.empty((n, self.slab_len(*gamma_star), 4, 3), dtype=torch.complex128, device=phi.device)
        st = (StatsC * 2)()
        p = (params or SolverParams()).c()
        sp = self._split(gamma, gamma_star, delta)
        _check(lib().lqcd_projected_factors(self._h, ctypes.byref(sp), field, n, _dev(phi, "phi"), _dev(xi, "xi"),
                                            _dev(eta, "eta"), ctypes.byref(p), st, _stream(stream)))
        return xi, eta, {"gamma_bar": st[0].as_dict(), "gamma_star": st[1].as_dict()}

    def projected_propagator(self, xi: torch.Tensor, eta: torch.Tensor, gamma, gamma_star, x_src, delta=None,
                             out: torch.Tensor | None = None, stream=None):
        """Case II with the quark line cut (eq. quark_prop_II_proj): fact[b](y) = -sum_i eta_i(y) xi_i(x)^dag[b]
        on Gamma* for the 12 point sources at x_src; fact [12, V, 4, 3] (zero elsewhere if out is None)."""
        fact = out if out is not None else torch.zeros((12, self.V, 4, 3), dtype=torch.complex128, device=xi.device)
        sp = self._split(gamma, gamma_star, delta)
        _check(lib().lqcd_projected_propagator(self._h, ctypes.byref(sp), xi.shape[0], _dev(xi, "xi"),
                                               _dev(eta, "eta"), (ctypes.c_int * 4)(*x_src), _dev(fact, "fact"),
                                               _stream(stream)))
        return fact

    def nucleon_blocks(self, s: torch.Tensor, slab, t0: int, n_t: int = 1, conj: bool = False, stream=None):
        """Blocks B[t][i][j][k][alpha] of eq. nucleon_prop_factorized for the fields s (complex128
        [n, slab sites, 4, 3] on `slab`; conj=True for the xi factors), slices t0 .. t0+n_t-1."""
        n = s.shape[0]
        B = torch.empty((n_t, n, n, n, 4), dtype=torch.complex128, device=s.device)
        _check(lib().lqcd_nucleon_blocks(self._h, ctypes.byref(Slab(*slab)), n, _dev(s, "s"), int(bool(conj)), t0,
                                         n_t, _dev(B, "B"), _stream(stream)))
        return B


def nucleon_contract(B_xi: torch.Tensor, B_eta: torch.Tensor, stream=None) -> torch.Tensor:
    """W[ix][iy] = (W1, W2) of eq. nucleon_prop_factorized for blocks B_xi [n_x, n, n, n, 4] (source
    slices) and B_eta [n_y, n, n, n, 4] (sink slices); complex128 [n_x, n_y, 2]."""
    nx, n = B_xi.shape[0], B_xi.shape[1]
    ny = B_eta.shape[0]
    W = torch.empty((nx, ny, 2), dtype=torch.complex128, device=B_xi.device)
    _check(lib().lqcd_nucleon_contract(n, nx, _dev(B_xi, "B_xi"), ny, _dev(B_eta, "B_eta"), _dev(W, "W"),
                                       _stream(stream)))
    return W


def level_mean(t: torch.Tensor, stream=None) -> torch.Tensor:
    """Mean over the leading (level-1) axis of a complex128 CUDA tensor, in the library's kernel."""
    n1 = t.shape[0]
    out = torch.empty(t.shape[1:], dtype=torch.complex128, device=t.device)
    _check(lib().lqcd_level_mean(out.numel(), n1, _dev(t, "in"), _dev(out, "out"), _stream(stream)))
    return out


def multilevel_nucleon(B_xi_levels: torch.Tensor, B_eta_levels: torch.Tensor, stream=None) -> torch.Tensor:
    """Level-1 part of eq. multilevel_estimator for the factorized nucleon (Sec. 2.2, Sec. 4.2): the
    blocks of each region averaged over their n1 level-1 fields (B_xi_levels [n1, n_x, n, n, n, 4],
    B_eta_levels [n1, n_y, n, n, n, 4]), then contracted: W [n_x, n_y, 2] (W1, W2).  The contraction
    is bilinear, so this equals the mean of the n1^2 contractions of level-1 pairs."""
    return nucleon_contract(level_mean(B_xi_levels, stream), level_mean(B_eta_levels, stream), stream)


class DomainPseudofermionAction(torch.autograd.Function):
    """S(omega) = phi^dag (D_L^dag D_L)^{-1} phi with U_mu(x) -> exp(i omega^a_mu(x) T_a) U_mu(x).

    forward(omega, lattice, dom, field, phi, params, store) evaluates S at
    omega = 0 (omega is a zero tensor [V,4,8] standing for the Lie-algebra
    coordinates of every link); backward returns grad_S * F, F the link force
    from the CUDA kernels.  Two ways to get F:
      store=True:  forward already solves for X and Y and computes F, which is
                   kept for backward (2 solves in all, one [V,4,8] FP64 tensor
                   held in between);
      store=False: forward solves D^dag only (S = |Y|^2) and backward
                   recomputes X and Y (3 solves, nothing of size V held);
      store=None:  store when F and three times its size of headroom fit in
                   the device's free memory, else recompute.
    """

    @staticmethod
    def forward(ctx, omega, lattice: Lattice, dom, field: int, phi: torch.Tensor, params=None, store=None):
        if store is None:
            free, _ = torch.cuda.mem_get_info(omega.device)
            store = 4 * lattice.V * 4 * 8 * 8 < free
        ctx.lattice, ctx.dom, ctx.field, ctx.params, ctx.store = lattice, dom, field, params, bool(store)
        if store:
            F, S, _ = lattice.link_force(phi, dom, field, params, want_force=True)
            ctx.save_for_backward(phi, F)
        else:
            _, S, _ = lattice.link_force(phi, dom, field, params, want_force=False)
            ctx.save_for_backward(phi)
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, grad_S):
        if ctx.store:
            _, F = ctx.saved_tensors
        else:
            (phi,) = ctx.saved_tensors
            F, _, _ = ctx.lattice.link_force(phi, ctx.dom, ctx.field, ctx.params, want_force=True)
        return grad_S * F, None, None, None, None, None, None
