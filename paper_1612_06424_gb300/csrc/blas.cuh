// Per-system vector kernels of the batched BiCGStab (van der Vorst 1992)
// and the FP64 defect-correction loop around it, with fused inner
// products.  Every kernel runs on a (system, site-block) grid; a block
// whose system is inactive returns at once.  Inner products accumulate in
// FP64 (per site, then a warp-shuffle tree, then one partial per block);
// `k_finalize_*` sum a system's block partials in a fixed order, so every
// result is deterministic for a given launch shape.
#pragma once

#include "dslash.cuh"

namespace lq {

struct VecArgs {
  const SysDesc* sys;
  const int* active;
  SolverScal* sc;
  double* partial;
  int nby;
};

#define LQ_VEC_PROLOGUE                                            \
  const int s = blockIdx.x;                                        \
  if (va.active && !va.active[s]) return;                          \
  const SysDesc sd = va.sys[s];                                    \
  if ((long long)blockIdx.y * blockDim.x >= sd.n) return;          \
  const long long j = (long long)blockIdx.y * blockDim.x + threadIdx.x; \
  const bool valid = j < sd.n;

template <typename R>
LQ_DI cx<R> c_of(double2 v) {
  return {(R)v.x, (R)v.y};
}

// s = r - alpha v
template <int P>
__global__ void __launch_bounds__(128) k_bicg_s(VecArgs va, const void* r, const float* rn, const void* v,
                                                const float* vn, void* so, float* son) {
  typedef typename Prec<P>::R R;
  LQ_VEC_PROLOGUE
  if (!valid) return;
  const cx<R> al = c_of<R>(va.sc[s].alpha);
  cx<R> a[12], b[12];
  Prec<P>::load(a, sys_ptr<P>(r, sd.off), nrm_ptr(rn, sd.off), sd.n, j);
  Prec<P>::load(b, sys_ptr<P>(v, sd.off), nrm_ptr(vn, sd.off), sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) a[k] = a[k] - al * b[k];
  Prec<P>::store(sys_ptr_w<P>(so, sd.off), nrm_ptr_w(son, sd.off), sd.n, j, a);
}

// x += alpha p + omega s ;  r = s - omega t ;  partials <r0, r>, |r|^2
template <int P>
__global__ void __launch_bounds__(128) k_bicg_xr(VecArgs va, void* x, float* xn, const void* p, const float* pn,
                                                 const void* sv, const float* svn, const void* t, const float* tn,
                                                 void* r, float* rn, const void* r0, const float* r0n) {
  typedef typename Prec<P>::R R;
  LQ_VEC_PROLOGUE
  double red[3] = {0.0, 0.0, 0.0};
  if (valid) {
    const cx<R> al = c_of<R>(va.sc[s].alpha), om = c_of<R>(va.sc[s].omega);
    cx<R> xv[12], pv[12], sv_[12], tv[12];
    Prec<P>::load(xv, sys_ptr<P>(x, sd.off), nrm_ptr(xn, sd.off), sd.n, j);
    Prec<P>::load(pv, sys_ptr<P>(p, sd.off), nrm_ptr(pn, sd.off), sd.n, j);
    Prec<P>::load(sv_, sys_ptr<P>(sv, sd.off), nrm_ptr(svn, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) xv[k] = xv[k] + al * pv[k] + om * sv_[k];
    Prec<P>::store(sys_ptr_w<P>(x, sd.off), nrm_ptr_w(xn, sd.off), sd.n, j, xv);
    Prec<P>::load(tv, sys_ptr<P>(t, sd.off), nrm_ptr(tn, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) sv_[k] = sv_[k] - om * tv[k];
    Prec<P>::store(sys_ptr_w<P>(r, sd.off), nrm_ptr_w(rn, sd.off), sd.n, j, sv_);
    Prec<P>::quantize(sv_);  // the values just stored
    cx<R> w[12];
    Prec<P>::load(w, sys_ptr<P>(r0, sd.off), nrm_ptr(r0n, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      red[0] += (double)w[k].re * sv_[k].re + (double)w[k].im * sv_[k].im;
      red[1] += (double)w[k].re * sv_[k].im - (double)w[k].im * sv_[k].re;
      red[2] += (double)sv_[k].re * sv_[k].re + (double)sv_[k].im * sv_[k].im;
    }
  }
  block_reduce_store<3>(red, va.partial + ((long long)s * va.nby + blockIdx.y) * 4);
}

// p = r + beta (p - omega v)
template <int P>
__global__ void __launch_bounds__(128) k_bicg_p(VecArgs va, void* p, float* pn, const void* r, const float* rn,
                                                const void* v, const float* vn) {
  typedef typename Prec<P>::R R;
  LQ_VEC_PROLOGUE
  if (!valid) return;
  const cx<R> be = c_of<R>(va.sc[s].beta), om = c_of<R>(va.sc[s].omega);
  cx<R> pv[12], rv[12], vv[12];
  Prec<P>::load(pv, sys_ptr<P>(p, sd.off), nrm_ptr(pn, sd.off), sd.n, j);
  Prec<P>::load(rv, sys_ptr<P>(r, sd.off), nrm_ptr(rn, sd.off), sd.n, j);
  Prec<P>::load(vv, sys_ptr<P>(v, sd.off), nrm_ptr(vn, sd.off), sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
  Prec<P>::store(sys_ptr_w<P>(p, sd.off), nrm_ptr_w(pn, sd.off), sd.n, j, pv);
}

// Start of an inner cycle: r = r0 = p = convert(r64), x = 0; partial |r|^2.
template <int P>
__global__ void __launch_bounds__(128) k_inner_init(VecArgs va, const double2* r64, void* r, float* rn, void* r0,
                                                    float* r0n, void* p, float* pn, void* x, float* xn) {
  typedef typename Prec<P>::R R;
  LQ_VEC_PROLOGUE
  double red[3] = {0.0, 0.0, 0.0};
  if (valid) {
    cx<double> a[12];
    Prec<64>::load(a, sys_ptr<64>(r64, sd.off), nullptr, sd.n, j);
    cx<R> b[12], z[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      b[k] = {(R)a[k].re, (R)a[k].im};
      z[k] = {0, 0};
    }
    Prec<P>::store(sys_ptr_w<P>(r, sd.off), nrm_ptr_w(rn, sd.off), sd.n, j, b);
    Prec<P>::store(sys_ptr_w<P>(r0, sd.off), nrm_ptr_w(r0n, sd.off), sd.n, j, b);
    Prec<P>::store(sys_ptr_w<P>(p, sd.off), nrm_ptr_w(pn, sd.off), sd.n, j, b);
    Prec<P>::store(sys_ptr_w<P>(x, sd.off), nrm_ptr_w(xn, sd.off), sd.n, j, z);
    Prec<P>::quantize(b);  // the values just stored
#pragma unroll
    for (int k = 0; k < 12; k++) red[2] += (double)b[k].re * b[k].re + (double)b[k].im * b[k].im;
  }
  block_reduce_store<3>(red, va.partial + ((long long)s * va.nby + blockIdx.y) * 4);
}

// x64 += x (inner solution of precision P)
// A cycle that ended in NaN or divergence (status 2) contributes nothing.
template <int P>
__global__ void __launch_bounds__(128) k_accum64(VecArgs va, double2* x64, const void* x, const float* xn) {
  typedef typename Prec<P>::R R;
  LQ_VEC_PROLOGUE
  if (!valid || va.sc[s].status == 2) return;
  cx<R> e[12];
  Prec<P>::load(e, sys_ptr<P>(x, sd.off), nrm_ptr(xn, sd.off), sd.n, j);
  cx<double> a[12];
  Prec<64>::load(a, sys_ptr<64>(x64, sd.off), nullptr, sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) a[k] = {a[k].re + (double)e[k].re, a[k].im + (double)e[k].im};
  Prec<64>::store(sys_ptr_w<64>(x64, sd.off), nullptr, sd.n, j, a);
}

// Sum of the NQ block partials of system s, in a fixed order (one warp).
LQ_DI void warp_sum_partials(const double* partial, int nby, int nb, int s, double out[3]) {
  const int lane = threadIdx.x & 31;
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = lane; b < nb; b += 32) {
    const double* q = partial + ((long long)s * nby + b) * 4;
    v[0] += q[0];
    v[1] += q[1];
    v[2] += q[2];
  }
#pragma unroll
  for (int q = 0; q < 3; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    out[q] = v[q];
  }
}

LQ_DI double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
LQ_DI double2 cmul2(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
LQ_DI bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// One warp per system: fold the block partials into the iteration scalars.
//  FIN_INIT : rr = rho = |r|^2, rr0 = rr, iters = 0, target2 = max(tau2*rr, floor2)
//  FIN_ALPHA: alpha = rho / <r0, v>
//  FIN_OMEGA: omega = <t, s> / |t|^2
//  FIN_BETA : rr = |r|^2, rho' = <r0, r>; stop the system when rr <= target2,
//             on breakdown, NaN or divergence (rr > 1e8 rr0); else
//             beta = (rho'/rho)(alpha/omega)
//  FIN_NORM : rr = |r|^2 only
// tau2 / floor2 are per call (FIN_INIT); floor2 is relative to bb.
__global__ void k_finalize(int mode, int nsys, const SysDesc* sys, int* active, SolverScal* sc, const double* partial,
                           int nby, int bdim, double tau2, double floor_rel2) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= nsys) return;
  if (active && !active[s]) return;
  const int nb = (int)((sys[s].n + bdim - 1) / bdim);
  double v[3];
  warp_sum_partials(partial, nby, nb, s, v);
  if ((threadIdx.x & 31) != 0) return;
  SolverScal c = sc[s];
  const double2 d = make_double2(v[0], v[1]);
  switch (mode) {
    case FIN_INIT:
      c.rr = c.rr0 = v[2];
      c.rho = make_double2(v[2], 0.0);
      c.iters = 0;
      c.status = 0;
      c.target2 = fmax(tau2 * v[2], floor_rel2 * c.bb);
      if (!(v[2] > c.target2)) active[s] = 0;
      if (!isfinite(v[2])) {
        c.status = 2;
        active[s] = 0;
      }
      break;
    case FIN_ALPHA:
      if (!finite2(d) || (d.x == 0.0 && d.y == 0.0)) {
        c.status = 1;
        active[s] = 0;
      } else {
        c.alpha = cdiv(c.rho, d);
      }
      break;
    case FIN_OMEGA:
      if (!(v[2] > 0.0) || !isfinite(v[2])) {
        c.omega = make_double2(0.0, 0.0);
        c.status = 1;
      } else {
        c.omega = make_double2(d.x / v[2], d.y / v[2]);
      }
      break;
    case FIN_BETA: {
      c.iters += 1;
      c.rr = v[2];
      if (!isfinite(v[2]) || !finite2(d) || v[2] > 1e8 * c.rr0) {  // NaN or divergence
        c.status = 2;
        active[s] = 0;
      } else if (v[2] <= c.target2) {
        active[s] = 0;
      } else if (c.status == 1 || (d.x == 0.0 && d.y == 0.0) || (c.omega.x == 0.0 && c.omega.y == 0.0)) {
        c.status = 1;
        active[s] = 0;
      } else {
        c.beta = cmul2(cdiv(d, c.rho), cdiv(c.alpha, c.omega));
        c.rho = d;
      }
      break;
    }
    case FIN_NORM:
      c.rr = v[2];
      break;
  }
  sc[s] = c;
}

__global__ void k_count_active(int nsys, const int* active, int* count) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int c = 0;
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) c += active[s] ? 1 : 0;
  atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) *count = tot;
}

// Precision conversion of a system vector set: out(P2) = in(P1).
template <int P1, int P2>
__global__ void __launch_bounds__(128) k_convert(VecArgs va, const void* in, const float* inn, void* out, float* outn) {
  typedef typename Prec<P1>::R R1;
  typedef typename Prec<P2>::R R2;
  LQ_VEC_PROLOGUE
  if (!valid) return;
  cx<R1> a[12];
  Prec<P1>::load(a, sys_ptr<P1>(in, sd.off), nrm_ptr(inn, sd.off), sd.n, j);
  cx<R2> b[12];
#pragma unroll
  for (int k = 0; k < 12; k++) b[k] = {(R2)a[k].re, (R2)a[k].im};
  Prec<P2>::store(sys_ptr_w<P2>(out, sd.off), nrm_ptr_w(outn, sd.off), sd.n, j, b);
}

// |v|^2 partials (FP64 vectors)
__global__ void __launch_bounds__(128) k_norm2_64(VecArgs va, const double2* v) {
  LQ_VEC_PROLOGUE
  double red[3] = {0.0, 0.0, 0.0};
  if (valid) {
    cx<double> a[12];
    Prec<64>::load(a, sys_ptr<64>(v, sd.off), nullptr, sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) red[2] += a[k].re * a[k].re + a[k].im * a[k].im;
  }
  block_reduce_store<3>(red, va.partial + ((long long)s * va.nby + blockIdx.y) * 4);
}

}  // namespace lq
