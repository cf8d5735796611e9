// Per-system vector kernels of the batched BiCGStab (van der Vorst 1992)
// and the FP64 defect-correction loop around it, with fused inner
// products.  Every kernel runs on a (system, block) grid; a block whose
// system is inactive returns at once.
//
// FP64 / FP32 vectors are streamed one 16-byte word per thread (a system's
// vector is a flat array of NV*n words: double2 = 1 complex, float4 = 2
// complex), so a thread holds a few registers and every access is one
// coalesced 128-bit load or store.  FP16 vectors carry one norm per site and
// are processed one site per thread.
//
// Inner products accumulate per thread and per warp in the kernel's own
// precision (FP32 for the FP32 / FP16 solver: FP64 arithmetic is a small
// fraction of the FP32 rate on this GPU), then in FP64 across the warps of a
// block and across blocks; `k_finalize` sums a system's block partials in a
// fixed order, so every result is deterministic for a given launch shape.  `wps` (words per site) tells the finalize how many blocks the
// producing kernel used per system.
#pragma once

#include "dslash.cuh"

namespace lq {

struct VecArgs {
  const SysDesc* sys;
  const int* active;
  SolverScal* sc;
  double* partial;
  int pstride;
  int nsys;
};

template <typename R>
LQ_DI cx<R> c_of(double2 v) {
  return {(R)v.x, (R)v.y};
}

// ---------------------------------------------------------------- word access
template <int P>
struct Word;
template <>
struct Word<64> {
  typedef double2 T;
  typedef double R;
  static constexpr int NC = 1;  // complex numbers per word
  LQ_DI static void get(const T* p, int i, cx<double> c[1]) {
    T v = __ldg(p + i);
    c[0] = {v.x, v.y};
  }
  LQ_DI static void put(T* p, int i, const cx<double> c[1]) { p[i] = make_double2(c[0].re, c[0].im); }
};
template <>
struct Word<32> {
  typedef float4 T;
  typedef float R;
  static constexpr int NC = 2;
  LQ_DI static void get(const T* p, int i, cx<float> c[2]) {
    T v = __ldg(p + i);
    c[0] = {v.x, v.y};
    c[1] = {v.z, v.w};
  }
  LQ_DI static void put(T* p, int i, const cx<float> c[2]) { p[i] = make_float4(c[0].re, c[0].im, c[1].re, c[1].im); }
};

template <int P>
LQ_DI const typename Word<P>::T* wptr(const void* pool, long long off) {
  return (const typename Word<P>::T*)pool + off * Prec<P>::NV;
}
template <int P>
LQ_DI typename Word<P>::T* wptr_w(void* pool, long long off) {
  return (typename Word<P>::T*)pool + off * Prec<P>::NV;
}

#define LQ_WORD_PROLOGUE(P)                                   \
  int s, by;                                                  \
  grid_pos(va.nsys, s, by);                                   \
  if (va.active && !va.active[s]) return;                     \
  const SysDesc sd = va.sys[s];                               \
  const int nw = sd.n * Prec<P>::NV;                          \
  if (by * (int)blockDim.x >= nw) return;                     \
  const int i = by * blockDim.x + threadIdx.x;                \
  const bool valid = i < nw;

#define LQ_SITE_PROLOGUE                                      \
  int s, by;                                                  \
  grid_pos(va.nsys, s, by);                                   \
  if (va.active && !va.active[s]) return;                     \
  const SysDesc sd = va.sys[s];                               \
  if (by * (int)blockDim.x >= sd.n) return;                   \
  const int j = by * blockDim.x + threadIdx.x;                \
  const bool valid = j < sd.n;

// ------------------------------------------------------------ s = r - alpha v
template <int P>
__global__ void __launch_bounds__(128) k_bicg_s_w(VecArgs va, const void* r, const void* v, void* so) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  if (!valid) return;
  const cx<R> al = c_of<R>(va.sc[s].alpha);
  cx<R> a[W::NC], b[W::NC];
  W::get(wptr<P>(r, sd.off), i, a);
  W::get(wptr<P>(v, sd.off), i, b);
#pragma unroll
  for (int k = 0; k < W::NC; k++) a[k] = a[k] - al * b[k];
  W::put(wptr_w<P>(so, sd.off), i, a);
}

__global__ void __launch_bounds__(128) k_bicg_s_h(VecArgs va, const void* r, const float* rn, const void* v,
                                                  const float* vn, void* so, float* son) {
  LQ_SITE_PROLOGUE
  if (!valid) return;
  const cx<float> al = c_of<float>(va.sc[s].alpha);
  cx<float> a[12], b[12];
  Prec<16>::load(a, sys_ptr<16>(r, sd.off), nrm_ptr(rn, sd.off), sd.n, j);
  Prec<16>::load(b, sys_ptr<16>(v, sd.off), nrm_ptr(vn, sd.off), sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) a[k] = a[k] - al * b[k];
  Prec<16>::store(sys_ptr_w<16>(so, sd.off), nrm_ptr_w(son, sd.off), sd.n, j, a);
}

// ------------------- x += alpha p + omega s ; r = s - omega t ; <r0,r>, |r|^2
template <int P>
__global__ void __launch_bounds__(128) k_bicg_xr_w(VecArgs va, void* x, const void* p, const void* sv, const void* t,
                                                   void* r, const void* r0) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  R red[3] = {0, 0, 0};
  if (valid) {
    const cx<R> al = c_of<R>(va.sc[s].alpha), om = c_of<R>(va.sc[s].omega);
    cx<R> xv[W::NC], pv[W::NC], sv_[W::NC], tv[W::NC], w[W::NC];
    W::get(wptr<P>(x, sd.off), i, xv);
    W::get(wptr<P>(p, sd.off), i, pv);
    W::get(wptr<P>(sv, sd.off), i, sv_);
    W::get(wptr<P>(t, sd.off), i, tv);
    W::get(wptr<P>(r0, sd.off), i, w);
#pragma unroll
    for (int k = 0; k < W::NC; k++) {
      xv[k] = xv[k] + al * pv[k] + om * sv_[k];
      sv_[k] = sv_[k] - om * tv[k];
    }
    W::put(wptr_w<P>(x, sd.off), i, xv);
    W::put(wptr_w<P>(r, sd.off), i, sv_);
#pragma unroll
    for (int k = 0; k < W::NC; k++) {
      red[0] += w[k].re * sv_[k].re + w[k].im * sv_[k].im;
      red[1] += w[k].re * sv_[k].im - w[k].im * sv_[k].re;
      red[2] += sv_[k].re * sv_[k].re + sv_[k].im * sv_[k].im;
    }
  }
  block_reduce_store<3, R>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

__global__ void __launch_bounds__(128) k_bicg_xr_h(VecArgs va, void* x, float* xn, const void* p, const float* pn,
                                                   const void* sv, const float* svn, const void* t, const float* tn,
                                                   void* r, float* rn, const void* r0, const float* r0n) {
  LQ_SITE_PROLOGUE
  float red[3] = {0.f, 0.f, 0.f};
  if (valid) {
    const cx<float> al = c_of<float>(va.sc[s].alpha), om = c_of<float>(va.sc[s].omega);
    cx<float> xv[12], pv[12], sv_[12], tv[12];
    Prec<16>::load(xv, sys_ptr<16>(x, sd.off), nrm_ptr(xn, sd.off), sd.n, j);
    Prec<16>::load(pv, sys_ptr<16>(p, sd.off), nrm_ptr(pn, sd.off), sd.n, j);
    Prec<16>::load(sv_, sys_ptr<16>(sv, sd.off), nrm_ptr(svn, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) xv[k] = xv[k] + al * pv[k] + om * sv_[k];
    Prec<16>::store(sys_ptr_w<16>(x, sd.off), nrm_ptr_w(xn, sd.off), sd.n, j, xv);
    Prec<16>::load(tv, sys_ptr<16>(t, sd.off), nrm_ptr(tn, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) sv_[k] = sv_[k] - om * tv[k];
    Prec<16>::store(sys_ptr_w<16>(r, sd.off), nrm_ptr_w(rn, sd.off), sd.n, j, sv_);
    Prec<16>::quantize(sv_);  // the values just stored
    cx<float> w[12];
    Prec<16>::load(w, sys_ptr<16>(r0, sd.off), nrm_ptr(r0n, sd.off), sd.n, j);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      red[0] += w[k].re * sv_[k].re + w[k].im * sv_[k].im;
      red[1] += w[k].re * sv_[k].im - w[k].im * sv_[k].re;
      red[2] += sv_[k].re * sv_[k].re + sv_[k].im * sv_[k].im;
    }
  }
  block_reduce_store<3, float>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

// ------------------------------------------------- p = r + beta (p - omega v)
template <int P>
__global__ void __launch_bounds__(128) k_bicg_p_w(VecArgs va, void* p, const void* r, const void* v) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  if (!valid) return;
  const cx<R> be = c_of<R>(va.sc[s].beta), om = c_of<R>(va.sc[s].omega);
  cx<R> pv[W::NC], rv[W::NC], vv[W::NC];
  W::get(wptr<P>(p, sd.off), i, pv);
  W::get(wptr<P>(r, sd.off), i, rv);
  W::get(wptr<P>(v, sd.off), i, vv);
#pragma unroll
  for (int k = 0; k < W::NC; k++) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
  W::put(wptr_w<P>(p, sd.off), i, pv);
}

__global__ void __launch_bounds__(128) k_bicg_p_h(VecArgs va, void* p, float* pn, const void* r, const float* rn,
                                                  const void* v, const float* vn) {
  LQ_SITE_PROLOGUE
  if (!valid) return;
  const cx<float> be = c_of<float>(va.sc[s].beta), om = c_of<float>(va.sc[s].omega);
  cx<float> pv[12], rv[12], vv[12];
  Prec<16>::load(pv, sys_ptr<16>(p, sd.off), nrm_ptr(pn, sd.off), sd.n, j);
  Prec<16>::load(rv, sys_ptr<16>(r, sd.off), nrm_ptr(rn, sd.off), sd.n, j);
  Prec<16>::load(vv, sys_ptr<16>(v, sd.off), nrm_ptr(vn, sd.off), sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
  Prec<16>::store(sys_ptr_w<16>(p, sd.off), nrm_ptr_w(pn, sd.off), sd.n, j, pv);
}

// CG on the normal equations (the fallback for systems whose BiCGStab
// stalls): x += alpha p, r -= alpha v (v = D^ p), partial |r|^2 (slot 2).
// alpha is real (stored in alpha.x).
template <int P>
__global__ void __launch_bounds__(128) k_cg_xr_w(VecArgs va, void* x, const void* p, void* r, const void* v) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  R red[3] = {0, 0, 0};
  if (valid) {
    const R al = (R)va.sc[s].alpha.x;
    cx<R> xv[W::NC], pv[W::NC], rv[W::NC], vv[W::NC];
    W::get(wptr<P>(x, sd.off), i, xv);
    W::get(wptr<P>(p, sd.off), i, pv);
    W::get(wptr<P>(r, sd.off), i, rv);
    W::get(wptr<P>(v, sd.off), i, vv);
#pragma unroll
    for (int k = 0; k < W::NC; k++) {
      xv[k] = xv[k] + al * pv[k];
      rv[k] = rv[k] - al * vv[k];
      red[2] += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
    }
    W::put(wptr_w<P>(x, sd.off), i, xv);
    W::put(wptr_w<P>(r, sd.off), i, rv);
  }
  block_reduce_store<3, R>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

// p = z + beta p (beta real, in beta.x); beta = 0 copies z.
template <int P>
__global__ void __launch_bounds__(128) k_cg_p_w(VecArgs va, void* p, const void* z) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  if (!valid) return;
  const R be = (R)va.sc[s].beta.x;
  cx<R> pv[W::NC], zv[W::NC];
  W::get(wptr<P>(z, sd.off), i, zv);
  if (be != (R)0) {
    W::get(wptr<P>(p, sd.off), i, pv);
#pragma unroll
    for (int k = 0; k < W::NC; k++) zv[k] = zv[k] + be * pv[k];
  }
  W::put(wptr_w<P>(p, sd.off), i, zv);
}

// Word i = q*n + j of a precision-P system vector holds the complex numbers
// q*NC .. q*NC+NC-1 of site j; complex c of site j is FP64 word c*n + j.
LQ_DI void split_word(int i, int n, int& q, int& j) {
  q = i / n;
  j = i - q * n;
}

// Start of an inner cycle: r = r0 = p = convert(r64), x = 0; partial |r|^2.
template <int P>
__global__ void __launch_bounds__(128) k_inner_init_w(VecArgs va, const double2* r64, void* r, void* r0, void* p,
                                                      void* x) {
  typedef Word<P> W;
  typedef typename W::R R;
  LQ_WORD_PROLOGUE(P)
  R red[3] = {0, 0, 0};
  if (valid) {
    int q, j;
    split_word(i, sd.n, q, j);
    const double2* src = r64 + sd.off * 12;
    cx<R> b[W::NC], z[W::NC];
#pragma unroll
    for (int k = 0; k < W::NC; k++) {
      double2 v = __ldg(src + (q * W::NC + k) * sd.n + j);
      b[k] = {(R)v.x, (R)v.y};
      z[k] = {0, 0};
      red[2] += b[k].re * b[k].re + b[k].im * b[k].im;
    }
    W::put(wptr_w<P>(r, sd.off), i, b);
    W::put(wptr_w<P>(r0, sd.off), i, b);
    W::put(wptr_w<P>(p, sd.off), i, b);
    W::put(wptr_w<P>(x, sd.off), i, z);
  }
  block_reduce_store<3, R>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

__global__ void __launch_bounds__(128) k_inner_init_h(VecArgs va, const double2* r64, void* r, float* rn, void* r0,
                                                      float* r0n, void* p, float* pn, void* x, float* xn) {
  LQ_SITE_PROLOGUE
  float red[3] = {0.f, 0.f, 0.f};
  if (valid) {
    cx<double> a[12];
    Prec<64>::load(a, sys_ptr<64>(r64, sd.off), nullptr, sd.n, j);
    cx<float> b[12], z[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      b[k] = {(float)a[k].re, (float)a[k].im};
      z[k] = {0, 0};
    }
    Prec<16>::store(sys_ptr_w<16>(r, sd.off), nrm_ptr_w(rn, sd.off), sd.n, j, b);
    Prec<16>::store(sys_ptr_w<16>(r0, sd.off), nrm_ptr_w(r0n, sd.off), sd.n, j, b);
    Prec<16>::store(sys_ptr_w<16>(p, sd.off), nrm_ptr_w(pn, sd.off), sd.n, j, b);
    Prec<16>::store(sys_ptr_w<16>(x, sd.off), nrm_ptr_w(xn, sd.off), sd.n, j, z);
    Prec<16>::quantize(b);  // the values just stored
#pragma unroll
    for (int k = 0; k < 12; k++) red[2] += b[k].re * b[k].re + b[k].im * b[k].im;
  }
  block_reduce_store<3, float>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

// x64 += x (inner solution of precision P).  A cycle that ended in NaN or
// divergence (status 2) contributes nothing.
template <int P>
__global__ void __launch_bounds__(128) k_accum64_w(VecArgs va, double2* x64, const void* x) {
  typedef Word<P> W;
  LQ_WORD_PROLOGUE(P)
  if (!valid || va.sc[s].status == 2) return;
  int q, j;
  split_word(i, sd.n, q, j);
  cx<typename W::R> e[W::NC];
  W::get(wptr<P>(x, sd.off), i, e);
  double2* dst = x64 + sd.off * 12;
#pragma unroll
  for (int k = 0; k < W::NC; k++) {
    const int w = (q * W::NC + k) * sd.n + j;
    double2 a = dst[w];
    dst[w] = make_double2(a.x + (double)e[k].re, a.y + (double)e[k].im);
  }
}

__global__ void __launch_bounds__(128) k_accum64_h(VecArgs va, double2* x64, const void* x, const float* xn) {
  LQ_SITE_PROLOGUE
  if (!valid || va.sc[s].status == 2) return;
  cx<float> e[12];
  Prec<16>::load(e, sys_ptr<16>(x, sd.off), nrm_ptr(xn, sd.off), sd.n, j);
  cx<double> a[12];
  Prec<64>::load(a, sys_ptr<64>(x64, sd.off), nullptr, sd.n, j);
#pragma unroll
  for (int k = 0; k < 12; k++) a[k] = {a[k].re + (double)e[k].re, a[k].im + (double)e[k].im};
  Prec<64>::store(sys_ptr_w<64>(x64, sd.off), nullptr, sd.n, j, a);
}

// |v|^2 partials of an FP64 vector set (word-parallel).
__global__ void __launch_bounds__(128) k_norm2_64(VecArgs va, const double2* v) {
  LQ_WORD_PROLOGUE(64)
  double red[3] = {0.0, 0.0, 0.0};
  if (valid) {
    double2 a = __ldg(v + sd.off * 12 + i);
    red[2] = a.x * a.x + a.y * a.y;
  }
  block_reduce_store<3, double>(red, va.partial + ((long long)s * va.pstride + by) * 4);
}

// Precision conversion of a system vector set, one site per thread.
template <int P1, int P2>
__global__ void __launch_bounds__(128) k_convert(VecArgs va, const void* in, const float* inn, void* out, float* outn) {
  typedef typename Prec<P1>::R R1;
  typedef typename Prec<P2>::R R2;
  LQ_SITE_PROLOGUE
  if (!valid) return;
  cx<R1> a[12];
  Prec<P1>::load(a, sys_ptr<P1>(in, sd.off), nrm_ptr(inn, sd.off), sd.n, j);
  cx<R2> b[12];
#pragma unroll
  for (int k = 0; k < 12; k++) b[k] = {(R2)a[k].re, (R2)a[k].im};
  Prec<P2>::store(sys_ptr_w<P2>(out, sd.off), nrm_ptr_w(outn, sd.off), sd.n, j, b);
}

// ---------------------------------------------------------------- finalize
// Sum of the block partials of system s = blockIdx.x, in a fixed order: each
// thread of the block sums a strided subset, the warps reduce by shuffles and
// warp 0 adds the warp sums in warp order.  Thread 0 receives the result.
constexpr int FIN_THREADS = 512;
LQ_DI void block_sum_partials(const double* partial, int pstride, int nb, int s, double out[3]) {
  __shared__ double sh[FIN_THREADS / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double* q = partial + ((long long)s * pstride + b) * 4;
    v[0] += q[0];
    v[1] += q[1];
    v[2] += q[2];
  }
#pragma unroll
  for (int q = 0; q < 3; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 3; q++) sh[wid][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < 3; q++) {
      double t = 0.0;
      for (int w = 0; w < nw; w++) t += sh[w][q];
      out[q] = t;
    }
  }
}

LQ_DI double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
LQ_DI double2 cmul2(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
LQ_DI bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// One block per system: fold the block partials into the iteration scalars.
//  FIN_INIT : rr = rho = |r|^2, rr0 = rr, iters = 0, target2 = max(tau2*rr, floor2)
//  FIN_ALPHA: alpha = rho / <r0, v>
//  FIN_OMEGA: omega = <t, s> / |t|^2
//  FIN_BETA : rr = |r|^2, rho' = <r0, r>; stop the system when rr <= target2,
//             on breakdown, NaN or divergence (rr > 1e8 rr0); else
//             beta = (rho'/rho)(alpha/omega)
//  FIN_NORM : rr = |r|^2 only
//  CG on the normal equations (real scalars in .x):
//  FIN_CG_RHO  : rho = |z|^2 (z = D^dag r), beta = 0 (the first direction is z)
//  FIN_CG_ALPHA: alpha = rho / |v|^2 (v = D^ p); breakdown if |v|^2 is not positive
//  FIN_CG_R    : rr = |r|^2; stop the system when rr <= target2, on NaN or divergence
//  FIN_CG_BETA : beta = |z|^2 / rho, rho = |z|^2
// tau2 / floor_rel2 are per call (FIN_INIT); floor_rel2 is relative to bb.
// wps: words per site of the kernel that wrote the partials (1: one site per
// thread), so that the system used ceil(n * wps / bdim) blocks.
__global__ void k_finalize(int mode, int nsys, const SysDesc* sys, int* active, SolverScal* sc, const double* partial,
                           int pstride, int wps, int bdim, double tau2, double floor_rel2) {
  const int s = blockIdx.x;
  if (s >= nsys) return;
  if (active && !active[s]) return;  // uniform over the block
  const int nb = (sys[s].n * wps + bdim - 1) / bdim;
  double v[3];
  block_sum_partials(partial, pstride, nb, s, v);
  if (threadIdx.x != 0) return;
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
    case FIN_CG_RHO:
      c.rho = make_double2(v[2], 0.0);
      c.beta = make_double2(0.0, 0.0);
      break;
    case FIN_CG_ALPHA:
      if (!(v[2] > 0.0) || !isfinite(v[2]) || !(c.rho.x > 0.0)) {
        c.status = 1;
        active[s] = 0;
      } else {
        c.alpha = make_double2(c.rho.x / v[2], 0.0);
      }
      break;
    case FIN_CG_R:
      c.iters += 1;
      c.rr = v[2];
      if (!isfinite(v[2]) || v[2] > 1e8 * c.rr0) {
        c.status = 2;
        active[s] = 0;
      } else if (v[2] <= c.target2) {
        active[s] = 0;
      }
      break;
    case FIN_CG_BETA:
      if (!(c.rho.x > 0.0) || !isfinite(v[2])) {
        c.status = 1;
        active[s] = 0;
      } else {
        c.beta = make_double2(v[2] / c.rho.x, 0.0);
        c.rho = make_double2(v[2], 0.0);
      }
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

}  // namespace lq
