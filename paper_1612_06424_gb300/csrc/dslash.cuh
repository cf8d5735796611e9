// Wilson hopping term with fused clover / linear-combination epilogues and
// fused per-system inner products.
//
//   (D_hop psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
//                         + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)
//   D = A - D_hop / 2,  A = 1/(2 kappa) + clover   (2 kappa D = 1 - kappa D_hop)
//
// Each (1 +- g_mu) has rank 2, so psi is projected to a half spinor h
// (2 spins x 3 colours), multiplied by the link (2 SU(3) mat-vecs instead
// of 4) and expanded back.  D^dag = g5 D g5 swaps the two projectors; A is
// Hermitian.  A hop whose target lies outside the system's slab is dropped
// (Dirichlet block operator, the exact sub-block of D); a hop across the
// time boundary is dropped (open BC) or wraps with sign +-1 when the slab
// is the whole lattice with periodic / antiperiodic BC.
#pragma once

#include "common.cuh"

namespace lq {

// h = upper half of (1 + S g_mu) psi.  psi[3*s + c].
template <int MU, int S, typename R>
LQ_DI void project(const cx<R> p[12], cx<R> h[6]) {
  const R s = (R)S;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    if (MU == 0) {
      h[c] = p[c] - s * p[6 + c];
      h[3 + c] = p[3 + c] - s * p[9 + c];
    } else if (MU == 1) {
      h[c] = p[c] - s * ti(p[9 + c]);
      h[3 + c] = p[3 + c] - s * ti(p[6 + c]);
    } else if (MU == 2) {
      h[c] = p[c] - s * p[9 + c];
      h[3 + c] = p[3 + c] + s * p[6 + c];
    } else {
      h[c] = p[c] - s * ti(p[6 + c]);
      h[3 + c] = p[3 + c] + s * ti(p[9 + c]);
    }
  }
}

// acc += (1 + S g_mu) expanded from the transported half spinor w.
template <int MU, int S, typename R>
LQ_DI void expand_add(cx<R> acc[12], const cx<R> w[6]) {
  const R s = (R)S;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = acc[c] + w[c];
    acc[3 + c] = acc[3 + c] + w[3 + c];
    if (MU == 0) {
      acc[6 + c] = acc[6 + c] - s * w[c];
      acc[9 + c] = acc[9 + c] - s * w[3 + c];
    } else if (MU == 1) {
      acc[6 + c] = acc[6 + c] + s * ti(w[3 + c]);
      acc[9 + c] = acc[9 + c] + s * ti(w[c]);
    } else if (MU == 2) {
      acc[6 + c] = acc[6 + c] + s * w[3 + c];
      acc[9 + c] = acc[9 + c] - s * w[c];
    } else {
      acc[6 + c] = acc[6 + c] + s * ti(w[c]);
      acc[9 + c] = acc[9 + c] - s * ti(w[3 + c]);
    }
  }
}

template <typename R>
LQ_DI void mul_u(const su3<R>& u, const cx<R> h[6], cx<R> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; sp++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> t = u.m[a][0] * h[3 * sp];
      fma_c(t, u.m[a][1], h[3 * sp + 1]);
      fma_c(t, u.m[a][2], h[3 * sp + 2]);
      w[3 * sp + a] = t;
    }
}

template <typename R>
LQ_DI void mul_udag(const su3<R>& u, const cx<R> h[6], cx<R> w[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; sp++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> t = cmulc(u.m[0][a], h[3 * sp]);
      fma_cc(t, u.m[1][a], h[3 * sp + 1]);
      fma_cc(t, u.m[2][a], h[3 * sp + 2]);
      w[3 * sp + a] = t;
    }
}

// Neighbour spinor fetch of the stencil: (local index, window hint) -> psi.
// Window hints: 0 the site's own row (x2, x3 hops), 1 / 2 the rows at
// x1 -+ 1, 3 / 4 the rows at x0 -+ 1.
template <int P>
struct GlobalFetch {
  const void* in;
  const float* inn;
  int n;
  LQ_DI void operator()(int q, int, cx<typename Prec<P>::R> psi[12]) const { Prec<P>::load(psi, in, inn, n, q); }
};

template <int P, bool DAG, int MU, typename Fetch>
LQ_DI void hop_dir_f(const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, const int x[4],
                     const Fetch& fetch, cx<typename Prec<P>::R> acc[12]) {
  typedef typename Prec<P>::R R;
  constexpr int SF = DAG ? +1 : -1;  // forward projector (1 + SF g_mu)
  constexpr int SB = -SF;           // backward projector
  const int pin = pout ^ 1;
  // ---- forward: U_mu(x) psi(x + mu)
  {
    int y[4] = {x[0], x[1], x[2], x[3]};
    bool ok = true;
    R sgn = (R)1;
    if (MU == 0) {
      if (x[0] == sd.t1) {
        ok = sd.wrap;
        y[0] = 0;
        sgn = (R)sd.tsign;
      } else {
        y[0] = x[0] + 1;
      }
    } else {
      y[MU] = (x[MU] + 1 == g.L[MU]) ? 0 : x[MU] + 1;
    }
    if (ok) {
      const int cy = eo_index(g, y);
      cx<R> psi[12], h[6], w[6];
      fetch(cy - sd.cb0, MU == 0 ? 4 : MU == 1 ? 2 : 0, psi);
      project<MU, SF>(psi, h);
      su3<R> u = LinkIO<P>::load(f, pout, MU, g.Vh, cb);
      mul_u(u, h, w);
      if (MU == 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) w[k] = sgn * w[k];
      }
      expand_add<MU, SF>(acc, w);
    }
  }
  // ---- backward: U_mu(x - mu)^dag psi(x - mu)
  {
    int y[4] = {x[0], x[1], x[2], x[3]};
    bool ok = true;
    R sgn = (R)1;
    if (MU == 0) {
      if (x[0] == sd.t0) {
        ok = sd.wrap;
        y[0] = g.L[0] - 1;
        sgn = (R)sd.tsign;
      } else {
        y[0] = x[0] - 1;
      }
    } else {
      y[MU] = (x[MU] == 0) ? g.L[MU] - 1 : x[MU] - 1;
    }
    if (ok) {
      const int cy = eo_index(g, y);
      cx<R> psi[12], h[6], w[6];
      fetch(cy - sd.cb0, MU == 0 ? 3 : MU == 1 ? 1 : 0, psi);
      project<MU, SB>(psi, h);
      su3<R> u = LinkIO<P>::load(f, pin, MU, g.Vh, cy);
      mul_udag(u, h, w);
      if (MU == 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) w[k] = sgn * w[k];
      }
      expand_add<MU, SB>(acc, w);
    }
  }
}

template <int P, bool DAG, int MU>
LQ_DI void hop_dir(const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, const int x[4],
                   const void* in, const float* inn, cx<typename Prec<P>::R> acc[12]) {
  hop_dir_f<P, DAG, MU>(g, sd, f, pout, cb, x, GlobalFetch<P>{in, inn, sd.n}, acc);
}

template <int P, bool DAG, typename Fetch>
LQ_DI void hop_sum_f(const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, const int x[4],
                     const Fetch& fetch, cx<typename Prec<P>::R> acc[12]) {
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0, 0};
  hop_dir_f<P, DAG, 0>(g, sd, f, pout, cb, x, fetch, acc);
  hop_dir_f<P, DAG, 1>(g, sd, f, pout, cb, x, fetch, acc);
  hop_dir_f<P, DAG, 2>(g, sd, f, pout, cb, x, fetch, acc);
  hop_dir_f<P, DAG, 3>(g, sd, f, pout, cb, x, fetch, acc);
}

// ---------------------------------------------------------------------------
// Software-pipelined hop sum (FP32 / FP16).  The eight hops are taken in a
// fixed order k = 2*mu + (0 forward, 1 backward); the raw words of hop k+D
// (neighbour spinor and link, as stored) are loaded before hop k is
// computed, so up to D hops' loads are in flight while the thread does
// arithmetic.  Loads are unconditional: a hop that leaves the slab (or
// crosses the open time boundary) reads the thread's own in-range words and
// is then weighted by 0, so the pipeline has no branches.
#ifndef LQ_HOP_PIPE
#define LQ_HOP_PIPE 1
#endif

template <int P>
struct HopRaw;
template <>
struct HopRaw<32> {
  float4 s[6];
  float4 u[3];
};
template <>
struct HopRaw<16> {
  uint4 s[3];
  float nu;
  uint2 u[3];
};

// Pipeline depth per precision (hops whose loads are in flight while one is
// computed): bounded by the register cap of the stencil kernels.  FP32 depth
// 2 at 4 blocks per SM measured best on GB300 (depth 1: -3%; depth 2 or 3 at
// 3 blocks per SM: -5% and -13%).
#ifndef LQ_HOP_DEPTH32
#define LQ_HOP_DEPTH32 2
#endif
#ifndef LQ_HOP_DEPTH16
#define LQ_HOP_DEPTH16 2
#endif
template <int P>
struct HopDepth {
  static constexpr int value = P == 16 ? LQ_HOP_DEPTH16 : LQ_HOP_DEPTH32;
};

LQ_DI void raw_load(HopRaw<32>& r, const void* in, const float*, int n, int q, const FieldPtrs& f, int p, int mu,
                    int Vh, int cl) {
  const float4* sp = (const float4*)in + q;
#pragma unroll
  for (int k = 0; k < 6; k++) r.s[k] = __ldg(sp + k * n);
  const float4* b = f.U32 + (p * 4 + mu) * 3 * Vh + cl;
#pragma unroll
  for (int k = 0; k < 3; k++) r.u[k] = ld_once(b + k * Vh);
}
LQ_DI void raw_load(HopRaw<16>& r, const void* in, const float* inn, int n, int q, const FieldPtrs& f, int p, int mu,
                    int Vh, int cl) {
  const uint4* sp = (const uint4*)in + q;
#pragma unroll
  for (int k = 0; k < 3; k++) r.s[k] = __ldg(sp + k * n);
  r.nu = __ldg(inn + q);
  const uint2* b = f.U16 + (p * 4 + mu) * 3 * Vh + cl;
#pragma unroll
  for (int k = 0; k < 3; k++) r.u[k] = ld_once(b + k * Vh);
}

LQ_DI void raw_spinor(const HopRaw<32>& r, cx<float> s[12]) {
#pragma unroll
  for (int k = 0; k < 6; k++) {
    s[2 * k] = {r.s[k].x, r.s[k].y};
    s[2 * k + 1] = {r.s[k].z, r.s[k].w};
  }
}
LQ_DI void raw_spinor(const HopRaw<16>& r, cx<float> s[12]) {
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const uint32_t w[4] = {r.s[k].x, r.s[k].y, r.s[k].z, r.s[k].w};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
      s[4 * k + q] = {v.x * r.nu, v.y * r.nu};
    }
  }
}

LQ_DI su3<float> raw_link(const HopRaw<32>& r) {
  su3<float> u;
  u.m[0][0] = {r.u[0].x, r.u[0].y};
  u.m[0][1] = {r.u[0].z, r.u[0].w};
  u.m[0][2] = {r.u[1].x, r.u[1].y};
  u.m[1][0] = {r.u[1].z, r.u[1].w};
  u.m[1][1] = {r.u[2].x, r.u[2].y};
  u.m[1][2] = {r.u[2].z, r.u[2].w};
  reconstruct_row2(u);
  return u;
}
LQ_DI su3<float> raw_link(const HopRaw<16>& r) {
  su3<float> u;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.u[k].x));
    float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.u[k].y));
    u.m[(2 * k) / 3][(2 * k) % 3] = {a.x, a.y};
    u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = {b.x, b.y};
  }
  reconstruct_row2(u);
  return u;
}

// Where hop k reads: neighbour index q within the system's input vector,
// link site and parity, and the weight (0 for a dropped hop, +-1 else).
struct HopTgt {
  int q, cl, pl;
  float w;
};

template <int K>
LQ_DI HopTgt hop_target(const Geom& g, const SysDesc& sd, int pout, int cb, int j, const int x[4]) {
  constexpr int MU = K >> 1;
  constexpr bool FWD = (K & 1) == 0;
  int y[4] = {x[0], x[1], x[2], x[3]};
  bool ok = true;
  float sgn = 1.f;
  if (MU == 0) {
    if (FWD) {
      if (x[0] == sd.t1) {
        ok = sd.wrap;
        y[0] = 0;
        sgn = sd.tsign;
      } else {
        y[0] = x[0] + 1;
      }
    } else {
      if (x[0] == sd.t0) {
        ok = sd.wrap;
        y[0] = g.L[0] - 1;
        sgn = sd.tsign;
      } else {
        y[0] = x[0] - 1;
      }
    }
  } else if (FWD) {
    y[MU] = (x[MU] + 1 == g.L[MU]) ? 0 : x[MU] + 1;
  } else {
    y[MU] = (x[MU] == 0) ? g.L[MU] - 1 : x[MU] - 1;
  }
  HopTgt t;
  const int cy = eo_index(g, y);
  t.q = ok ? cy - sd.cb0 : j;
  t.cl = FWD ? cb : (ok ? cy : cb);
  t.pl = FWD ? pout : pout ^ 1;
  t.w = ok ? sgn : 0.f;
  return t;
}

template <int P, int K>
LQ_DI void raw_fetch(HopRaw<P>& r, const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, int j,
                     const int x[4], const void* in, const float* inn) {
  const HopTgt t = hop_target<K>(g, sd, pout, cb, j, x);
  raw_load(r, in, inn, sd.n, t.q, f, t.pl, K >> 1, g.Vh, t.cl);
}

// Packed FP32 pairs (f32x2 arithmetic of sm_100+): one instruction operates
// on two FP32 values held in an aligned register pair.
typedef unsigned long long f2_t;
LQ_DI f2_t f2_pack(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
LQ_DI void f2_unpack(f2_t r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
LQ_DI f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
LQ_DI f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// LQ_HOP_PACK 1: the FP32 / FP16 hop sum transports and accumulates spin
// pairs with f32x2 arithmetic (measured 2-6% faster on GB300 than scalar
// FP32); 0: scalar.
#ifndef LQ_HOP_PACK
#define LQ_HOP_PACK 1
#endif
// Colour transport of the two spins of a half spinor with packed pairs: the
// pair index is the spin, so one link element (broadcast to both halves)
// multiplies both spins in one instruction.  w[sp][a] = sum_c U[a][c] h[sp][c]
// (forward) or sum_c conj(U[c][a]) h[sp][c] (backward).
template <bool FWD>
LQ_DI void mul_u_pairs(const su3<float>& u, const cx<float> h[6], f2_t wr[3], f2_t wi[3]) {
  f2_t hr[3], hi[3], hn[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    hr[c] = f2_pack(h[c].re, h[3 + c].re);
    hi[c] = f2_pack(h[c].im, h[3 + c].im);
    hn[c] = f2_pack(FWD ? -h[c].im : -h[c].re, FWD ? -h[3 + c].im : -h[3 + c].re);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    f2_t r = 0ull, i = 0ull;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const cx<float> e = FWD ? u.m[a][c] : u.m[c][a];
      const f2_t br = f2_pack(e.re, e.re), bi = f2_pack(e.im, e.im);
      if (FWD) {  // (er + i ei)(hr + i hi)
        r = c ? f2_fma(br, hr[c], r) : f2_mul(br, hr[c]);
        r = f2_fma(bi, hn[c], r);
        i = c ? f2_fma(br, hi[c], i) : f2_mul(br, hi[c]);
        i = f2_fma(bi, hr[c], i);
      } else {  // (er - i ei)(hr + i hi)
        r = c ? f2_fma(br, hr[c], r) : f2_mul(br, hr[c]);
        r = f2_fma(bi, hi[c], r);
        i = c ? f2_fma(br, hi[c], i) : f2_mul(br, hi[c]);
        i = f2_fma(bi, hn[c], i);
      }
    }
    wr[a] = r;
    wi[a] = i;
  }
}

LQ_DI f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
LQ_DI f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Accumulator of the packed hop sum: for colour a the spin pairs
// (acc[s=0][a], acc[s=1][a]) and (acc[2][a], acc[3][a]), real and imaginary.
struct AccP {
  f2_t ur[3], ui[3], lr[3], li[3];
};

// acc += (1 + S g_mu) expanded from the transported half spinor w (pairs).
template <int MU, int S>
LQ_DI void expand_add_p(AccP& A, const f2_t wr[3], const f2_t wi[3]) {
  const float s = (float)S;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    A.ur[c] = f2_add(A.ur[c], wr[c]);
    A.ui[c] = f2_add(A.ui[c], wi[c]);
    if (MU == 0) {  // lower += -s (w0, w1)
      A.lr[c] = S > 0 ? f2_sub(A.lr[c], wr[c]) : f2_add(A.lr[c], wr[c]);
      A.li[c] = S > 0 ? f2_sub(A.li[c], wi[c]) : f2_add(A.li[c], wi[c]);
    } else if (MU == 3) {  // lower += (s, -s) i (w0, w1)
      A.lr[c] = f2_fma(f2_pack(-s, s), wi[c], A.lr[c]);
      A.li[c] = f2_fma(f2_pack(s, -s), wr[c], A.li[c]);
    } else {  // spins swapped: scalar updates of the pair halves
      float l0r, l1r, l0i, l1i, w0r, w1r, w0i, w1i;
      f2_unpack(A.lr[c], l0r, l1r);
      f2_unpack(A.li[c], l0i, l1i);
      f2_unpack(wr[c], w0r, w1r);
      f2_unpack(wi[c], w0i, w1i);
      if (MU == 1) {  // lower0 += s i w1, lower1 += s i w0
        l0r -= s * w1i;
        l0i += s * w1r;
        l1r -= s * w0i;
        l1i += s * w0r;
      } else {  // MU == 2: lower0 += s w1, lower1 -= s w0
        l0r += s * w1r;
        l0i += s * w1i;
        l1r -= s * w0r;
        l1i -= s * w0i;
      }
      A.lr[c] = f2_pack(l0r, l1r);
      A.li[c] = f2_pack(l0i, l1i);
    }
  }
}

// Hop k from its raw words: acc += weight * (1 -+ g_mu) U psi (forward) or
// (1 +- g_mu) U^dag psi (backward).
template <int P, bool DAG, int K>
LQ_DI void hop_apply(const HopRaw<P>& r, float wgt, cx<float> (&acc)[12]) {
  constexpr int MU = K >> 1;
  constexpr bool FWD = (K & 1) == 0;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int S = FWD ? SF : -SF;
  cx<float> h[6], w[6];
  {
    cx<float> psi[12];
    raw_spinor(r, psi);
    project<MU, S>(psi, h);
  }
  const su3<float> u = raw_link(r);
  if (FWD)
    mul_u(u, h, w);
  else
    mul_udag(u, h, w);
  if (MU == 0) {
#pragma unroll
    for (int k = 0; k < 6; k++) w[k] = wgt * w[k];
  }
  expand_add<MU, S>(acc, w);
}

// hop_apply with the packed accumulator.
template <int P, bool DAG, int K>
LQ_DI void hop_apply(const HopRaw<P>& r, float wgt, AccP& A) {
  constexpr int MU = K >> 1;
  constexpr bool FWD = (K & 1) == 0;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int S = FWD ? SF : -SF;
  cx<float> h[6];
  {
    cx<float> psi[12];
    raw_spinor(r, psi);
    project<MU, S>(psi, h);
  }
  const su3<float> u = raw_link(r);
  f2_t wr[3], wi[3];
  mul_u_pairs<FWD>(u, h, wr, wi);
  if (MU == 0) {
    const f2_t bw = f2_pack(wgt, wgt);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      wr[c] = f2_mul(bw, wr[c]);
      wi[c] = f2_mul(bw, wi[c]);
    }
  }
  expand_add_p<MU, S>(A, wr, wi);
}

// One step of the pipeline: issue the loads of hop K + D, then compute hop K.
// Only the time hops (K = 0, 1) carry a weight other than 1.
template <int P, bool DAG, int K, int D, typename ACC>
LQ_DI void hop_pipe_step(HopRaw<P> (&buf)[D + 1], const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout,
                         int cb, int j, const int x[4], const void* in, const float* inn, float w0, float w1,
                         ACC& acc) {
  if constexpr (K + D < 8) raw_fetch<P, K + D>(buf[(K + D) % (D + 1)], g, sd, f, pout, cb, j, x, in, inn);
  hop_apply<P, DAG, K>(buf[K % (D + 1)], K == 0 ? w0 : w1, acc);
  if constexpr (K + 1 < 8) hop_pipe_step<P, DAG, K + 1, D>(buf, g, sd, f, pout, cb, j, x, in, inn, w0, w1, acc);
}

template <int P, bool DAG, int D>
LQ_DI void hop_sum_pipe(const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, int j, const int x[4],
                        const void* in, const float* inn, cx<float> acc[12]) {
  HopRaw<P> buf[D + 1];
  raw_fetch<P, 0>(buf[0], g, sd, f, pout, cb, j, x, in, inn);
  if constexpr (D > 1) raw_fetch<P, 1>(buf[1], g, sd, f, pout, cb, j, x, in, inn);
  if constexpr (D > 2) raw_fetch<P, 2>(buf[2], g, sd, f, pout, cb, j, x, in, inn);
  static_assert(D >= 1 && D <= 3, "pipeline depth");
  const float w0 = hop_target<0>(g, sd, pout, cb, j, x).w, w1 = hop_target<1>(g, sd, pout, cb, j, x).w;
  if constexpr (LQ_HOP_PACK) {
    AccP A;
#pragma unroll
    for (int c = 0; c < 3; c++) A.ur[c] = A.ui[c] = A.lr[c] = A.li[c] = 0ull;
    hop_pipe_step<P, DAG, 0, D>(buf, g, sd, f, pout, cb, j, x, in, inn, w0, w1, A);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      f2_unpack(A.ur[c], acc[c].re, acc[3 + c].re);
      f2_unpack(A.ui[c], acc[c].im, acc[3 + c].im);
      f2_unpack(A.lr[c], acc[6 + c].re, acc[9 + c].re);
      f2_unpack(A.li[c], acc[6 + c].im, acc[9 + c].im);
    }
  } else {
    cx<float>(&a12)[12] = *reinterpret_cast<cx<float>(*)[12]>(acc);
#pragma unroll
    for (int k = 0; k < 12; k++) a12[k] = {0.f, 0.f};
    hop_pipe_step<P, DAG, 0, D>(buf, g, sd, f, pout, cb, j, x, in, inn, w0, w1, a12);
  }
}

template <int P, bool DAG, int D = HopDepth<P>::value>
LQ_DI void hop_sum(const Geom& g, const SysDesc& sd, const FieldPtrs& f, int pout, int cb, int j, const int x[4],
                   const void* in, const float* inn, cx<typename Prec<P>::R> acc[12]) {
  if constexpr ((P == 32 || P == 16) && LQ_HOP_PIPE)
    hop_sum_pipe<P, DAG, D>(g, sd, f, pout, cb, j, x, in, inn, acc);
  else
    hop_sum_f<P, DAG>(g, sd, f, pout, cb, x, GlobalFetch<P>{in, inn, sd.n}, acc);
}

// Clover block apply (A or A^{-1}) on a full spinor.
template <int P>
LQ_DI void clover_apply(const FieldPtrs& f, bool inverse, int p, int Vh, int cb, const cx<typename Prec<P>::R> in[12],
                        cx<typename Prec<P>::R> out[12]) {
  if constexpr (P == 64) {
    const double2* base = inverse ? f.Ai64 : f.A64 + p * 36 * Vh;
    ClovIO<64>::apply(base, Vh, cb, in, out);
    ClovIO<64>::apply(base + 18 * Vh, Vh, cb, in + 6, out + 6);
  } else {
    const float4* base = inverse ? f.Ai32 : f.A32 + p * 18 * Vh;
    ClovIO<32>::apply(base, Vh, cb, in, out);
    ClovIO<32>::apply(base + 9 * Vh, Vh, cb, in + 6, out + 6);
  }
}

// Arguments of the hop kernels.  Vector pointers are pool bases; system s
// uses words [off*NV, (off+n)*NV) of each pool (norms: [off, off+n)).
struct HopArgs {
  Geom g;
  const SysDesc* sys;
  const FieldPtrs* fields;
  const int* active;  // per-system flag (NULL: all active)
  int pout;           // output parity
  const void* x;      // hop input, parity pout^1
  const float* xn;
  const void* y;      // clover-term input, parity pout
  const float* yn;
  const void* z;      // additive term, parity pout
  const float* zn;
  const void* w;      // inner-product partner (RED_DOT_W)
  const float* wn;
  void* out;
  float* outn;
  double alpha, beta, gamma, diag;  // see the kernels
  double* partial;                  // [nsys][pstride][4]
  int pstride;
  int nsys;                         // systems of the (linearised) grid
  int nby;                          // site blocks per system in the grid
  int tile;                         // blocks per time tile of the grid order (0: systems fastest)
  int tblk;                         // 1: a block covers 32 sites x 4 time slices (site_of_block)
};

// Epilogue terms present (compile time): D_hop x, A y, z.
enum { EPI_X = 1, EPI_Y = 2, EPI_Z = 4 };

// Registers are capped so that HopMinBlocks<P> blocks of 128 threads fit on
// an SM: the FP32 / FP16 stencil is latency-bound, and occupancy together
// with the hop pipeline is what hides its loads (with the depth-2 pipeline,
// 4 blocks measured best for FP32 on GB300: 5 blocks spill and lose 10%;
// LQ_HOP_MINB overrides both for experiments).  FP64 is ALU-bound and left
// uncapped (a cap makes it spill).
template <int P>
struct HopMinBlocks {
#ifdef LQ_HOP_MINB
  static constexpr int value = P == 64 ? 1 : LQ_HOP_MINB;
#else
  static constexpr int value = P == 64 ? 1 : P == 32 ? 4 : 5;
#endif
};

// Launch configurations of the one-thread-per-site stencil that the autotuner
// chooses from (lq_tune_hop): CFG 0 is the default above; CFG 1 and 2 trade
// blocks per SM (the register cap) against the depth of the hop pipeline.
// FP64 has the default only.
template <int P, int CFG>
struct HopCfg {
  static constexpr int minb = HopMinBlocks<P>::value;
  static constexpr int depth = HopDepth<P>::value;
};
template <>
struct HopCfg<32, 1> {
  static constexpr int minb = 3, depth = 3;
};
template <>
struct HopCfg<32, 2> {
  static constexpr int minb = 5, depth = 1;
};
template <>
struct HopCfg<16, 1> {
  static constexpr int minb = 4, depth = 3;
};
template <>
struct HopCfg<16, 2> {
  static constexpr int minb = 6, depth = 1;
};
constexpr int kHopCfgs = 3;

struct HopArgs;
// alternative configurations of the forward stencil (hop_tuned*.cu), cfg 1 or 2
template <int P>
int hop_lin_tuned(int cfg, bool clov, int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st);
template <int P>
int hop_clinv_tuned(int cfg, bool clov, int epi, dim3 gr, const HopArgs& a, cudaStream_t st);

// Block reduction of NQ per-thread partial sums of type A (the kernel's own
// precision: FP32 for the FP32 / FP16 solver, whose FP64 rate on this GPU is a
// small fraction of its FP32 rate) through a warp-shuffle tree; the per-warp
// sums are widened to FP64 and combined in FP64, and one partial per block is
// stored.  The order is fixed, so results are deterministic.
template <int NQ, typename A>
LQ_DI void block_reduce_store(A v[NQ], double* dst) {
  __shared__ double sh[32][NQ > 0 ? NQ : 1];
#pragma unroll
  for (int q = 0; q < NQ; q++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; q++) sh[wid][q] = (double)v[q];
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
      double t = lane < nw ? sh[lane][q] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) dst[q] = t;
    }
  }
}

template <int P>
LQ_DI const void* sys_ptr(const void* pool, long long off) {
  return pool ? (const void*)((const char*)pool + off * (long long)Prec<P>::NV * 16) : nullptr;
}
template <int P>
LQ_DI void* sys_ptr_w(void* pool, long long off) {
  return pool ? (void*)((char*)pool + off * (long long)Prec<P>::NV * 16) : nullptr;
}
LQ_DI const float* nrm_ptr(const float* pool, long long off) { return pool ? pool + off : nullptr; }
LQ_DI float* nrm_ptr_w(float* pool, long long off) { return pool ? pool + off : nullptr; }

// out = beta * A(y) + alpha * D_hop x + gamma * z   on parity pout
// (terms present per EPI; A = diag * 1 without clover), with an optional
// fused per-system reduction over the stored values:
//   RED_DOT_W: <w, out> (slots 0,1);  RED_TS: <out, y> (0,1) and |out|^2 (2);
//   RED_NORM: |out|^2 (slot 2).
template <int P, bool DAG, bool CLOV, int RED, int EPI, int CFG = 0>
__global__ void __launch_bounds__(128, (HopCfg<P, CFG>::minb)) k_hop_lin(HopArgs a) {
  typedef typename Prec<P>::R R;
  int s, by;
  grid_pos_tiled((int)blockIdx.x, a.nsys, a.nby, a.tile, s, by);
  if (s >= a.nsys) return;
  if (a.active && !a.active[s]) return;
  const SysDesc sd = a.sys[s];
  if (by * (int)blockDim.x >= sd.n) return;  // whole block beyond this system
  const int j = site_of_block(a.tblk, a.g.S3h, by, threadIdx.x);
  const FieldPtrs f = a.fields[sd.field];
  R red[3] = {0, 0, 0};
  if (j < sd.n) {
    const int cb = sd.cb0 + j;
    cx<R> res[12];
    if (EPI & EPI_X) {
      int x[4];
      eo_coords(a.g, cb, a.pout, x);
      hop_sum<P, DAG, HopCfg<P, CFG>::depth>(a.g, sd, f, a.pout, cb, j, x, sys_ptr<P>(a.x, sd.off),
                                             nrm_ptr(a.xn, sd.off), res);
      const R al = (R)a.alpha;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = al * res[k];
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = {0, 0};
    }
    cx<R> yv[12];
    if ((EPI & EPI_Y) || RED == RED_TS) Prec<P>::load(yv, sys_ptr<P>(a.y, sd.off), nrm_ptr(a.yn, sd.off), sd.n, j);
    if (EPI & EPI_Y) {
      cx<R> ay[12];
      if (CLOV) {
        clover_apply<P>(f, false, a.pout, a.g.Vh, cb, yv, ay);
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) ay[k] = (R)a.diag * yv[k];
      }
      const R be = (R)a.beta;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = res[k] + be * ay[k];
    }
    if (EPI & EPI_Z) {
      cx<R> zv[12];
      Prec<P>::load(zv, sys_ptr<P>(a.z, sd.off), nrm_ptr(a.zn, sd.off), sd.n, j);
      const R ga = (R)a.gamma;
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = res[k] + ga * zv[k];
    }
    Prec<P>::store(sys_ptr_w<P>(a.out, sd.off), nrm_ptr_w(a.outn, sd.off), sd.n, j, res);
    if (RED != RED_NONE) {
      Prec<P>::quantize(res);  // reduce over the stored (rounded) values
      if (RED == RED_DOT_W) {
        cx<R> wv[12];
        Prec<P>::load(wv, sys_ptr<P>(a.w, sd.off), nrm_ptr(a.wn, sd.off), sd.n, j);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          red[0] += wv[k].re * res[k].re + wv[k].im * res[k].im;
          red[1] += wv[k].re * res[k].im - wv[k].im * res[k].re;
        }
      } else if (RED == RED_TS) {
#pragma unroll
        for (int k = 0; k < 12; k++) {
          red[0] += res[k].re * yv[k].re + res[k].im * yv[k].im;
          red[1] += res[k].re * yv[k].im - res[k].im * yv[k].re;
          red[2] += res[k].re * res[k].re + res[k].im * res[k].im;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) red[2] += res[k].re * res[k].re + res[k].im * res[k].im;
      }
    }
  }
  if (RED != RED_NONE) block_reduce_store<3, R>(red, a.partial + ((long long)s * a.pstride + by) * 4);
}

// out = A^{-1} (alpha * D_hop x + beta * y) on even sites (pout = 0), terms
// present per EPI (EPI_X, EPI_Y); A^{-1} = 1/diag without clover.
template <int P, bool DAG, bool CLOV, int EPI, int CFG = 0>
__global__ void __launch_bounds__(128, (HopCfg<P, CFG>::minb)) k_hop_clinv(HopArgs a) {
  typedef typename Prec<P>::R R;
  int s, by;
  grid_pos_tiled((int)blockIdx.x, a.nsys, a.nby, a.tile, s, by);
  if (s >= a.nsys) return;
  if (a.active && !a.active[s]) return;
  const SysDesc sd = a.sys[s];
  if (by * (int)blockDim.x >= sd.n) return;
  const int j = site_of_block(a.tblk, a.g.S3h, by, threadIdx.x);
  const FieldPtrs f = a.fields[sd.field];
  if (j >= sd.n) return;
  const int cb = sd.cb0 + j;
  cx<R> res[12];
  if (EPI & EPI_X) {
    int x[4];
    eo_coords(a.g, cb, a.pout, x);
    hop_sum<P, DAG, HopCfg<P, CFG>::depth>(a.g, sd, f, a.pout, cb, j, x, sys_ptr<P>(a.x, sd.off),
                                           nrm_ptr(a.xn, sd.off), res);
    const R al = (R)a.alpha;
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = al * res[k];
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = {0, 0};
  }
  if (EPI & EPI_Y) {
    cx<R> yv[12];
    Prec<P>::load(yv, sys_ptr<P>(a.y, sd.off), nrm_ptr(a.yn, sd.off), sd.n, j);
    const R be = (R)a.beta;
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = res[k] + be * yv[k];
  }
  cx<R> o[12];
  if (CLOV) {
    clover_apply<P>(f, true, 0, a.g.Vh, cb, res, o);
  } else {
    const R inv = (R)(1.0 / a.diag);
#pragma unroll
    for (int k = 0; k < 12; k++) o[k] = inv * res[k];
  }
  Prec<P>::store(sys_ptr_w<P>(a.out, sd.off), nrm_ptr_w(a.outn, sd.off), sd.n, j, o);
}

// ---------------------------------------------------------------------------
#ifndef LQ_HOP2_MINB
#define LQ_HOP2_MINB 5
#endif
// FP32 stencil with two threads per output site.  A block of 128 threads
// covers 64 sites; warps 0-1 (half 0) sum the hops in directions 0 and 1,
// warps 2-3 (half 1) those in directions 2 and 3, so the split is uniform per
// warp (no divergence) and each warp still reads 32 consecutive sites.  The
// halves swap the half-spinor the other one needs through shared memory; then
// half h owns chirality block h (spins 2h, 2h+1, i.e. float4 words 3h..3h+2):
// its y / z / w words, its 6x6 clover block and its output words.
LQ_DI void load_half32(cx<float> s[6], const void* base, int n, int j, int h) {
  const float4* p = (const float4*)base + 3 * h * n + j;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float4 v = __ldg(p + k * n);
    s[2 * k] = {v.x, v.y};
    s[2 * k + 1] = {v.z, v.w};
  }
}
LQ_DI void store_half32(void* base, int n, int j, int h, const cx<float> s[6]) {
  float4* p = (float4*)base + 3 * h * n + j;
#pragma unroll
  for (int k = 0; k < 3; k++) p[k * n] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
}

// Sum of the hops of this thread's two directions, combined with the other
// half's sum: returns chirality block h of D_hop x (6 complex).
template <bool DAG>
LQ_DI void hop_pair32(const HopArgs& a, const SysDesc& sd, const FieldPtrs& f, int cb, bool valid, int h, int tl,
                      cx<float> mine[6]) {
  __shared__ float2 xch[2][6][64];
  cx<float> part[12];
#pragma unroll
  for (int k = 0; k < 12; k++) part[k] = {0.f, 0.f};
  if (valid) {
    int x[4];
    eo_coords(a.g, cb, a.pout, x);
    const void* in = sys_ptr<32>(a.x, sd.off);
    if (h == 0) {
      hop_dir<32, DAG, 0>(a.g, sd, f, a.pout, cb, x, in, nullptr, part);
      hop_dir<32, DAG, 1>(a.g, sd, f, a.pout, cb, x, in, nullptr, part);
    } else {
      hop_dir<32, DAG, 2>(a.g, sd, f, a.pout, cb, x, in, nullptr, part);
      hop_dir<32, DAG, 3>(a.g, sd, f, a.pout, cb, x, in, nullptr, part);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const cx<float> send = h == 0 ? part[6 + k] : part[k];
    xch[h][k][tl] = make_float2(send.re, send.im);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const float2 o = xch[h ^ 1][k][tl];
    const cx<float> keep = h == 0 ? part[k] : part[6 + k];
    mine[k] = {keep.re + o.x, keep.im + o.y};
  }
}

template <bool DAG, bool CLOV, int RED, int EPI>
__global__ void __launch_bounds__(128, LQ_HOP2_MINB) k_hop2_lin(HopArgs a) {
  int s, by;
  grid_pos_tiled((int)blockIdx.x, a.nsys, a.nby, a.tile, s, by);
  if (s >= a.nsys) return;
  if (a.active && !a.active[s]) return;
  const SysDesc sd = a.sys[s];
  if (by * 64 >= sd.n) return;
  const int h = threadIdx.x >> 6, tl = threadIdx.x & 63;
  const int j = by * 64 + tl;
  const bool valid = j < sd.n;
  const FieldPtrs f = a.fields[sd.field];
  const int cb = sd.cb0 + j;
  cx<float> res[6];
  if (EPI & EPI_X) {
    hop_pair32<DAG>(a, sd, f, cb, valid, h, tl, res);
    const float al = (float)a.alpha;
#pragma unroll
    for (int k = 0; k < 6; k++) res[k] = al * res[k];
  } else {
#pragma unroll
    for (int k = 0; k < 6; k++) res[k] = {0.f, 0.f};
  }
  float red[3] = {0.f, 0.f, 0.f};
  if (valid) {
    cx<float> yv[6];
    if ((EPI & EPI_Y) || RED == RED_TS) load_half32(yv, sys_ptr<32>(a.y, sd.off), sd.n, j, h);
    if (EPI & EPI_Y) {
      cx<float> ay[6];
      if (CLOV) {
        ClovIO<32>::apply(f.A32 + (a.pout * 18 + 9 * h) * a.g.Vh, a.g.Vh, cb, yv, ay);
      } else {
#pragma unroll
        for (int k = 0; k < 6; k++) ay[k] = (float)a.diag * yv[k];
      }
      const float be = (float)a.beta;
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = res[k] + be * ay[k];
    }
    if (EPI & EPI_Z) {
      cx<float> zv[6];
      load_half32(zv, sys_ptr<32>(a.z, sd.off), sd.n, j, h);
      const float ga = (float)a.gamma;
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = res[k] + ga * zv[k];
    }
    store_half32(sys_ptr_w<32>(a.out, sd.off), sd.n, j, h, res);
    if (RED == RED_DOT_W) {
      cx<float> wv[6];
      load_half32(wv, sys_ptr<32>(a.w, sd.off), sd.n, j, h);
#pragma unroll
      for (int k = 0; k < 6; k++) {
        red[0] += wv[k].re * res[k].re + wv[k].im * res[k].im;
        red[1] += wv[k].re * res[k].im - wv[k].im * res[k].re;
      }
    } else if (RED == RED_TS) {
#pragma unroll
      for (int k = 0; k < 6; k++) {
        red[0] += res[k].re * yv[k].re + res[k].im * yv[k].im;
        red[1] += res[k].re * yv[k].im - res[k].im * yv[k].re;
        red[2] += res[k].re * res[k].re + res[k].im * res[k].im;
      }
    } else if (RED == RED_NORM) {
#pragma unroll
      for (int k = 0; k < 6; k++) red[2] += res[k].re * res[k].re + res[k].im * res[k].im;
    }
  }
  if (RED != RED_NONE) block_reduce_store<3, float>(red, a.partial + ((long long)s * a.pstride + by) * 4);
}

template <bool DAG, bool CLOV, int EPI>
__global__ void __launch_bounds__(128, LQ_HOP2_MINB) k_hop2_clinv(HopArgs a) {
  int s, by;
  grid_pos_tiled((int)blockIdx.x, a.nsys, a.nby, a.tile, s, by);
  if (s >= a.nsys) return;
  if (a.active && !a.active[s]) return;
  const SysDesc sd = a.sys[s];
  if (by * 64 >= sd.n) return;
  const int h = threadIdx.x >> 6, tl = threadIdx.x & 63;
  const int j = by * 64 + tl;
  const bool valid = j < sd.n;
  const FieldPtrs f = a.fields[sd.field];
  const int cb = sd.cb0 + j;
  cx<float> res[6];
  if (EPI & EPI_X) {
    hop_pair32<DAG>(a, sd, f, cb, valid, h, tl, res);
    const float al = (float)a.alpha;
#pragma unroll
    for (int k = 0; k < 6; k++) res[k] = al * res[k];
  } else {
#pragma unroll
    for (int k = 0; k < 6; k++) res[k] = {0.f, 0.f};
  }
  if (!valid) return;
  if (EPI & EPI_Y) {
    cx<float> yv[6];
    load_half32(yv, sys_ptr<32>(a.y, sd.off), sd.n, j, h);
    const float be = (float)a.beta;
#pragma unroll
    for (int k = 0; k < 6; k++) res[k] = res[k] + be * yv[k];
  }
  cx<float> o[6];
  if (CLOV) {
    ClovIO<32>::apply(f.Ai32 + 9 * h * a.g.Vh, a.g.Vh, cb, res, o);
  } else {
    const float inv = (float)(1.0 / a.diag);
#pragma unroll
    for (int k = 0; k < 6; k++) o[k] = inv * res[k];
  }
  store_half32(sys_ptr_w<32>(a.out, sd.off), sd.n, j, h, o);
}

}  // namespace lq
