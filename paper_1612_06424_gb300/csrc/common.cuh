// Device-side types and layouts shared by the kernels of the library.
//
// Even-odd (checkerboard) order.  A site x with natural index
// i = ((x0*L1+x1)*L2+x2)*L3+x3 has parity p = (x0+x1+x2+x3) & 1 and
// checkerboard index cb = i >> 1 (L3 even, so the two sites of a pair
// (x3, x3+1) have opposite parity and share cb).  Time is slowest, so the
// sites of parity p on the time slab t0..t1 are the contiguous cb range
// [t0*S3h, (t1+1)*S3h) with S3h = L1*L2*L3/2: a domain is a contiguous
// sub-array of each parity, which is what makes batched Dirichlet
// domains cheap.
//
// Vectors of one system in precision P live in a pool at a per-system site
// offset `off`, as structure-of-arrays over the system's n sites of one
// parity:  element k of site j at pool[off*NV + k*n + j], NV vector words
// per site (FP64: 12 x double2, FP32: 6 x float4, FP16: 3 x uint4 of 8
// halves plus one float norm per site in a parallel pool).  Consecutive
// threads therefore read consecutive 16-byte words: every spinor load is a
// fully coalesced 128-bit load.
//
// Links of field f, parity p, direction mu: [p][mu][NL][Vh] words, with
// FP64 keeping all 18 reals (9 x double2: FP64 is ALU-bound on this GPU, so
// rebuilding the third row would cost more than the bytes it saves) and
// FP32 / FP16 the first two rows (12 reals: 3 x float4 or 3 x uint2); the
// third row is conj(row0 x row1), rebuilt in registers (storing all 18 FP32
// reals measured 8-24% slower: the extra loads and registers cost more than
// the rebuild).
//
// Clover blocks.  In the chiral basis gamma_5 = diag(1,1,-1,-1) commutes
// with sigma_mu_nu, so A(x) is two 6x6 Hermitian blocks (spins {0,1} and
// {2,3}, index 3*(s&1)+c).  A block is stored as 36 reals: the 6 real
// diagonal entries, then the 15 complex entries below the diagonal, row by
// row ((1,0), (2,0), (2,1), (3,0), ...).  Layout [p][18 x double2 per block
// x 2 blocks = 36][Vh] (FP64) or [p][18 x float4][Vh] (FP32).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define LQ_DI __device__ __forceinline__
#define LQ_HDI __host__ __device__ __forceinline__

namespace lq {

template <typename R>
struct cx {
  R re, im;
};

template <typename R>
LQ_HDI cx<R> mk(R a, R b) {
  return cx<R>{a, b};
}
template <typename R>
LQ_HDI cx<R> operator+(cx<R> a, cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
LQ_HDI cx<R> operator-(cx<R> a, cx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
LQ_HDI cx<R> operator-(cx<R> a) {
  return {-a.re, -a.im};
}
template <typename R>
LQ_HDI cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
LQ_HDI cx<R> operator*(R s, cx<R> a) {
  return {s * a.re, s * a.im};
}
template <typename R>
LQ_HDI cx<R> conj(cx<R> a) {
  return {a.re, -a.im};
}
// conj(a) * b
template <typename R>
LQ_HDI cx<R> cmulc(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename R>
LQ_HDI cx<R> ti(cx<R> a) {
  return {-a.im, a.re};
}
template <typename R>
LQ_HDI R norm2(cx<R> a) {
  return a.re * a.re + a.im * a.im;
}
// acc += a * b
template <typename R>
LQ_HDI void fma_c(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
LQ_HDI void fma_cc(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];   // T, L1, L2, L3
  int L3h;    // L3 / 2
  int Vh;   // sites per parity
  int S3h;  // sites per parity and time slice
  int bc_t;   // 0 open, 1 periodic, 2 antiperiodic
  unsigned m3h, m2, m1;  // division magics of L3h, L2, L1 (fast_magic)
};

// n / d by one multiply-high: with m = ceil(2^32 / d) (d >= 2),
// floor(n m / 2^32) = floor(n / d) whenever n d < 2^32, because
// n m / 2^32 - n / d < n / 2^32 < 1 / d.  m = 0 stands for d = 1.  The
// lattice constructor checks n d < 2^32 for every site index n.
LQ_HDI unsigned fast_magic(unsigned d) { return d <= 1 ? 0u : (unsigned)((0x100000000ull + d - 1) / d); }
LQ_DI int fast_div(int n, unsigned m) { return m ? (int)__umulhi((unsigned)n, m) : n; }

// Coordinates of checkerboard site cb of parity p.
LQ_DI void eo_coords(const Geom& g, int cb, int p, int x[4]) {
  int q = fast_div(cb, g.m3h);
  const int x3h = cb - q * g.L3h;
  int r = q;
  q = fast_div(r, g.m2);
  x[2] = r - q * g.L[2];
  r = q;
  q = fast_div(r, g.m1);
  x[1] = r - q * g.L[1];
  x[0] = q;
  x[3] = 2 * x3h + ((x[0] + x[1] + x[2] + p) & 1);
}

LQ_DI int eo_index(const Geom& g, const int x[4]) {
  return (((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3]) >> 1;
}

// ------------------------------------------------------------ system / field
// One linear system of a batch: its gauge field, time slab and storage.
struct SysDesc {
  int field;       // index into the field table
  int t0, t1;      // inclusive time slab
  int wrap;        // 1: the slab is the whole lattice and time hops wrap
  float tsign;     // sign of a wrapping time hop (-1 antiperiodic)
  int pad;
  int n;           // sites per parity in the slab
  int cb0;         // first checkerboard index of the slab = t0 * S3h
  long long off;   // site offset of this system in the vector pools
};

struct FieldPtrs {
  const double2* U64;   // [2][4][9][Vh]
  const float4* U32;    // [2][4][3][Vh]
  const uint2* U16;     // [2][4][3][Vh]
  const double2* A64;   // [2][36][Vh]  clover blocks A on both parities
  const double2* Ai64;  // [36][Vh]     A^{-1} on even sites
  const float4* A32;    // [2][18][Vh]
  const float4* Ai32;   // [18][Vh]
};

// Per-system scalars of the Krylov iteration (device memory).
struct SolverScal {
  double2 rho, alpha, omega, beta;
  double target2;  // |r|^2 below which the current solve stops
  double rr;       // last |r|^2
  double rr0;      // |r|^2 at the start of the current inner cycle
  double bb;       // |eta|^2 of the full system (tolerance reference)
  int iters;       // iterations of the current inner cycle
  int status;      // 0 ok, 1 breakdown, 2 nan
};

// Fused reductions of the hop kernels and modes of the scalar finalize.
enum { RED_NONE = 0, RED_DOT_W = 1, RED_TS = 2, RED_NORM = 3 };
enum { FIN_ALPHA = 0, FIN_OMEGA = 1, FIN_BETA = 2, FIN_INIT = 3, FIN_NORM = 4,
       FIN_CG_RHO = 5, FIN_CG_ALPHA = 6, FIN_CG_R = 7, FIN_CG_BETA = 8 };

// ------------------------------------------------------------ precision I/O
template <int P>
struct Prec;

template <>
struct Prec<64> {
  typedef double R;
  static constexpr int NV = 12;  // double2 words per spinor
  LQ_DI static void load(cx<double> s[12], const void* base, const float*, int n, int j) {
    const double2* p = (const double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = __ldg(p + k * n + j);
      s[k] = {v.x, v.y};
    }
  }
  LQ_DI static void quantize(cx<double>*) {}
  LQ_DI static void store(void* base, float*, int n, int j, const cx<double> s[12]) {
    double2* p = (double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) p[k * n + j] = make_double2(s[k].re, s[k].im);
  }
};

template <>
struct Prec<32> {
  typedef float R;
  static constexpr int NV = 6;  // float4 words per spinor
  LQ_DI static void load(cx<float> s[12], const void* base, const float*, int n, int j) {
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = __ldg(p + k * n + j);
      s[2 * k] = {v.x, v.y};
      s[2 * k + 1] = {v.z, v.w};
    }
  }
  LQ_DI static void quantize(cx<float>*) {}
  LQ_DI static void store(void* base, float*, int n, int j, const cx<float> s[12]) {
    float4* p = (float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) p[k * n + j] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
  }
};

// FP16 spinor: 24 halves holding psi / nu, nu = max |component| (FP32, one per site).
template <>
struct Prec<16> {
  typedef float R;
  static constexpr int NV = 3;  // uint4 words (8 halves) per spinor
  LQ_DI static void load(cx<float> s[12], const void* base, const float* nrm, int n, int j) {
    const uint4* p = (const uint4*)base;
    float nu = __ldg(nrm + j);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v = __ldg(p + k * n + j);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        __half2 h = *reinterpret_cast<const __half2*>(&w[q]);
        float2 f = __half22float2(h);
        s[4 * k + q] = {f.x * nu, f.y * nu};
      }
    }
  }
  // The values a store followed by a load would return (same rounding).
  LQ_DI static void quantize(cx<float> s[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      float2 f = __half22float2(__floats2half2_rn(s[k].re * inv, s[k].im * inv));
      s[k] = {f.x * m, f.y * m};
    }
  }
  LQ_DI static void store(void* base, float* nrm, int n, int j, const cx<float> s[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
    float inv = m > 0.f ? 1.f / m : 0.f;
    uint4* p = (uint4*)base;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        __half2 h = __floats2half2_rn(s[4 * k + q].re * inv, s[4 * k + q].im * inv);
        w[q] = *reinterpret_cast<uint32_t*>(&h);
      }
      p[k * n + j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    nrm[j] = m;
  }
};

// Read-once loads of links and clover (a no-L1-allocate variant measured no
// faster on GB300, so these are plain read-only loads).
LQ_DI float4 ld_once(const float4* p) { return __ldg(p); }
LQ_DI uint2 ld_once(const uint2* p) { return __ldg(p); }

// Position of a block in a linearised (system, block) grid: the system index
// runs fastest, so the blocks of all systems that cover the same sites (and
// share a gauge field) run together and meet their links in L2.
LQ_DI void grid_pos(int nsys, int& s, int& by) {
  s = (int)(blockIdx.x % (unsigned)nsys);
  by = (int)(blockIdx.x / (unsigned)nsys);
}

// Time-tiled order of a (system, block) grid of nsys x nby blocks for the
// stencil: the blocks of tb consecutive site blocks (a few time slices) of every
// system run together, then the next tile.  Within a tile the systems follow one
// another, so a site row and its neighbour rows in time are read within a
// window of tb blocks of one system (they stay in L2), while links and clover
// are shared by the systems of the tile.  tb <= 0 (or >= nby) gives grid_pos.
// A bijection of [0, nsys * nby) onto the (system, block) pairs.
LQ_HDI void grid_pos_tiled(int bid, int nsys, int nby, int tb, int& s, int& by) {
  if (tb <= 0 || tb >= nby) {
    s = bid % nsys;
    by = bid / nsys;
    return;
  }
  const int per_tile = nsys * tb;
  const int full = nby / tb;  // tiles of tb blocks; the last one holds the rest
  if (bid < full * per_tile) {
    const int t = bid / per_tile, w = bid - t * per_tile;
    s = w / tb;
    by = t * tb + (w - s * tb);
  } else {
    const int r = nby - full * tb;
    const int w = bid - full * per_tile;
    s = w / r;
    by = full * tb + (w - s * r);
  }
}

// Site (within the system's slab, one parity) of thread t of block `by` of a
// 128-thread stencil block.  Plain: 128 consecutive sites.  Time-blocked
// (tblk): warp w covers 32 consecutive sites of time slice 4*g + w, the four
// warps the same 32 positions of four consecutive slices, so a block reads
// most of its own time-direction neighbours (x0 -+ 1) itself.  Time-blocked
// order needs S3h % 32 == 0 and every slab's slice count % 4 == 0 (checked on
// the host); it maps the blocks 0 .. n/128 - 1 onto the same n sites.
LQ_HDI int site_of_block(int tblk, int S3h, int by, int t) {
  if (!tblk) return by * 128 + t;
  const int nchunk = S3h >> 5;
  const int g = by / nchunk, chunk = by - g * nchunk;
  return ((g << 2) + (t >> 5)) * S3h + (chunk << 5) + (t & 31);
}

// ------------------------------------------------------------------- links
template <typename R>
struct su3 {
  cx<R> m[3][3];
};

template <typename R>
LQ_DI void reconstruct_row2(su3<R>& u) {
  u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
  u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
  u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
}

template <int P>
struct LinkIO;

template <>
struct LinkIO<64> {
  LQ_DI static su3<double> load(const FieldPtrs& f, int p, int mu, int Vh, int cb) {
    const double2* b = f.U64 + (p * 4 + mu) * 9 * Vh + cb;
    su3<double> u;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 v = __ldg(b + k * Vh);
      u.m[k / 3][k % 3] = {v.x, v.y};
    }
    return u;
  }
};

template <>
struct LinkIO<32> {
  LQ_DI static su3<float> load(const FieldPtrs& f, int p, int mu, int Vh, int cb) {
    const float4* b = f.U32 + (p * 4 + mu) * 3 * Vh + cb;
    su3<float> u;
    float4 a = ld_once(b), c = ld_once(b + Vh), d = ld_once(b + 2 * Vh);
    u.m[0][0] = {a.x, a.y};
    u.m[0][1] = {a.z, a.w};
    u.m[0][2] = {c.x, c.y};
    u.m[1][0] = {c.z, c.w};
    u.m[1][1] = {d.x, d.y};
    u.m[1][2] = {d.z, d.w};
    reconstruct_row2(u);
    return u;
  }
};

template <>
struct LinkIO<16> {
  LQ_DI static su3<float> load(const FieldPtrs& f, int p, int mu, int Vh, int cb) {
    const uint2* b = f.U16 + (p * 4 + mu) * 3 * Vh + cb;
    su3<float> u;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint2 v = ld_once(b + k * Vh);
      float2 x = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      float2 y = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
      u.m[(2 * k) / 3][(2 * k) % 3] = {x.x, x.y};
      u.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = {y.x, y.y};
    }
    reconstruct_row2(u);
    return u;
  }
};

// Clover block access: FP64 for P = 64, FP32 otherwise.
template <int P>
struct ClovIO {
  typedef float R;
  // 36 reals of block b of parity p at cb -> Hermitian 6x6 mat-vec
  LQ_DI static void apply(const float4* base, int Vh, int cb, const cx<float> in[6], cx<float> out[6]) {
    float a[36];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float4 v = ld_once(base + k * Vh + cb);
      a[4 * k] = v.x;
      a[4 * k + 1] = v.y;
      a[4 * k + 2] = v.z;
      a[4 * k + 3] = v.w;
    }
    herm6_apply<float>(a, in, out);
  }
  template <typename T>
  LQ_DI static void herm6_apply(const T* a, const cx<T> in[6], cx<T> out[6]) {
#pragma unroll
    for (int r = 0; r < 6; r++) out[r] = a[r] * in[r];
    int q = 6;
#pragma unroll
    for (int r = 1; r < 6; r++)
#pragma unroll
      for (int c = 0; c < r; c++) {
        cx<T> e = {a[q], a[q + 1]};  // A[r][c]; A[c][r] = conj(e)
        q += 2;
        fma_c(out[r], e, in[c]);
        fma_cc(out[c], e, in[r]);
      }
  }
};

template <>
struct ClovIO<64> {
  typedef double R;
  LQ_DI static void apply(const double2* base, int Vh, int cb, const cx<double> in[6], cx<double> out[6]) {
    double a[36];
#pragma unroll
    for (int k = 0; k < 18; k++) {
      double2 v = __ldg(base + k * Vh + cb);
      a[2 * k] = v.x;
      a[2 * k + 1] = v.y;
    }
    ClovIO<32>::herm6_apply<double>(a, in, out);
  }
};

}  // namespace lq
