// Host launchers for the stencil and vector kernels, plus the layout
// kernels (natural <-> even-odd), point sources and the boundary hop of
// the Schur-complement assembly.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "blas.cuh"
#include "internal.h"

using namespace lq;

static std::atomic<long long> g_launches{0};
void lq_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void lq_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" long long lqcd_kernel_launches(void) { return g_launches.load(); }

// Linearised (system, block) grids: block x = by * nsys + s (see grid_pos).
static inline dim3 grid_lin(const Batch& b, long long blocks_per_sys, unsigned z = 1) {
  return dim3((unsigned)(b.nsys * blocks_per_sys), 1, z);
}
static inline dim3 grid_of(const Batch& b) { return grid_lin(b, b.nby); }
// word-parallel grid: NV 16-byte words per site
static inline dim3 grid_words(const Batch& b, int P) {
  const long long nv = P == 64 ? 12 : 6;
  return grid_lin(b, (b.max_n * nv + LQ_BLOCK - 1) / LQ_BLOCK);
}

static inline int launched() {
  lq_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  return 0;
}

// Time slices per tile of the stencil's block order: LQCD_HOP_TILE forces a
// value for every batch, else the batch's (chosen by lq_tune_hop).
static int tile_of(const Batch& b) {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("LQCD_HOP_TILE");
    forced = e ? atoi(e) : -1;
  }
  return forced >= 0 ? forced : b.hop_tile;
}

// site blocks per system and blocks per time tile for blocks of `sites_per_block` sites
// Time-blocked sites: LQCD_HOP_TBLK=0|1 forces, else the batch's choice; only
// for 128-site blocks of batches whose slabs allow it.
static int tblk_of(const Batch& b) {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("LQCD_HOP_TBLK");
    forced = e ? atoi(e) : -1;
  }
  return b.tblk_ok && (forced >= 0 ? forced : b.hop_tblk) ? 1 : 0;
}

static void set_grid_order(HopArgs& a, const lqcd_lattice* L, const Batch& b, int sites_per_block) {
  a.nby = (int)((b.max_n + sites_per_block - 1) / sites_per_block);
  const int h = tile_of(b);
  a.tile = h > 0 ? (int)((h * L->S3h + sites_per_block - 1) / sites_per_block) : 0;
  a.tblk = sites_per_block == LQ_BLOCK ? tblk_of(b) : 0;
}

static HopArgs hop_args(const lqcd_lattice* L, const Batch& b, int pout) {
  HopArgs a{};
  a.g = L->g;
  a.sys = b.sys;
  a.fields = L->d_fields;
  a.active = b.active;
  a.pout = pout;
  a.partial = b.partial;
  a.pstride = b.pstride;
  a.nsys = b.nsys;
  a.diag = 1.0 / (2.0 * L->kappa);
  set_grid_order(a, L, b, LQ_BLOCK);
  return a;
}

// Stencil variant of a batch (FP32 / FP16; FP64 always 1):
//   1 = one thread per site, default launch configuration (HopCfg 0),
//   2 = two threads per site (k_hop2_*, FP32 only),
//   3 / 4 = one thread per site in launch configuration HopCfg 1 / 2 (the
//       forward operator; dagger launches keep configuration 0).
// LQCD_HOP_VARIANT=1..4 (or the older LQCD_HOP_SPLIT=1|2) forces one for
// every batch.
static int forced_variant() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("LQCD_HOP_VARIANT");
    if (!e) e = getenv("LQCD_HOP_SPLIT");
    v = (e && e[0] >= '1' && e[0] <= '4') ? e[0] - '0' : 0;
  }
  return v;
}

static int variant_of(int P, const Batch& b) {
  if (P == 64) return 1;
  const int f = forced_variant();
  const int v = f ? f : b.hop_variant;
  if (v == 2) return P == 32 ? 2 : 1;
  return (v == 3 || v == 4) ? v : 1;
}

int lq_hop_wps(int P, const Batch& b) { return variant_of(P, b) == 2 ? 2 : 1; }

template <bool DAG, bool CLOV>
static int launch_lin2(int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  constexpr int XY = EPI_X | EPI_Y, XZ = EPI_X | EPI_Z, XYZ = EPI_X | EPI_Y | EPI_Z;
  if (red == RED_NONE && epi == XY) k_hop2_lin<DAG, CLOV, RED_NONE, XY><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (red == RED_NONE && epi == XZ) k_hop2_lin<DAG, CLOV, RED_NONE, XZ><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (red == RED_DOT_W && epi == XY) k_hop2_lin<DAG, CLOV, RED_DOT_W, XY><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (red == RED_TS && epi == XY) k_hop2_lin<DAG, CLOV, RED_TS, XY><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (red == RED_NORM && epi == XYZ) k_hop2_lin<DAG, CLOV, RED_NORM, XYZ><<<gr, LQ_BLOCK, 0, st>>>(a);
  else return -1;
  return 0;
}

template <bool DAG, bool CLOV>
static int launch_clinv2(int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (epi == EPI_X) k_hop2_clinv<DAG, CLOV, EPI_X><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (epi == EPI_Y) k_hop2_clinv<DAG, CLOV, EPI_Y><<<gr, LQ_BLOCK, 0, st>>>(a);
  else if (epi == (EPI_X | EPI_Y)) k_hop2_clinv<DAG, CLOV, EPI_X | EPI_Y><<<gr, LQ_BLOCK, 0, st>>>(a);
  else return -1;
  return 0;
}

template <int P>
static void hop_go(void (*k)(HopArgs), dim3 gr, const HopArgs& a, cudaStream_t st) {
  k<<<gr, LQ_BLOCK, 0, st>>>(a);
}

// (reduction, epilogue) pairs the solver uses
template <int P, bool DAG, bool CLOV>
static int launch_lin(int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  constexpr int XY = EPI_X | EPI_Y, XZ = EPI_X | EPI_Z, XYZ = EPI_X | EPI_Y | EPI_Z;
  if (red == RED_NONE && epi == XY) hop_go<P>(k_hop_lin<P, DAG, CLOV, RED_NONE, XY>, gr, a, st);
  else if (red == RED_NONE && epi == XZ) hop_go<P>(k_hop_lin<P, DAG, CLOV, RED_NONE, XZ>, gr, a, st);
  else if (red == RED_DOT_W && epi == XY) hop_go<P>(k_hop_lin<P, DAG, CLOV, RED_DOT_W, XY>, gr, a, st);
  else if (red == RED_TS && epi == XY) hop_go<P>(k_hop_lin<P, DAG, CLOV, RED_TS, XY>, gr, a, st);
  else if (red == RED_NORM && epi == XYZ) hop_go<P>(k_hop_lin<P, DAG, CLOV, RED_NORM, XYZ>, gr, a, st);
  else return -1;
  return 0;
}

template <int P>
static int launch_lin_p(bool dag, bool clov, int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (dag) return clov ? launch_lin<P, true, true>(red, epi, gr, a, st) : launch_lin<P, true, false>(red, epi, gr, a, st);
  return clov ? launch_lin<P, false, true>(red, epi, gr, a, st) : launch_lin<P, false, false>(red, epi, gr, a, st);
}

int lq_hop_lin(int P, bool dag, bool clov, int red, const lqcd_lattice* L, const Batch& b, int pout, VecP x, VecP y,
               VecP z, VecP w, VecP out, double alpha, double beta, double gamma, cudaStream_t st) {
  HopArgs a = hop_args(L, b, pout);
  a.x = x.d; a.xn = x.nrm;
  a.y = y.d; a.yn = y.nrm;
  a.z = z.d; a.zn = z.nrm;
  a.w = w.d; a.wn = w.nrm;
  a.out = out.d; a.outn = out.nrm;
  a.alpha = alpha; a.beta = beta; a.gamma = gamma;
  const int epi = (alpha != 0.0 ? EPI_X : 0) | (beta != 0.0 ? EPI_Y : 0) | (gamma != 0.0 ? EPI_Z : 0);
  dim3 gr = grid_of(b);
  if (variant_of(P, b) == 2) {
    const dim3 g2 = grid_lin(b, (b.max_n + 63) / 64);
    set_grid_order(a, L, b, 64);
    int rc = dag ? (clov ? launch_lin2<true, true>(red, epi, g2, a, st) : launch_lin2<true, false>(red, epi, g2, a, st))
                 : (clov ? launch_lin2<false, true>(red, epi, g2, a, st) : launch_lin2<false, false>(red, epi, g2, a, st));
    if (rc) {
      lq_set_error("hop kernel: unsupported (reduction, epilogue) pair");
      return LQCD_EBADARG;
    }
    return launched();
  }
  const int v = variant_of(P, b);
  int rc;
  if (!dag && v >= 3)
    rc = P == 32 ? hop_lin_tuned<32>(v - 2, clov, red, epi, gr, a, st) : hop_lin_tuned<16>(v - 2, clov, red, epi, gr, a, st);
  else
    rc = P == 64 ? launch_lin_p<64>(dag, clov, red, epi, gr, a, st)
       : P == 32 ? launch_lin_p<32>(dag, clov, red, epi, gr, a, st)
                 : launch_lin_p<16>(dag, clov, red, epi, gr, a, st);
  if (rc) {
    lq_set_error("hop kernel: unsupported (reduction, epilogue) pair");
    return LQCD_EBADARG;
  }
  return launched();
}

template <int P, bool DAG, bool CLOV>
static int launch_clinv(int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (epi == EPI_X) hop_go<P>(k_hop_clinv<P, DAG, CLOV, EPI_X>, gr, a, st);
  else if (epi == EPI_Y) hop_go<P>(k_hop_clinv<P, DAG, CLOV, EPI_Y>, gr, a, st);
  else if (epi == (EPI_X | EPI_Y)) hop_go<P>(k_hop_clinv<P, DAG, CLOV, EPI_X | EPI_Y>, gr, a, st);
  else return -1;
  return 0;
}

template <int P>
static int launch_clinv_p(bool dag, bool clov, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (dag) return clov ? launch_clinv<P, true, true>(epi, gr, a, st) : launch_clinv<P, true, false>(epi, gr, a, st);
  return clov ? launch_clinv<P, false, true>(epi, gr, a, st) : launch_clinv<P, false, false>(epi, gr, a, st);
}

int lq_hop_clinv(int P, bool dag, bool clov, const lqcd_lattice* L, const Batch& b, VecP x, VecP y, VecP out,
                 double alpha, double beta, cudaStream_t st) {
  HopArgs a = hop_args(L, b, 0);
  a.x = x.d; a.xn = x.nrm;
  a.y = y.d; a.yn = y.nrm;
  a.out = out.d; a.outn = out.nrm;
  a.alpha = alpha; a.beta = beta;
  const int epi = (alpha != 0.0 ? EPI_X : 0) | (beta != 0.0 ? EPI_Y : 0);
  dim3 gr = grid_of(b);
  if (variant_of(P, b) == 2) {
    const dim3 g2 = grid_lin(b, (b.max_n + 63) / 64);
    set_grid_order(a, L, b, 64);
    int rc = dag ? (clov ? launch_clinv2<true, true>(epi, g2, a, st) : launch_clinv2<true, false>(epi, g2, a, st))
                 : (clov ? launch_clinv2<false, true>(epi, g2, a, st) : launch_clinv2<false, false>(epi, g2, a, st));
    if (rc) {
      lq_set_error("clover-inverse hop kernel: unsupported epilogue");
      return LQCD_EBADARG;
    }
    return launched();
  }
  const int v = variant_of(P, b);
  int rc;
  if (!dag && v >= 3)
    rc = P == 32 ? hop_clinv_tuned<32>(v - 2, clov, epi, gr, a, st) : hop_clinv_tuned<16>(v - 2, clov, epi, gr, a, st);
  else
    rc = P == 64 ? launch_clinv_p<64>(dag, clov, epi, gr, a, st)
       : P == 32 ? launch_clinv_p<32>(dag, clov, epi, gr, a, st)
                 : launch_clinv_p<16>(dag, clov, epi, gr, a, st);
  if (rc) {
    lq_set_error("clover-inverse hop kernel: unsupported epilogue");
    return LQCD_EBADARG;
  }
  return launched();
}

// out_p = kappa D_hop x (the Wilson hopping term on the slab, Dirichlet at
// its ends), output parity pout, FP64: the clover-free inverse-diagonal
// kernel with alpha = 1/2, since 1 / diag = 2 kappa.
int lq_hop_kappa(const lqcd_lattice* L, const Batch& b, int pout, const double2* x, double2* out, cudaStream_t st) {
  HopArgs a = hop_args(L, b, pout);
  a.x = x;
  a.out = out;
  a.alpha = 0.5;
  k_hop_clinv<64, false, false, EPI_X><<<grid_of(b), LQ_BLOCK, 0, st>>>(a);
  return launched();
}

static VecArgs vec_args(const Batch& b) {
  VecArgs v;
  v.sys = b.sys;
  v.active = b.active;
  v.sc = b.sc;
  v.partial = b.partial;
  v.pstride = b.pstride;
  v.nsys = b.nsys;
  return v;
}

int lq_words_per_site(int P) { return P == 64 ? 12 : P == 32 ? 6 : 1; }

int lq_bicg_s(int P, const Batch& b, VecP r, VecP v, VecP s, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_bicg_s_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, r.d, v.d, s.d);
  else if (P == 32) k_bicg_s_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, r.d, v.d, s.d);
  else k_bicg_s_h<<<grid_of(b), LQ_BLOCK, 0, st>>>(va, r.d, r.nrm, v.d, v.nrm, s.d, s.nrm);
  return launched();
}

int lq_bicg_xr(int P, const Batch& b, VecP x, VecP p, VecP s, VecP t, VecP r, VecP r0, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_bicg_xr_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, x.d, p.d, s.d, t.d, r.d, r0.d);
  else if (P == 32) k_bicg_xr_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, x.d, p.d, s.d, t.d, r.d, r0.d);
  else
    k_bicg_xr_h<<<grid_of(b), LQ_BLOCK, 0, st>>>(va, x.d, x.nrm, p.d, p.nrm, s.d, s.nrm, t.d, t.nrm, r.d, r.nrm, r0.d,
                                                 r0.nrm);
  return launched();
}

int lq_bicg_p(int P, const Batch& b, VecP p, VecP r, VecP v, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_bicg_p_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, p.d, r.d, v.d);
  else if (P == 32) k_bicg_p_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, p.d, r.d, v.d);
  else k_bicg_p_h<<<grid_of(b), LQ_BLOCK, 0, st>>>(va, p.d, p.nrm, r.d, r.nrm, v.d, v.nrm);
  return launched();
}

int lq_cg_xr(int P, const Batch& b, VecP x, VecP p, VecP r, VecP v, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_cg_xr_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, x.d, p.d, r.d, v.d);
  else if (P == 32) k_cg_xr_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, x.d, p.d, r.d, v.d);
  else return LQCD_EBADARG;
  return launched();
}

int lq_cg_p(int P, const Batch& b, VecP p, VecP z, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_cg_p_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, p.d, z.d);
  else if (P == 32) k_cg_p_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, p.d, z.d);
  else return LQCD_EBADARG;
  return launched();
}

int lq_inner_init(int P, const Batch& b, const double2* r64, VecP r, VecP r0, VecP p, VecP x, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_inner_init_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, r64, r.d, r0.d, p.d, x.d);
  else if (P == 32) k_inner_init_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, r64, r.d, r0.d, p.d, x.d);
  else
    k_inner_init_h<<<grid_of(b), LQ_BLOCK, 0, st>>>(va, r64, r.d, r.nrm, r0.d, r0.nrm, p.d, p.nrm, x.d, x.nrm);
  return launched();
}

int lq_accum64(int P, const Batch& b, double2* x64, VecP x, cudaStream_t st) {
  VecArgs va = vec_args(b);
  if (P == 64) k_accum64_w<64><<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(va, x64, x.d);
  else if (P == 32) k_accum64_w<32><<<grid_words(b, 32), LQ_BLOCK, 0, st>>>(va, x64, x.d);
  else k_accum64_h<<<grid_of(b), LQ_BLOCK, 0, st>>>(va, x64, x.d, x.nrm);
  return launched();
}

int lq_norm2_64(const Batch& b, const double2* v, cudaStream_t st) {
  k_norm2_64<<<grid_words(b, 64), LQ_BLOCK, 0, st>>>(vec_args(b), v);
  return launched();
}

int lq_finalize(int mode, const Batch& b, double tau2, double floor_rel2, int wps, cudaStream_t st) {
  k_finalize<<<b.nsys, FIN_THREADS, 0, st>>>(mode, b.nsys, b.sys, b.active, b.sc, b.partial, b.pstride, wps, LQ_BLOCK,
                                             tau2, floor_rel2);
  return launched();
}

int lq_count_active(const Batch& b, int* d_count, cudaStream_t st) {
  k_count_active<<<1, 256, 0, st>>>(b.nsys, b.active, d_count);
  return launched();
}

int lq_convert(int Pin, int Pout, const Batch& b, VecP in, VecP out, cudaStream_t st) {
  VecArgs va = vec_args(b);
  dim3 gr = grid_of(b);
  if (Pin == 64 && Pout == 32) k_convert<64, 32><<<gr, LQ_BLOCK, 0, st>>>(va, in.d, in.nrm, out.d, out.nrm);
  else if (Pin == 64 && Pout == 16) k_convert<64, 16><<<gr, LQ_BLOCK, 0, st>>>(va, in.d, in.nrm, out.d, out.nrm);
  else if (Pin == 32 && Pout == 64) k_convert<32, 64><<<gr, LQ_BLOCK, 0, st>>>(va, in.d, in.nrm, out.d, out.nrm);
  else if (Pin == 16 && Pout == 64) k_convert<16, 64><<<gr, LQ_BLOCK, 0, st>>>(va, in.d, in.nrm, out.d, out.nrm);
  else k_convert<64, 64><<<gr, LQ_BLOCK, 0, st>>>(va, in.d, in.nrm, out.d, out.nrm);
  return launched();
}

// ------------------------------------------------------------ layout kernels
// Natural slab vector of system s (src[s], sites t0*S3 .. (t1+1)*S3 - 1)
// <-> the system's even and odd FP64 vectors.  G5: multiply by gamma_5
// (spin components 2, 3 negated) on the way in.
template <bool G5>
__global__ void __launch_bounds__(128) k_nat_to_eo(Geom g, int nsys, const SysDesc* sys, const int* active,
                                                   const double2* const* src, double2* ve, double2* vo) {
  int s, by;
  grid_pos(nsys, s, by);
  if (active && !active[s]) return;
  const SysDesc sd = sys[s];
  const long long j = (long long)by * blockDim.x + threadIdx.x;
  if (j >= sd.n) return;
  const int p = blockIdx.z;
  int x[4];
  eo_coords(g, sd.cb0 + j, p, x);
  const long long nat = ((((long long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3]);
  const long long loc = nat - (long long)sd.t0 * (2 * g.S3h);
  const double2* in = src[s] + loc * 12;
  double2* out = (p == 0 ? ve : vo) + sd.off * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const double2 v = in[k];
    out[k * sd.n + j] = (G5 && k >= 6) ? make_double2(-v.x, -v.y) : v;
  }
}

__global__ void __launch_bounds__(128) k_eo_to_nat(Geom g, int nsys, const SysDesc* sys, const double2* ve,
                                                   const double2* vo, double2* const* dst, double scale) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const long long j = (long long)by * blockDim.x + threadIdx.x;
  if (j >= sd.n) return;
  const int p = blockIdx.z;
  int x[4];
  eo_coords(g, sd.cb0 + j, p, x);
  const long long nat = ((((long long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3]);
  const long long loc = nat - (long long)sd.t0 * (2 * g.S3h);
  double2* out = dst[s] + loc * 12;
  const double2* in = (p == 0 ? ve : vo) + sd.off * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 v = in[k * sd.n + j];
    out[k] = make_double2(scale * v.x, scale * v.y);
  }
}

int lq_nat_to_eo(const lqcd_lattice* L, const Batch& b, const double2* const* src, double2* ve, double2* vo,
                 cudaStream_t st) {
  k_nat_to_eo<false><<<grid_lin(b, b.nby, 2), LQ_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, nullptr, src, ve, vo);
  return launched();
}

int lq_nat_to_eo_g5(const lqcd_lattice* L, const Batch& b, const double2* const* src, double2* ve, double2* vo,
                    cudaStream_t st) {
  k_nat_to_eo<true><<<grid_lin(b, b.nby, 2), LQ_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, nullptr, src, ve, vo);
  return launched();
}

int lq_eo_to_nat(const lqcd_lattice* L, const Batch& b, const double2* ve, const double2* vo, double2* const* dst,
                 double scale, cudaStream_t st) {
  k_eo_to_nat<<<grid_lin(b, b.nby, 2), LQ_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, ve, vo, dst, scale);
  return launched();
}

// Zero both parities of every system and place 1 at (xsrc[s], column cols[s]).
__global__ void __launch_bounds__(128) k_point_source(Geom g, int nsys, const SysDesc* sys, const int* cols,
                                                      const int4* xsrc, double2* ve, double2* vo) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const int j = by * blockDim.x + threadIdx.x;
  if (j >= sd.n) return;
  const int p = blockIdx.z;
  const int4 q = xsrc[s];
  const int xs[4] = {q.x, q.y, q.z, q.w};
  const int ps = (q.x + q.y + q.z + q.w) & 1;
  const int cbs = eo_index(g, xs);
  double2* out = (p == 0 ? ve : vo) + sd.off * 12;
  const bool here = (p == ps) && (sd.cb0 + j == cbs);
  const int col = cols[s];
#pragma unroll
  for (int k = 0; k < 12; k++) out[k * sd.n + j] = make_double2((here && k == col) ? 1.0 : 0.0, 0.0);
}

int lq_point_source(const lqcd_lattice* L, const Batch& b, const int* d_cols, const int4* d_xsrc, double2* ve,
                    double2* vo, cudaStream_t st) {
  k_point_source<<<grid_lin(b, b.nby, 2), LQ_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, d_cols, d_xsrc, ve, vo);
  return launched();
}

// Boundary source of the Schur assembly, Sec. 3 eq. quark_prop_II:
//   chi = P_Gamma* D P_Gamma psi,  Gamma = 0..g1, Gamma* = g1+1..T-1.
// Only time hops from a site y of Gamma* to a site of Gamma survive:
//   slot 0, y0 = g1+1 :  -1/2 (1 + g_0) U_0(y-0)^dag psi(y-0)
//   slot 1, y0 = T-1  :  -1/2 (1 - g_0) U_0(y) psi(y+0) * sign   (periodic / antiperiodic only)
// chi is stored compactly, natural order within a time slice:
//   chi[c][slot][site of slice][12].  psi: the Gammabar solution of system s
// (its eo pools), written to chi column cols[s].
__global__ void __launch_bounds__(128) k_boundary_chi(Geom g, int nsys, const FieldPtrs* fields, const SysDesc* sin,
                                                      const int* cols, int g1, const double2* in_e,
                                                      const double2* in_o, double2* chi) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc si = sin[s];
  const int S3 = 2 * g.S3h;
  const int i = by * blockDim.x + threadIdx.x;  // site within the slice
  const int slot = blockIdx.z;
  if (i >= S3) return;
  double2* out = chi + ((long long)(cols[s] * 2 + slot) * S3 + i) * 12;
  cx<double> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0.0, 0.0};
  const bool active = slot == 0 || g.bc_t != 0;
  if (active) {
    int x[4];
    x[3] = i % g.L[3];
    x[2] = (i / g.L[3]) % g.L[2];
    x[1] = i / (g.L[3] * g.L[2]);
    x[0] = slot == 0 ? g1 + 1 : g.L[0] - 1;
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const FieldPtrs f = fields[si.field];
    const double2* inb = (p == 0 ? in_o : in_e) + si.off * 12;  // neighbour parity
    cx<double> psi[12], h[6], w[6];
    if (slot == 0) {
      int y[4] = {x[0] - 1, x[1], x[2], x[3]};
      const int cy = eo_index(g, y);
      Prec<64>::load(psi, inb, nullptr, si.n, cy - si.cb0);
      project<0, +1>(psi, h);
      su3<double> u = LinkIO<64>::load(f, p ^ 1, 0, g.Vh, cy);
      mul_udag(u, h, w);
      expand_add<0, +1>(acc, w);
    } else {
      const double sg = g.bc_t == 2 ? -1.0 : 1.0;
      int y[4] = {0, x[1], x[2], x[3]};
      const int cy = eo_index(g, y);
      Prec<64>::load(psi, inb, nullptr, si.n, cy - si.cb0);
      project<0, -1>(psi, h);
      su3<double> u = LinkIO<64>::load(f, p, 0, g.Vh, eo_index(g, x));
      mul_u(u, h, w);
#pragma unroll
      for (int k = 0; k < 6; k++) w[k] = sg * w[k];
      expand_add<0, -1>(acc, w);
    }
  }
#pragma unroll
  for (int k = 0; k < 12; k++) out[k] = make_double2(-0.5 * acc[k].re, -0.5 * acc[k].im);
}

int lq_boundary_chi(const lqcd_lattice* L, const Batch& bin, const int* d_cols, int g1, const double2* in_e,
                    const double2* in_o, double2* chi, cudaStream_t st) {
  const int S3 = 2 * L->g.S3h;
  k_boundary_chi<<<grid_lin(bin, (S3 + LQ_BLOCK - 1) / LQ_BLOCK, 2), LQ_BLOCK, 0, st>>>(L->g, bin.nsys, L->d_fields,
                                                                                      bin.sys, d_cols, g1, in_e,
                                                                                      in_o, chi);
  return launched();
}

// Source of a Gamma* system: chi (compact, column cols[s]) scattered into the
// system's even / odd FP64 vectors, zero elsewhere.
__global__ void __launch_bounds__(128) k_chi_to_eo(Geom g, int nsys, const SysDesc* sys, const int* cols, int g1,
                                                   const double2* chi, double2* ve, double2* vo) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const int j = by * blockDim.x + threadIdx.x;
  if (j >= sd.n) return;
  const int p = blockIdx.z;
  int x[4];
  eo_coords(g, sd.cb0 + j, p, x);
  const int S3 = 2 * g.S3h;
  const int i = (x[1] * g.L[2] + x[2]) * g.L[3] + x[3];
  double2 v[12];
#pragma unroll
  for (int k = 0; k < 12; k++) v[k] = make_double2(0.0, 0.0);
  for (int slot = 0; slot < 2; slot++) {
    const bool on = slot == 0 ? x[0] == g1 + 1 : (g.bc_t != 0 && x[0] == g.L[0] - 1);
    if (!on) continue;
    const double2* c = chi + ((long long)(cols[s] * 2 + slot) * S3 + i) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) v[k] = make_double2(v[k].x + c[k].x, v[k].y + c[k].y);
  }
  double2* out = (p == 0 ? ve : vo) + sd.off * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) out[k * sd.n + j] = v[k];
}

int lq_chi_to_eo(const lqcd_lattice* L, const Batch& b, const int* d_cols, int g1, const double2* chi, double2* ve,
                 double2* vo, cudaStream_t st) {
  k_chi_to_eo<<<grid_lin(b, b.nby, 2), LQ_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, d_cols, g1, chi, ve, vo);
  return launched();
}

__global__ void k_sub_inplace(double2* a, const double2* b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 x = a[i], y = b[i];
    a[i] = make_double2(x.x - y.x, x.y - y.y);
  }
}

int lq_sub_inplace(double2* a, const double2* b, long long n, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_sub_inplace<<<(unsigned)blocks, 256, 0, st>>>(a, b, n);
  return launched();
}

// Deterministic pseudo-random fill in [-1, 1) (a hash of the word index).
__global__ void k_fill64(double2* p, long long n, unsigned seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    const double a = (double)(h & 0xffffffffull) * (2.0 / 4294967296.0) - 1.0;
    const double b = (double)(h >> 32) * (2.0 / 4294967296.0) - 1.0;
    p[i] = make_double2(a, b);
  }
}

int lq_fill64(double2* p, long long n, unsigned seed, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_fill64<<<(unsigned)blocks, 256, 0, st>>>(p, n, seed);
  return launched();
}

// --------------------------------------------------------------- autotuner
// Decisions per batch shape (precision, systems, sites per parity of the
// largest system), kept for the process and, if LQCD_TUNE_CACHE names a file,
// read from and appended to it ("P nsys max_n variant" per line).
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, long long>, int> g_tune;
bool g_tune_loaded = false;

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("LQCD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int P, n, v;
  long long m;
  while (fscanf(f, "%d %d %lld %d", &P, &n, &m, &v) == 4) g_tune[std::make_tuple(P, n, m)] = v;
  fclose(f);
}

void tune_store(int P, int n, long long m, int v) {
  const char* path = getenv("LQCD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%d %d %lld %d\n", P, n, m, v);
  fclose(f);
}
}  // namespace

int lq_tune_hop(const lqcd_lattice* L, const Batch& b, int P, bool clov, VecP x, VecP y, VecP out, cudaStream_t st) {
  if (P == 64) return 1;
  if (forced_variant()) return forced_variant();
  const auto key = std::make_tuple(P, b.nsys, b.max_n);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1;
  VecP none;
  // candidates: the default, the alternative launch configurations and (FP32)
  // the two-thread kernel; each warmed, then timed in three alternating rounds
  // of five launches of the solver's second half of D^ and of the clover-inverse
  // first half; the best round of each counts, and a candidate must beat the
  // default by 3% to be chosen
  std::vector<int> cand = {1, 3, 4};
  if (P == 32) cand.push_back(2);
  std::vector<float> best(cand.size(), 1e30f);
  for (int round = -1; round < 3; round++)
    for (size_t c = 0; c < cand.size(); c++) {
      Batch t = b;
      t.hop_variant = cand[c];
      t.active = nullptr;  // time every system
      const int reps = round < 0 ? 1 : 5;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps; r++) {
        lq_hop_clinv(P, false, clov, L, t, y, none, x, 1.0, 0.0, st);
        lq_hop_lin(P, false, clov, RED_NONE, L, t, 1, x, y, none, none, out, -0.25, 1.0, 0.0, st);
      }
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (round >= 0 && ms < best[c]) best[c] = ms;
    }
  int pick = 1;
  float pick_ms = 0.97f * best[0];
  for (size_t c = 1; c < cand.size(); c++)
    if (best[c] < pick_ms) {
      pick = cand[c];
      pick_ms = best[c];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = pick;
  tune_store(P, b.nsys, b.max_n, pick);
  return pick;
}
