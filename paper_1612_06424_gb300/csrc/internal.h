// Internal interfaces of the library: the lattice object, batches of
// systems and the host launchers of the kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lqcd.h"
#include "common.cuh"

void lq_count_launch();
void lq_count_launches(long long n);
extern "C" long long lqcd_kernel_launches(void);
void lq_set_error(const std::string& msg);

// A vector of a batch in one precision: pool base (and FP16 norm pool).
struct VecP {
  void* d = nullptr;
  float* nrm = nullptr;
};

// Device view of a batch of systems: descriptors, activity flags, iteration
// scalars and the block-partial buffer of the fused reductions.
struct Batch {
  int nsys = 0;
  int nby = 0;               // site blocks (one site per thread) of the largest system
  int pstride = 0;           // partial-buffer blocks per system (>= any kernel's grid.y)
  int hop_variant = 1;       // stencil variant (lq_tune_hop): launch configuration / threads per site
  int hop_tile = 0;          // time slices per tile of the stencil's block order (0: systems fastest)
  int hop_tblk = 1;          // 1: time-blocked sites (32 sites x 4 slices per block) where allowed
  int tblk_ok = 0;           // every slab has a multiple of 4 slices and S3h % 32 == 0
  long long max_n = 0;
  long long total = 0;       // sum of n over systems (sites per parity)
  const lq::SysDesc* sys = nullptr;
  int* active = nullptr;
  lq::SolverScal* sc = nullptr;
  double* partial = nullptr;
};

constexpr int LQ_BLOCK = 128;

struct FieldData {
  double2* Unat = nullptr;  // natural-order copy of U (FP64), used by the force
  double2* U64 = nullptr;
  float4* U32 = nullptr;
  uint2* U16 = nullptr;
  double2* A64 = nullptr;
  double2* Ai64 = nullptr;
  float4* A32 = nullptr;
  float4* Ai32 = nullptr;
};

struct lqcd_lattice {
  int dims[4];
  int bc;
  long long V, Vh, S3, S3h;
  lq::Geom g;
  double kappa = 0.125, csw = 0.0;
  std::vector<FieldData> fields;
  lq::FieldPtrs* d_fields = nullptr;
  int device = 0;
  cudaStream_t graph_stream = nullptr;  // private stream the solver's CUDA graphs run on
  cudaEvent_t graph_event = nullptr;
};

// ---------------------------------------------------------------- launchers
int lq_launch_pack_links(const lq::Geom& g, const double2* U, double2* U64, float4* U32, uint2* U16,
                         unsigned long long* maxdev, cudaStream_t st);
int lq_launch_clover(const lq::Geom& g, const double2* U, double kappa, double csw, double2* A64, double2* Ai64,
                     float4* A32, float4* Ai32, int* fail, cudaStream_t st);

// out = beta*A(y) + alpha*D_hop x + gamma*z on parity pout (+ fused reduction)
int lq_hop_lin(int P, bool dag, bool clov, int red, const lqcd_lattice* L, const Batch& b, int pout, VecP x, VecP y,
               VecP z, VecP w, VecP out, double alpha, double beta, double gamma, cudaStream_t st);
// out = A^{-1}(alpha*D_hop x + beta*y) on even sites
int lq_hop_clinv(int P, bool dag, bool clov, const lqcd_lattice* L, const Batch& b, VecP x, VecP y, VecP out,
                 double alpha, double beta, cudaStream_t st);

int lq_bicg_s(int P, const Batch& b, VecP r, VecP v, VecP s, cudaStream_t st);
int lq_bicg_xr(int P, const Batch& b, VecP x, VecP p, VecP s, VecP t, VecP r, VecP r0, cudaStream_t st);
int lq_bicg_p(int P, const Batch& b, VecP p, VecP r, VecP v, cudaStream_t st);
int lq_inner_init(int P, const Batch& b, const double2* r64, VecP r, VecP r0, VecP p, VecP x, cudaStream_t st);
// CG on the normal equations (P = 64 or 32): x += alpha p, r -= alpha v (|r|^2); p = z + beta p
int lq_cg_xr(int P, const Batch& b, VecP x, VecP p, VecP r, VecP v, cudaStream_t st);
int lq_cg_p(int P, const Batch& b, VecP p, VecP z, cudaStream_t st);
int lq_accum64(int P, const Batch& b, double2* x64, VecP x, cudaStream_t st);
int lq_norm2_64(const Batch& b, const double2* v, cudaStream_t st);
int lq_finalize(int mode, const Batch& b, double tau2, double floor_rel2, int wps, cudaStream_t st);
// 16-byte words per site of the word-parallel vector kernels of precision P (1 for FP16: one site per thread)
int lq_words_per_site(int P);
// blocks-per-site factor of the hop kernels' reductions (2: two threads per site)
int lq_hop_wps(int P, const Batch& b);
// Autotuner: the fastest FP32 stencil variant for this batch shape, timed on
// the given vectors (x on even sites, y / out on odd sites) once per shape and
// cached; returns the variant (1 or 2).
int lq_tune_hop(const lqcd_lattice* L, const Batch& b, int P, bool clov, VecP x, VecP y, VecP out, cudaStream_t st);
int lq_count_active(const Batch& b, int* d_count, cudaStream_t st);
int lq_convert(int Pin, int Pout, const Batch& b, VecP in, VecP out, cudaStream_t st);

// layout conversion: natural complex128 slab vectors <-> even-odd FP64 pools
int lq_nat_to_eo(const lqcd_lattice* L, const Batch& b, const double2* const* src, double2* ve, double2* vo,
                 cudaStream_t st);
int lq_nat_to_eo_g5(const lqcd_lattice* L, const Batch& b, const double2* const* src, double2* ve, double2* vo,
                    cudaStream_t st);
int lq_hop_kappa(const lqcd_lattice* L, const Batch& b, int pout, const double2* x, double2* out, cudaStream_t st);
int lq_slice_dot(const lqcd_lattice* L, const Batch& b, const double2* const* eta, const double2* ye,
                 const double2* yo, const int* slot, double2* trace, cudaStream_t st);
int lq_mean_sources(const double2* trace, int n_src, long long per_src, double2* mean, cudaStream_t st);
// N complex FP64 columns over one or two row segments (e.g. the even and odd
// halves of a batch of equal systems): column k of segment s starts at
// p[s] + k * ld[s] and holds rows[s] entries.
struct ColMat {
  double2* p[2] = {nullptr, nullptr};
  long long ld[2] = {0, 0};
  long long rows[2] = {0, 0};
  int nseg = 1;
  int ncol = 0;
};
int lq_orthonormalize(ColMat v, ColMat tmp, cudaStream_t st);
int lq_slice_plus(const lqcd_lattice* L, const Batch& b, int g1, const double2* ve, const double2* vo, double2* phi,
                  cudaStream_t st);
int lq_slice_source(const lqcd_lattice* L, const Batch& b, const int* d_ids, int g1, const double2* phi, double2* ve,
                    double2* vo, cudaStream_t st);
int lq_proj_prop(const lqcd_lattice* L, int n, long long nsite_gb, long long xloc, const double2* xi, long long nsite_gs,
                 long long y0, const double2* eta, double2* fact, cudaStream_t st);
int lq_eo_to_nat(const lqcd_lattice* L, const Batch& b, const double2* ve, const double2* vo, double2* const* dst,
                 double scale, cudaStream_t st);
// point sources: system k gets the unit vector of column cols[k] at xsrc[k]
int lq_point_source(const lqcd_lattice* L, const Batch& b, const int* d_cols, const int4* d_xsrc, double2* ve,
                    double2* vo, cudaStream_t st);
// compact boundary source chi[col][slot][slice site][12] of Gamma* from the Gammabar solutions
int lq_boundary_chi(const lqcd_lattice* L, const Batch& bin, const int* d_cols, int g1, const double2* in_e,
                    const double2* in_o, double2* chi, cudaStream_t st);
// Gamma* sources from chi
int lq_chi_to_eo(const lqcd_lattice* L, const Batch& b, const int* d_cols, int g1, const double2* chi, double2* ve,
                 double2* vo, cudaStream_t st);
// a -= b elementwise over n double2 words
int lq_sub_inplace(double2* a, const double2* b, long long n, cudaStream_t st);

// force
int lq_force(const lqcd_lattice* L, int field, const lqcd_slab& dom, const double2* X, const double2* Y, double* F,
             cudaStream_t st);
int lq_fill64(double2* p, long long n, unsigned seed, cudaStream_t st);
// nucleon point correlators W[p][t] = (W1, W2) of propagators prop[p] ([12][V][12] double2)
// over slices t0..t0+n_t-1; partial: lq_nucleon_point_partial_words(...) double2 of scratch
// nucleon blocks on the tensor cores (nucleon_tc.cu); returns after the kernel finished
int lq_nucleon_blocks_tc(int n, long long nsite, const double2* s, int conj, int S3, long long lo0, int n_t,
                         double2* B, cudaStream_t st);
int lq_nucleon_point(const lqcd_lattice* L, int n_prop, const double2* prop, int t0, int n_t, double2* partial,
                     double2* W, cudaStream_t st);
long long lq_nucleon_point_partial_words(const lqcd_lattice* L, int n_prop, int n_t);
