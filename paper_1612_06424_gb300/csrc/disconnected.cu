// Contraction of the stochastic disconnected-trace estimator, Sec. 5 eq.
// stochastic_estimator: per source, slab and time slice,
//   t(x0) = sum_{xvec} eta^dag(x) y(x),   y = (kappa D_hop)^8 D_L^{-1} g5 eta,
// and the mean over the sources.
#include "internal.h"

using namespace lq;

namespace {

constexpr int DOT_BLOCK = 256;

// One block per (system, time slice of its slab).  eta[s]: the system's
// source on the whole lattice (natural order, 12 complex per site); y: the
// systems' even / odd FP64 vectors.  Writes trace[slot[s] * T + x0].
__global__ void __launch_bounds__(DOT_BLOCK) k_slice_dot(Geom g, int nsys, const SysDesc* sys,
                                                        const double2* const* eta, const double2* ye,
                                                        const double2* yo, const int* slot, double2* trace) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const int t = sd.t0 + by;
  if (t > sd.t1) return;
  const int S3 = 2 * g.S3h;
  const double2* e = eta[s];
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < S3; i += DOT_BLOCK) {
    const long long nat = (long long)t * S3 + i;
    const int x3 = i % g.L[3];
    const int x2 = (i / g.L[3]) % g.L[2];
    const int x1 = i / (g.L[3] * g.L[2]);
    const int p = (t + x1 + x2 + x3) & 1;
    const int j = (int)(nat >> 1) - sd.cb0;
    const double2* yv = (p == 0 ? ye : yo) + sd.off * 12 + j;
    const double2* ev = e + nat * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 a = ev[k], b = yv[(long long)k * sd.n];
      re += a.x * b.x + a.y * b.y;  // conj(a) * b
      im += a.x * b.y - a.y * b.x;
    }
  }
  __shared__ double sre[DOT_BLOCK / 32], sim[DOT_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sre[w] = re;
    sim[w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < DOT_BLOCK / 32; k++) {
      a += sre[k];
      b += sim[k];
    }
    trace[(long long)slot[s] * g.L[0] + t] = make_double2(a, b);
  }
}

// mean[k] = (1/n_src) sum_i trace[i * per_src + k], summed in source order.
__global__ void k_mean_sources(const double2* trace, int n_src, long long per_src, double2* mean) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per_src) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < n_src; i++) {
    const double2 v = trace[(long long)i * per_src + k];
    a += v.x;
    b += v.y;
  }
  mean[k] = make_double2(a / n_src, b / n_src);
}

int launched_here() {
  lq_count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  return 0;
}

}  // namespace

int lq_slice_dot(const lqcd_lattice* L, const Batch& b, const double2* const* eta, const double2* ye,
                 const double2* yo, const int* slot, double2* trace, cudaStream_t st) {
  if (b.nsys < 1) return 0;
  const unsigned blocks = (unsigned)b.nsys * (unsigned)L->dims[0];  // up to T slices per system
  k_slice_dot<<<blocks, DOT_BLOCK, 0, st>>>(L->g, b.nsys, b.sys, eta, ye, yo, slot, trace);
  return launched_here();
}

int lq_mean_sources(const double2* trace, int n_src, long long per_src, double2* mean, cudaStream_t st) {
  if (per_src < 1 || n_src < 1) return 0;
  k_mean_sources<<<(unsigned)((per_src + 127) / 128), 128, 0, st>>>(trace, n_src, per_src, mean);
  return launched_here();
}
