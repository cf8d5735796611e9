// Quark-line projection (Sec. 3.3 eqs. projection, quark_prop_II_proj) and
// the inverse-iteration projection vectors of Sec. 6:
//   * orthonormalisation of N FP64 complex columns by Cholesky QR, twice
//     (Gram matrix G = V^dag V, G = L L^dag, W = V L^{-dag}; the second pass
//     restores orthogonality lost to cond(V)^2 in the first);
//   * slice extraction with P_+ = (1 + gamma_0)/2 and slice sources;
//   * the projected case-II propagator  -sum_i eta_i(y) xi_i(x)^dag.
#include "internal.h"

using namespace lq;

#define RC(call)            \
  do {                      \
    int r_ = (call);        \
    if (r_ != 0) return r_; \
  } while (0)

namespace {

constexpr int GT = 16;   // Gram / apply column tile
constexpr int GR = 32;   // rows per shared-memory stage of the Gram kernel
constexpr int AJ = 64;   // coefficient rows per shared-memory stage of the apply kernel

int launched_here() {
  lq_count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  return 0;
}

LQ_DI double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Element (row r, column k) of a column matrix; r runs over the segments.
LQ_DI double2 cm_get(const ColMat& m, long long r, int k) {
  if (k >= m.ncol) return make_double2(0.0, 0.0);
  if (r < m.rows[0]) return m.p[0][(long long)k * m.ld[0] + r];
  r -= m.rows[0];
  if (m.nseg > 1 && r < m.rows[1]) return m.p[1][(long long)k * m.ld[1] + r];
  return make_double2(0.0, 0.0);
}

// Partial Gram matrices: block (tile pair (ta <= tb), split z) sums
// conj(V[r][a]) V[r][b] over its row chunk into part[z][a][b].
__global__ void __launch_bounds__(GT * GT) k_gram(ColMat m, long long chunk, int npad, const int2* pairs,
                                                 double2* part) {
  __shared__ double2 sa[GR][GT], sb[GR][GT];
  const int2 tp = pairs[blockIdx.x];
  const int a0 = tp.x * GT, b0 = tp.y * GT;
  const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
  const long long R = m.rows[0] + (m.nseg > 1 ? m.rows[1] : 0);
  const long long r_lo = (long long)blockIdx.y * chunk;
  const long long r_hi = r_lo + chunk < R ? r_lo + chunk : R;
  double2 acc = make_double2(0.0, 0.0);
  for (long long r0 = r_lo; r0 < r_hi; r0 += GR) {
    for (int e = threadIdx.x; e < GR * GT; e += GT * GT) {
      const int rr = e % GR, c = e / GR;
      const long long r = r0 + rr;
      const bool in = r < r_hi;
      sa[rr][c] = in ? cm_get(m, r, a0 + c) : make_double2(0.0, 0.0);
      sb[rr][c] = in ? cm_get(m, r, b0 + c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GR; rr++) {
      const double2 x = sa[rr][ty], y = sb[rr][tx];
      acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
      acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
    }
    __syncthreads();
  }
  part[((long long)blockIdx.y * npad + a0 + ty) * npad + b0 + tx] = acc;
}

// G[a][b] = sum over splits, mirrored from the computed upper tiles.
__global__ void k_gram_reduce(const double2* part, int nsplit, int npad, int n, double2* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int a = t / n, b = t % n;
  const bool up = a / GT <= b / GT;
  const int i = up ? a : b, j = up ? b : a;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < nsplit; z++) {
    const double2 v = part[((long long)z * npad + i) * npad + j];
    s.x += v.x;
    s.y += v.y;
  }
  G[(long long)a * n + b] = up ? s : make_double2(s.x, -s.y);
}

// One block: G = L L^dag in place (lower triangle), then Linv = L^{-1}.
// status = 1 when a pivot falls below 1e-14 of its column's squared norm
// (the column's part orthogonal to the previous ones is below 1e-7 of its
// norm: linearly dependent at FP64 precision for Cholesky QR).  n <= 1024.
__global__ void __launch_bounds__(1024) k_chol_inv(double2* G, int n, double2* Linv, int* status) {
  __shared__ int bad;
  __shared__ double diag0[1024];
  if (threadIdx.x == 0) bad = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) diag0[k] = G[(long long)k * n + k].x;
  __syncthreads();
  for (int k = 0; k < n; k++) {
    if (threadIdx.x == 0) {
      const double d = G[(long long)k * n + k].x;
      if (!(d > 1e-14 * diag0[k]) || !isfinite(d)) bad = 1;
      G[(long long)k * n + k] = make_double2(bad ? 1.0 : sqrt(d), 0.0);
    }
    __syncthreads();
    if (bad) break;
    const double piv = G[(long long)k * n + k].x;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double2 v = G[(long long)i * n + k];
      G[(long long)i * n + k] = make_double2(v.x / piv, v.y / piv);
    }
    __syncthreads();
    const int m = n - k - 1;  // trailing block (i, j), k < j <= i < n
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j > i) continue;
      const double2 li = G[(long long)i * n + k], lj = G[(long long)j * n + k];
      double2 g = G[(long long)i * n + j];
      // g -= li * conj(lj)
      g.x -= li.x * lj.x + li.y * lj.y;
      g.y -= li.y * lj.x - li.x * lj.y;
      G[(long long)i * n + j] = g;
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) *status = 1;
    return;
  }
  // forward substitution, one column c of L^{-1} per thread
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < c; i++) Linv[(long long)i * n + c] = make_double2(0.0, 0.0);
    for (int i = c; i < n; i++) {
      double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int j = c; j < i; j++) {
        const double2 t = cmul(G[(long long)i * n + j], Linv[(long long)j * n + c]);
        s.x -= t.x;
        s.y -= t.y;
      }
      const double d = G[(long long)i * n + i].x;
      Linv[(long long)i * n + c] = make_double2(s.x / d, s.y / d);
    }
  }
}

// W[r][k] = sum_{j <= k} V[r][j] conj(Linv[k][j])   (W = V L^{-dag}).
__global__ void __launch_bounds__(128) k_apply_rinv(ColMat in, ColMat out, const double2* Linv, int n) {
  __shared__ double2 cf[AJ][GT];
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * GT;
  const long long R = in.rows[0] + (in.nseg > 1 ? in.rows[1] : 0);
  double2 acc[GT];
#pragma unroll
  for (int q = 0; q < GT; q++) acc[q] = make_double2(0.0, 0.0);
  const int jend = min(n, k0 + GT);
  for (int j0 = 0; j0 < jend; j0 += AJ) {
    for (int e = threadIdx.x; e < AJ * GT; e += blockDim.x) {
      const int jj = e / GT, q = e % GT;
      const int j = j0 + jj, k = k0 + q;
      double2 c = make_double2(0.0, 0.0);
      if (j < n && k < n && j <= k) {
        const double2 l = Linv[(long long)k * n + j];
        c = make_double2(l.x, -l.y);
      }
      cf[jj][q] = c;
    }
    __syncthreads();
    if (r < R) {
      const int jn = min(AJ, jend - j0);
      for (int jj = 0; jj < jn; jj++) {
        const double2 v = cm_get(in, r, j0 + jj);
#pragma unroll
        for (int q = 0; q < GT; q++) {
          const double2 c = cf[jj][q];
          acc[q].x = fma(v.x, c.x, fma(-v.y, c.y, acc[q].x));
          acc[q].y = fma(v.x, c.y, fma(v.y, c.x, acc[q].y));
        }
      }
    }
    __syncthreads();
  }
  if (r >= R) return;
  int sg = 0;
  long long rr = r;
  if (rr >= out.rows[0]) {
    rr -= out.rows[0];
    sg = 1;
  }
#pragma unroll
  for (int q = 0; q < GT; q++) {
    const int k = k0 + q;
    if (k < n) out.p[sg][(long long)k * out.ld[sg] + rr] = acc[q];
  }
}

// phi[s][site of slice g1][12] = P_+ v_s(x), x on slice g1 of system s
// (P_+ = (1 + gamma_0)/2: upper = (u - l)/2, lower = -upper in the chiral basis).
__global__ void __launch_bounds__(128) k_slice_plus(Geom g, int nsys, const SysDesc* sys, int g1, const double2* ve,
                                                    const double2* vo, double2* phi) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const int S3 = 2 * g.S3h;
  const int i = by * blockDim.x + threadIdx.x;
  if (i >= S3) return;
  const int x3 = i % g.L[3], x2 = (i / g.L[3]) % g.L[2], x1 = i / (g.L[3] * g.L[2]);
  const int p = (g1 + x1 + x2 + x3) & 1;
  const long long nat = (long long)g1 * S3 + i;
  const int j = (int)(nat >> 1) - sd.cb0;
  const double2* v = (p == 0 ? ve : vo) + sd.off * 12 + j;
  double2* o = phi + ((long long)s * S3 + i) * 12;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double2 u = v[(long long)k * sd.n], l = v[(long long)(k + 6) * sd.n];
    const double2 h = make_double2(0.5 * (u.x - l.x), 0.5 * (u.y - l.y));
    o[k] = h;
    o[k + 6] = make_double2(-h.x, -h.y);
  }
}

// Source of system s: phi[ids[s]] on slice g1, zero elsewhere in its slab.
__global__ void __launch_bounds__(128) k_slice_source(Geom g, int nsys, const SysDesc* sys, const int* ids, int g1,
                                                      const double2* phi, double2* ve, double2* vo) {
  int s, by;
  grid_pos(nsys, s, by);
  const SysDesc sd = sys[s];
  const int j = by * blockDim.x + threadIdx.x;
  if (j >= sd.n) return;
  const int p = blockIdx.z;
  int x[4];
  eo_coords(g, sd.cb0 + j, p, x);
  const int S3 = 2 * g.S3h;
  double2* out = (p == 0 ? ve : vo) + sd.off * 12;
  if (x[0] == g1) {
    const int i = (x[1] * g.L[2] + x[2]) * g.L[3] + x[3];
    const double2* f = phi + ((long long)ids[s] * S3 + i) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) out[k * sd.n + j] = f[k];
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) out[k * sd.n + j] = make_double2(0.0, 0.0);
  }
}

// fact[b][y][a] = -sum_i eta_i(y)[a] conj(xi_i(x)[b]) for y in Gamma*; one
// thread per (site of Gamma*, a).  xi_x[i][b] = xi_i(x)[b] is staged in
// shared memory (n * 12 entries).
__global__ void __launch_bounds__(128) k_proj_prop(int n, long long nsite, long long y0, long long V,
                                                   const double2* eta, const double2* xi_x, double2* fact) {
  extern __shared__ double2 xs[];
  for (int e = threadIdx.x; e < n * 12; e += blockDim.x) xs[e] = xi_x[e];
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsite * 12) return;
  double2 acc[12];
#pragma unroll
  for (int b = 0; b < 12; b++) acc[b] = make_double2(0.0, 0.0);
  for (int i = 0; i < n; i++) {
    const double2 e = eta[(long long)i * nsite * 12 + t];
#pragma unroll
    for (int b = 0; b < 12; b++) {
      const double2 c = xs[i * 12 + b];
      // e * conj(c)
      acc[b].x = fma(e.x, c.x, fma(e.y, c.y, acc[b].x));
      acc[b].y = fma(e.y, c.x, fma(-e.x, c.y, acc[b].y));
    }
  }
  const long long y = y0 + t / 12;
  const int a = (int)(t % 12);
#pragma unroll
  for (int b = 0; b < 12; b++) fact[((long long)b * V + y) * 12 + a] = make_double2(-acc[b].x, -acc[b].y);
}

// xi_x[i][b] = xi_i(x)[b]
__global__ void k_gather_site(int n, long long nsite_gb, long long xloc, const double2* xi, double2* xi_x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 12) return;
  const int i = t / 12, b = t % 12;
  xi_x[t] = xi[((long long)i * nsite_gb + xloc) * 12 + b];
}

struct Scratch {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
  int alloc(size_t bytes, cudaStream_t s) {
    st = s;
    if (cudaMallocAsync(&p, bytes ? bytes : 16, s) != cudaSuccess) {
      cudaGetLastError();
      lq_set_error("device allocation failed (orthonormalisation scratch)");
      return LQCD_ENOMEM;
    }
    return 0;
  }
};

// One Cholesky-QR pass: out = in R^{-1}, in = out R.
int chol_qr(const ColMat& in, const ColMat& out, double2* G, double2* Linv, int2* d_pairs, int npairs,
            double2* part, int nsplit, long long chunk, int npad, int* d_status, cudaStream_t st) {
  const int n = in.ncol;
  k_gram<<<dim3((unsigned)npairs, (unsigned)nsplit), GT * GT, 0, st>>>(in, chunk, npad, d_pairs, part);
  RC(launched_here());
  k_gram_reduce<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(part, nsplit, npad, n, G);
  RC(launched_here());
  k_chol_inv<<<1, 1024, 0, st>>>(G, n, Linv, d_status);
  RC(launched_here());
  const long long R = in.rows[0] + (in.nseg > 1 ? in.rows[1] : 0);
  k_apply_rinv<<<dim3((unsigned)((R + 127) / 128), (unsigned)((n + GT - 1) / GT)), 128, 0, st>>>(in, out, Linv, n);
  return launched_here();
}

}  // namespace

int lq_orthonormalize(ColMat v, ColMat tmp, cudaStream_t st) {
  const int n = v.ncol;
  if (n < 1 || n > 1024) {
    lq_set_error("orthonormalisation: 1..1024 columns");
    return LQCD_EBADARG;
  }
  const long long R = v.rows[0] + (v.nseg > 1 ? v.rows[1] : 0);
  if (R < n) {
    lq_set_error("orthonormalisation: fewer rows than columns");
    return LQCD_ERANK;
  }
  const int nt = (n + GT - 1) / GT, npad = nt * GT;
  std::vector<int2> pairs;
  for (int a = 0; a < nt; a++)
    for (int b = a; b < nt; b++) pairs.push_back(make_int2(a, b));
  const int npairs = (int)pairs.size();
  int nsplit = (152 * 8 + npairs - 1) / npairs;
  long long chunk = (R + nsplit - 1) / nsplit;
  chunk = (chunk + GR - 1) / GR * GR;
  nsplit = (int)((R + chunk - 1) / chunk);
  const size_t b_pairs = sizeof(int2) * npairs, b_part = sizeof(double2) * (size_t)nsplit * npad * npad,
               b_g = sizeof(double2) * (size_t)n * n;
  Scratch s;
  RC(s.alloc(b_pairs + b_part + 2 * b_g + 256 + 64, st));
  char* base = (char*)s.p;
  int2* d_pairs = (int2*)base;
  double2* part = (double2*)(base + ((b_pairs + 255) / 256) * 256);
  double2* G = (double2*)((char*)part + b_part);
  double2* Linv = (double2*)((char*)G + b_g);
  int* d_status = (int*)((char*)Linv + b_g);
  if (cudaMemcpyAsync(d_pairs, pairs.data(), b_pairs, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d_status, 0, sizeof(int), st) != cudaSuccess) {
    lq_set_error("orthonormalisation: copy failed");
    return LQCD_ECUDA;
  }
  RC(chol_qr(v, tmp, G, Linv, d_pairs, npairs, part, nsplit, chunk, npad, d_status, st));
  RC(chol_qr(tmp, v, G, Linv, d_pairs, npairs, part, nsplit, chunk, npad, d_status, st));
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    lq_set_error("orthonormalisation: synchronisation failed");
    return LQCD_ECUDA;
  }
  if (h_status) {
    lq_set_error("orthonormalisation: the vectors are linearly dependent");
    return LQCD_ERANK;
  }
  return 0;
}

int lq_slice_plus(const lqcd_lattice* L, const Batch& b, int g1, const double2* ve, const double2* vo, double2* phi,
                  cudaStream_t st) {
  const int S3 = 2 * L->g.S3h;
  k_slice_plus<<<(unsigned)(b.nsys * ((S3 + 127) / 128)), 128, 0, st>>>(L->g, b.nsys, b.sys, g1, ve, vo, phi);
  return launched_here();
}

int lq_slice_source(const lqcd_lattice* L, const Batch& b, const int* d_ids, int g1, const double2* phi, double2* ve,
                    double2* vo, cudaStream_t st) {
  k_slice_source<<<dim3((unsigned)(b.nsys * b.nby), 1, 2), 128, 0, st>>>(L->g, b.nsys, b.sys, d_ids, g1, phi, ve, vo);
  return launched_here();
}

int lq_proj_prop(const lqcd_lattice* L, int n, long long nsite_gb, long long xloc, const double2* xi, long long nsite_gs,
                 long long y0, const double2* eta, double2* fact, cudaStream_t st) {
  Scratch s;
  RC(s.alloc(sizeof(double2) * 12 * (size_t)n, st));
  double2* xi_x = (double2*)s.p;
  k_gather_site<<<(unsigned)((n * 12 + 127) / 128), 128, 0, st>>>(n, nsite_gb, xloc, xi, xi_x);
  RC(launched_here());
  const size_t sm = sizeof(double2) * 12 * (size_t)n;
  if (sm > 48 * 1024) {
    if (cudaFuncSetAttribute(k_proj_prop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
      cudaGetLastError();
      lq_set_error("projected propagator: too many modes for shared memory");
      return LQCD_EBADARG;
    }
  }
  k_proj_prop<<<(unsigned)((nsite_gs * 12 + 127) / 128), 128, sm, st>>>(n, nsite_gs, y0, L->V, eta, xi_x, fact);
  return launched_here();
}
