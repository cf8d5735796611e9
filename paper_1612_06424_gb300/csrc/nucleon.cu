// Nucleon blocks on projected quark lines (Sec. 4.2 eq. nucleon_prop_factorized):
//   B[i][j][k][alpha](t) = sum_{x in slice t} eps^{abc} {[s_i^T]^a(x) C g5 [s_j]^b(x)} [s_k]^c_alpha(x)
// as a contraction over (x, c) of the diquark D[(i,j)][(x,c)] with
// S[(x,c)][(k,alpha)] = s_k(x)[alpha][c]: a dense O(N^3 L^3) product, run on
// the FP32 pipes (the GB300's FP64 rate is 1/62 of FP32): per-thread FP32
// partial sums over 64 sites are added into FP32 running sums (two-level
// summation); the diquark tiles are generated in shared memory and never stored.  Then the two Wick contractions
//   W1 = -sum_ijk B_xi[j,i,k]^T g5 P_- B_eta[i,j,k],  W2 = -sum_ijk B_xi[k,i,j]^T g5 P_- B_eta[i,j,k].
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"

using namespace lq;

namespace {

constexpr int TI = 8, TJ = 8;  // (i, j) pair tile: 64 rows
constexpr int TK = 16;         // k tile: 64 (k, alpha) columns
constexpr int XS = 8;          // sites per shared-memory stage
constexpr int FLUSH = 8;       // stages per first-level partial sum (64 sites)
constexpr int TOT_BYTES = 16 * 256 * 8;  // dynamic shared memory of the second-level sums

#define RC_LAUNCH()                     \
  do {                                  \
    const int r_ = launched_here();     \
    if (r_ != 0) return r_;             \
  } while (0)

int launched_here() {
  lq_count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  return 0;
}

// C g5 with C = g0 g2 in the chiral basis of lqcd.h (g0 = [[0,-1],[-1,0]],
// g2 = [[0,-i s2],[i s2,0]], g5 = diag(1,1,-1,-1)): its non-zero entries are
// (0,1) = -1, (1,0) = +1, (2,3) = -1, (3,2) = +1, so
// s^T C g5 t = -s0 t1 + s1 t0 - s2 t3 + s3 t2   (spin indices).
LQ_DI float2 cg5_pair(const float2* si, const float2* tj, int a, int b) {
  // si, tj: 12 complex [spin*3 + colour]; colour a of s, colour b of t
  float2 r = make_float2(0.f, 0.f);
  const int sp[4][2] = {{0, 1}, {1, 0}, {2, 3}, {3, 2}};
  const float sg[4] = {-1.f, 1.f, -1.f, 1.f};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float2 u = si[sp[q][0] * 3 + a], v = tj[sp[q][1] * 3 + b];
    r.x += sg[q] * (u.x * v.x - u.y * v.y);
    r.y += sg[q] * (u.x * v.y + u.y * v.x);
  }
  return r;
}

// One block: a 64 x 64 tile of B[(i,j)][(k,alpha)] of one time slice.
// s: n slab vectors (FP64, [n][nsite][12]); slice blockIdx.z covers the
// slab-local sites lo0 + z * t_stride_sites .. + S3.
__global__ void __launch_bounds__(256, 2) k_nucleon_block(int n, long long nsite, const double2* s, int conj,
                                                       int S3, long long lo0, int t_stride_sites, double2* B) {
  __shared__ float2 fi[XS][TI][13], fj[XS][TJ][13];  // 13: rows on distinct banks
  __shared__ __align__(16) float2 Ds[XS * 3][TI * TJ], Ss[XS * 3][TK * 4];
  extern __shared__ float2 tot[];  // [16][256]: second-level sums of each thread's 4 x 4 tile
  const int nti = (n + TI - 1) / TI, ntj = (n + TJ - 1) / TJ;
  const int tile = blockIdx.x;
  const int i0 = (tile % nti) * TI, j0 = ((tile / nti) % ntj) * TJ;
  const int k0 = blockIdx.y * TK;
  const int t = blockIdx.z;
  const long long lo = lo0 + (long long)t * t_stride_sites;
  // thread tile: rows tr*4 .. tr*4+3 and columns 2tc, 2tc+1, 32+2tc, 32+2tc+1 (so that the
  // 16 threads of a row read 256 contiguous bytes of S per 16-byte load)
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  float2 acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      acc[p][q] = make_float2(0.f, 0.f);
      tot[(p * 4 + q) * 256 + threadIdx.x] = make_float2(0.f, 0.f);
    }
  const float cs = conj ? -1.f : 1.f;
  int stage = 0;
  for (int x0 = 0; x0 < S3; x0 += XS, stage++) {
    // the i and j fields of the stage's sites, FP64 -> FP32 (conjugated for the xi side)
    for (int e = threadIdx.x; e < XS * (TI + TJ) * 12; e += blockDim.x) {
      const int comp = e % 12, r = e / 12;
      const int x = r % XS, w = r / XS;  // w: 0..TI+TJ-1
      const int f = w < TI ? i0 + w : j0 + w - TI;
      float2 v = make_float2(0.f, 0.f);
      if (f < n && x0 + x < S3) {
        const double2 d = s[((long long)f * nsite + lo + x0 + x) * 12 + comp];
        v = make_float2((float)d.x, cs * (float)d.y);
      }
      if (w < TI) fi[x][w][comp] = v;
      else fj[x][w - TI][comp] = v;
    }
    // S[(x, c)][(k, alpha)] = s_k(x)[alpha][c]; consecutive threads read one site's 12 components
    for (int e = threadIdx.x; e < XS * TK * 12; e += blockDim.x) {
      const int comp = e % 12, r = e / 12;
      const int x = r % XS, kk = r / XS;
      const int al = comp / 3, c = comp % 3;
      const int k = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (k < n && x0 + x < S3) {
        const double2 d = s[((long long)k * nsite + lo + x0 + x) * 12 + comp];
        v = make_float2((float)d.x, cs * (float)d.y);
      }
      Ss[x * 3 + c][kk * 4 + al] = v;
    }
    __syncthreads();
    // diquark D[(x, c)][(i, j)], the three colours c of one (x, i, j) from one read of s_i(x), s_j(x)
    for (int e = threadIdx.x; e < XS * TI * TJ; e += blockDim.x) {
      const int pr = e % (TI * TJ), x = e / (TI * TJ);
      const int ii = pr / TJ, jj = pr % TJ;
      float2 u[12], v[12];
#pragma unroll
      for (int q = 0; q < 12; q++) {
        u[q] = fi[x][ii][q];
        v[q] = fj[x][jj][q];
      }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;  // eps^{abc} = +1 for (a, b) and -1 for (b, a)
        const float2 p = cg5_pair(u, v, a, b), m = cg5_pair(u, v, b, a);
        Ds[x * 3 + c][pr] = make_float2(p.x - m.x, p.y - m.y);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < XS * 3; r++) {
      float2 av[4], bv[4];
      {
        const float4* pa = reinterpret_cast<const float4*>(&Ds[r][tr * 4]);
        const float4 a0 = pa[0], a1 = pa[1];
        const float4 b0 = *reinterpret_cast<const float4*>(&Ss[r][2 * tc]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Ss[r][32 + 2 * tc]);
        av[0] = make_float2(a0.x, a0.y);
        av[1] = make_float2(a0.z, a0.w);
        av[2] = make_float2(a1.x, a1.y);
        av[3] = make_float2(a1.z, a1.w);
        bv[0] = make_float2(b0.x, b0.y);
        bv[1] = make_float2(b0.z, b0.w);
        bv[2] = make_float2(b1.x, b1.y);
        bv[3] = make_float2(b1.z, b1.w);
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          acc[p][q].x = fmaf(av[p].x, bv[q].x, fmaf(-av[p].y, bv[q].y, acc[p][q].x));
          acc[p][q].y = fmaf(av[p].x, bv[q].y, fmaf(av[p].y, bv[q].x, acc[p][q].y));
        }
    }
    __syncthreads();
    if ((stage + 1) % FLUSH == 0) {
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          float2& t2 = tot[(p * 4 + q) * 256 + threadIdx.x];
          t2.x += acc[p][q].x;
          t2.y += acc[p][q].y;
          acc[p][q] = make_float2(0.f, 0.f);
        }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const int pr = tr * 4 + p;
    const int i = i0 + pr / TJ, j = j0 + pr % TJ;
    if (i >= n || j >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int col = q < 2 ? 2 * tc + q : 32 + 2 * tc + q - 2;
      const int k = k0 + col / 4, al = col % 4;
      if (k >= n) continue;
      const float2 t2 = tot[(p * 4 + q) * 256 + threadIdx.x];
      const double2 v = make_double2((double)t2.x + acc[p][q].x, (double)t2.y + acc[p][q].y);
      B[((((long long)t * n + i) * n + j) * n + k) * 4 + al] = v;
    }
  }
}

// W[ix][iy] = (W1, W2) for slices ix of B_xi and iy of B_eta; one block per
// (ix, iy), FP64.  g5 P_- = g5 (1 - g0)/2 in the chiral basis: rows
// (1/2)[[1,0,1,0],[0,1,0,1],[1,0,1,0],[0,1,0,1]] times diag(1,1,-1,-1) on the
// left: M = (1/2)[[1,0,1,0],[0,1,0,1],[-1,0,-1,0],[0,-1,0,-1]].
__global__ void __launch_bounds__(256) k_nucleon_contract(int n, int ny, const double2* Bx, const double2* By,
                                                          double2* W) {
  const int ix = blockIdx.x / ny, iy = blockIdx.x % ny;
  const long long n3 = (long long)n * n * n;
  const double2* bx = Bx + (long long)ix * n3 * 4;
  const double2* by = By + (long long)iy * n3 * 4;
  const double M[4][4] = {{0.5, 0, 0.5, 0}, {0, 0.5, 0, 0.5}, {-0.5, 0, -0.5, 0}, {0, -0.5, 0, -0.5}};
  double w1r = 0, w1i = 0, w2r = 0, w2i = 0;
  for (long long e = threadIdx.x; e < n3; e += blockDim.x) {
    const int k = (int)(e % n), j = (int)((e / n) % n), i = (int)(e / ((long long)n * n));
    const double2* yv = by + e * 4;                                      // B_eta[i][j][k]
    const double2* x1 = bx + ((((long long)j * n + i) * n) + k) * 4;   // B_xi[j][i][k]
    const double2* x2 = bx + ((((long long)k * n + i) * n) + j) * 4;   // B_xi[k][i][j]
    double2 my[4];
#pragma unroll
    for (int g = 0; g < 4; g++) {
      double re = 0, im = 0;
#pragma unroll
      for (int d = 0; d < 4; d++) {
        re += M[g][d] * yv[d].x;
        im += M[g][d] * yv[d].y;
      }
      my[g] = make_double2(re, im);
    }
#pragma unroll
    for (int g = 0; g < 4; g++) {
      const double2 a = x1[g], b = x2[g];
      w1r += a.x * my[g].x - a.y * my[g].y;
      w1i += a.x * my[g].y + a.y * my[g].x;
      w2r += b.x * my[g].x - b.y * my[g].y;
      w2i += b.x * my[g].y + b.y * my[g].x;
    }
  }
  __shared__ double sh[4][8];
  double v[4] = {w1r, w1i, w2r, w2i};
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 4; q++) sh[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; q++)
      for (int w = 0; w < 8; w++) r[q] += sh[q][w];
    W[(long long)blockIdx.x * 2] = make_double2(-r[0], -r[1]);
    W[(long long)blockIdx.x * 2 + 1] = make_double2(-r[2], -r[3]);
  }
}

// out[e] = (1/count) sum_j in[j * size + e], summed in j order (FP64).
__global__ void k_level_mean(long long size, int count, const double2* in, double2* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < size;
       e += (long long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < count; j++) {
      const double2 v = in[(long long)j * size + e];
      re += v.x;
      im += v.y;
    }
    out[e] = make_double2(re / count, im / count);
  }
}

// The two nucleon Wick contractions from a point source to every sink y of a
// time slice (the contractions behind eq. nucleon_prop_factorized), one warp
// per site y, FP64.  S(y) = the 12 x 12 propagator matrix at y,
// S_{(mu a),(nu b)} = prop[3 nu + b][y][mu][a], staged in shared memory; with
// the non-zero entries of C g5 (mu -> nu(mu), sign) and of g5 P_- (M above):
//   W1 = sum_{cc'} T^{cc'} U^{cc'},
//     T^{cc'} = sum eps_{abc} eps_{a'b'c'} cg5(mu) cg5(mu') S_{mu a, nu(mu') b'} S_{nu(mu) b, mu' a'},
//     U^{cc'} = sum_{gam del} M_{gam del} S_{del c, gam c'};
//   W2 = sum eps_{abc} eps_{a'b'c'} cg5(mu) cg5(mu') M_{gam del}
//            S_{mu a, nu(mu') b'} S_{nu(mu) b, gam c'} S_{del c, mu' a'}.
// Each block sums its sites; partial[prop][slice][block] = (W1, W2).
constexpr int NP_WARPS = 4;

LQ_DI double2 cmul_d(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__global__ void __launch_bounds__(32 * NP_WARPS) k_nucleon_point(int S3, long long V, const double2* prop,
                                                                 long long prop_stride, int t0, double2* partial) {
  __shared__ double2 sm[NP_WARPS][144];
  __shared__ double2 red[NP_WARPS][2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int site = blockIdx.x * NP_WARPS + w;  // site within the slice
  const int slice = blockIdx.y;
  const double2* P = prop + (long long)blockIdx.z * prop_stride;
  const bool on = site < S3;
  const long long y = (long long)(t0 + slice) * S3 + site;
  if (on)
    for (int q = lane; q < 144; q += 32) {
      const int col = q / 12, e = q - col * 12;
      sm[w][q] = P[((long long)col * V + y) * 12 + e];
    }
  __syncwarp();
  // S_{(mu a),(nu b)} = sm[(3 nu + b) * 12 + 3 mu + a]
  auto Sx = [&](int mu, int a, int nu, int b) { return sm[w][(3 * nu + b) * 12 + 3 * mu + a]; };
  const int nu_of[4] = {1, 0, 3, 2};
  const double cg[4] = {-1.0, 1.0, -1.0, 1.0};
  // g5 P_-: row gam has entries at del = gam % 2 and gam % 2 + 2, value +1/2 (gam < 2) or -1/2
  const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  const double psg[6] = {1, 1, 1, -1, -1, -1};
  double2 w1 = make_double2(0.0, 0.0), w2 = make_double2(0.0, 0.0);
  if (on) {
    // W1: 36 tasks (c, c', mu), each a 16-term part of T^{cc'} times U^{cc'}
    for (int task = lane; task < 36; task += 32) {
      const int c = task / 12, cp = (task / 4) % 3, mu = task % 4;
      const int a0 = (c + 1) % 3, b0 = (c + 2) % 3, ap0 = (cp + 1) % 3, bp0 = (cp + 2) % 3;
      double2 t = make_double2(0.0, 0.0);
      for (int o = 0; o < 2; o++) {
        const int a = o ? b0 : a0, b = o ? a0 : b0;
        const double so = o ? -1.0 : 1.0;  // eps_{abc}
        for (int op = 0; op < 2; op++) {
          const int ap = op ? bp0 : ap0, bp = op ? ap0 : bp0;
          const double sop = op ? -1.0 : 1.0;  // eps_{a'b'c'}
          for (int mup = 0; mup < 4; mup++) {
            const double f = so * sop * cg[mu] * cg[mup];
            const double2 p = cmul_d(Sx(mu, a, nu_of[mup], bp), Sx(nu_of[mu], b, mup, ap));
            t.x += f * p.x;
            t.y += f * p.y;
          }
        }
      }
      double2 u = make_double2(0.0, 0.0);
      for (int gam = 0; gam < 4; gam++) {
        const double m = gam < 2 ? 0.5 : -0.5;
        for (int k = 0; k < 2; k++) {
          const double2 v = Sx(gam % 2 + 2 * k, c, gam, cp);
          u.x += m * v.x;
          u.y += m * v.y;
        }
      }
      const double2 tu = cmul_d(t, u);
      w1.x += tu.x;
      w1.y += tu.y;
    }
    // W2: 36 colour pairs x 4 mu x 4 mu' x 8 (gam, del) = 4608 terms, 144 per lane
    for (int e = lane; e < 4608; e += 32) {
      const int pc = e / 128, r = e % 128;
      const int mu = r / 32, mup = (r / 8) % 4, gd = r % 8;
      const int gam = gd / 2, del = gam % 2 + 2 * (gd % 2);
      const int* pa = perm[pc / 6];
      const int* pb = perm[pc % 6];
      const double f = psg[pc / 6] * psg[pc % 6] * cg[mu] * cg[mup] * (gam < 2 ? 0.5 : -0.5);
      const double2 p = cmul_d(cmul_d(Sx(mu, pa[0], nu_of[mup], pb[1]), Sx(nu_of[mu], pa[1], gam, pb[2])),
                               Sx(del, pa[2], mup, pb[0]));
      w2.x += f * p.x;
      w2.y += f * p.y;
    }
  }
  double v[4] = {w1.x, w1.y, w2.x, w2.y};
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0) {
    red[w][0] = make_double2(v[0], v[1]);
    red[w][1] = make_double2(v[2], v[3]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 r1 = make_double2(0.0, 0.0), r2 = make_double2(0.0, 0.0);
    for (int q = 0; q < NP_WARPS; q++) {
      r1.x += red[q][0].x;
      r1.y += red[q][0].y;
      r2.x += red[q][1].x;
      r2.y += red[q][1].y;
    }
    const long long o = (((long long)blockIdx.z * gridDim.y + slice) * gridDim.x + blockIdx.x) * 2;
    partial[o] = r1;
    partial[o + 1] = r2;
  }
}

// W[p][t] = sum over the blocks of (prop p, slice t), in block order.
__global__ void k_nucleon_point_sum(int nblk, int n_t, int n_prop, const double2* partial, double2* W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t * n_prop) return;
  double2 r1 = make_double2(0.0, 0.0), r2 = make_double2(0.0, 0.0);
  const double2* p = partial + (long long)i * nblk * 2;
  for (int b = 0; b < nblk; b++) {
    r1.x += p[2 * b].x;
    r1.y += p[2 * b].y;
    r2.x += p[2 * b + 1].x;
    r2.y += p[2 * b + 1].y;
  }
  W[2 * i] = r1;
  W[2 * i + 1] = r2;
}

// The tensor-core block kernel (nucleon_tc.cu) unless LQCD_NUCLEON_TC=0 selects the FP32-FMA
// one; read at every call
bool use_tensor_cores() {
  const char* e = getenv("LQCD_NUCLEON_TC");
  return e ? atoi(e) != 0 : true;
}

}  // namespace

int lq_nucleon_point(const lqcd_lattice* L, int n_prop, const double2* prop, int t0, int n_t, double2* partial,
                     double2* W, cudaStream_t st) {
  const int S3 = (int)L->S3;
  const int nblk = (S3 + NP_WARPS - 1) / NP_WARPS;
  k_nucleon_point<<<dim3((unsigned)nblk, (unsigned)n_t, (unsigned)n_prop), 32 * NP_WARPS, 0, st>>>(
      S3, L->V, prop, (long long)12 * L->V * 12, t0, partial);
  RC_LAUNCH();
  k_nucleon_point_sum<<<(unsigned)((n_t * n_prop + 127) / 128), 128, 0, st>>>(nblk, n_t, n_prop, partial, W);
  return launched_here();
}

long long lq_nucleon_point_partial_words(const lqcd_lattice* L, int n_prop, int n_t) {
  return (long long)((L->S3 + NP_WARPS - 1) / NP_WARPS) * n_t * n_prop * 2;
}

extern "C" int lqcd_nucleon_point(lqcd_lattice* L, int n_prop, const double* prop, int t0, int n_t, double* W,
                                  void* stream) {
  if (!L || !prop || !W || n_prop < 1 || n_t < 1 || t0 < 0 || t0 + n_t > L->dims[0] || n_prop > 65535) {
    lq_set_error("nucleon_point: bad arguments (1 <= n_prop, slices t0..t0+n_t-1 inside the lattice)");
    return LQCD_EBADARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* partial = nullptr;
  const size_t bytes = sizeof(double2) * (size_t)lq_nucleon_point_partial_words(L, n_prop, n_t);
  if (cudaMallocAsync(&partial, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    lq_set_error("nucleon_point: device allocation failed");
    return LQCD_ENOMEM;
  }
  const int rc = lq_nucleon_point(L, n_prop, (const double2*)prop, t0, n_t, (double2*)partial, (double2*)W, st);
  cudaFreeAsync(partial, st);
  return rc;
}

extern "C" int lqcd_level_mean(long long size, int count, const double* in, double* out, void* stream) {
  if (!in || !out || size < 1 || count < 1) {
    lq_set_error("level_mean: bad arguments");
    return LQCD_EBADARG;
  }
  long long blocks = (size + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_level_mean<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(size, count, (const double2*)in, (double2*)out);
  return launched_here();
}

extern "C" int lqcd_nucleon_blocks(lqcd_lattice* L, const lqcd_slab* slab, int n, const double* s, int conj, int t0,
                                   int n_t, double* B, void* stream) {
  if (!L || !slab || !s || !B || n < 1 || n > 1024 || n_t < 1 || slab->t0 < 0 || slab->t1 < slab->t0 ||
      slab->t1 >= L->dims[0] || t0 < slab->t0 || t0 + n_t - 1 > slab->t1) {
    lq_set_error("nucleon_blocks: bad arguments (1 <= n <= 1024, slices t0..t0+n_t-1 inside the slab)");
    return LQCD_EBADARG;
  }
  const int S3 = (int)L->S3;
  const long long nsite = (long long)(slab->t1 - slab->t0 + 1) * S3;
  if (use_tensor_cores())
    return lq_nucleon_blocks_tc(n, nsite, (const double2*)s, conj, S3, (long long)(t0 - slab->t0) * S3, n_t,
                                (double2*)B, (cudaStream_t)stream);
  const int nti = (n + TI - 1) / TI, ntj = (n + TJ - 1) / TJ, ntk = (n + TK - 1) / TK;
  {
    // static + dynamic shared memory exceed the 48 KB default: opt in once per device
    static std::mutex mu;
    static std::vector<int> opted;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      lq_set_error("nucleon_blocks: no current device");
      return LQCD_ECUDA;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(opted.begin(), opted.end(), dev) == opted.end()) {
      if (cudaFuncSetAttribute(k_nucleon_block, cudaFuncAttributeMaxDynamicSharedMemorySize, TOT_BYTES) !=
          cudaSuccess) {
        cudaGetLastError();
        lq_set_error("nucleon_blocks: shared-memory opt-in failed");
        return LQCD_ECUDA;
      }
      opted.push_back(dev);
    }
  }
  k_nucleon_block<<<dim3((unsigned)(nti * ntj), (unsigned)ntk, (unsigned)n_t), 256, TOT_BYTES, (cudaStream_t)stream>>>(
      n, nsite, (const double2*)s, conj, S3, (long long)(t0 - slab->t0) * S3, S3, (double2*)B);
  return launched_here();
}

extern "C" int lqcd_nucleon_contract(int n, int n_x, const double* B_xi, int n_y, const double* B_eta, double* W,
                                     void* stream) {
  if (!B_xi || !B_eta || !W || n < 1 || n > 1024 || n_x < 1 || n_y < 1 || (long long)n_x * n_y >= (1LL << 31)) {
    lq_set_error("nucleon_contract: bad arguments");
    return LQCD_EBADARG;
  }
  k_nucleon_contract<<<(unsigned)(n_x * n_y), 256, 0, (cudaStream_t)stream>>>(n, n_y, (const double2*)B_xi,
                                                                              (const double2*)B_eta, (double2*)W);
  return launched_here();
}
