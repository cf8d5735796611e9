// Gauge-field preparation: even-odd link packing in three precisions with
// an SU(3) check, and the clover blocks A(x) with their inverses.
//
// Clover term (Sheikholeslami-Wohlert), added to the diagonal of D:
//   A(x) = 1/(2 kappa) + c_sw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu(x),
//   Fhat_mu_nu = (Q_mu_nu - Q_mu_nu^dag) / 8,  Q = the four plaquette leaves.
// In the chiral basis sigma_mu_nu = (i/2)[g_mu, g_nu] is block diagonal:
//   sigma_0k = diag(+s_k, -s_k),  sigma_jk = -eps_jkl diag(s_l, s_l),
// so with E_l = Fhat_0l and M_1 = Fhat_23, M_2 = Fhat_31, M_3 = Fhat_12,
//   A = diag(B+, B-),  B+- = 1/(2 kappa) + sum_l s_l (x) H+-_l,
//   H+-_l = c_sw (i/2) (+-E_l - M_l)   (Hermitian 3x3),
//   B = [[d + H_3, H_1 - i H_2], [H_1 + i H_2, d - H_3]].
// Open time BC: the link U_0 leaving the last time slice is absent, so every
// leaf through it is zero.
#include <cstdio>

#include "internal.h"

namespace lq {

typedef cx<double> cd;

LQ_DI su3<double> ld_nat(const double2* U, long long i, int mu) {
  su3<double> u;
  const double2* b = U + (i * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = b[k];
    u.m[k / 3][k % 3] = {v.x, v.y};
  }
  return u;
}

LQ_DI su3<double> mm(const su3<double>& a, const su3<double>& b) {
  su3<double> r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd t = a.m[i][0] * b.m[0][j];
      fma_c(t, a.m[i][1], b.m[1][j]);
      fma_c(t, a.m[i][2], b.m[2][j]);
      r.m[i][j] = t;
    }
  return r;
}

// a * b^dag
LQ_DI su3<double> mmd(const su3<double>& a, const su3<double>& b) {
  su3<double> r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd t = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) t = t + a.m[i][k] * conj(b.m[j][k]);
      r.m[i][j] = t;
    }
  return r;
}

// a^dag * b
LQ_DI su3<double> mdm(const su3<double>& a, const su3<double>& b) {
  su3<double> r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd t = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) t = t + conj(a.m[k][i]) * b.m[k][j];
      r.m[i][j] = t;
    }
  return r;
}

LQ_DI long long nat_index(const Geom& g, const int x[4]) {
  return (((long long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

LQ_DI void nat_coords(const Geom& g, long long i, int x[4]) {
  x[3] = (int)(i % g.L[3]);
  i /= g.L[3];
  x[2] = (int)(i % g.L[2]);
  i /= g.L[2];
  x[1] = (int)(i % g.L[1]);
  x[0] = (int)(i / g.L[1]);
}

// ------------------------------------------------------------- link packing
__global__ void k_pack_links(Geom g, const double2* U, double2* U64, float4* U32, uint2* U16,
                             unsigned long long* maxdev) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  int x[4];
  nat_coords(g, i, x);
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long long cb = i >> 1;
  double dev = 0.0;
  for (int mu = 0; mu < 4; mu++) {
    su3<double> u = ld_nat(U, i, mu);
    // unitarity: |U U^dag - 1|, |det U - 1|
    su3<double> uu = mmd(u, u);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        cd e = uu.m[a][b];
        if (a == b) e.re -= 1.0;
        dev = fmax(dev, sqrt(norm2(e)));
      }
    cd det = u.m[0][0] * (u.m[1][1] * u.m[2][2] - u.m[1][2] * u.m[2][1]) -
             u.m[0][1] * (u.m[1][0] * u.m[2][2] - u.m[1][2] * u.m[2][0]) +
             u.m[0][2] * (u.m[1][0] * u.m[2][1] - u.m[1][1] * u.m[2][0]);
    det.re -= 1.0;
    dev = fmax(dev, sqrt(norm2(det)));
    const long long base = (long long)(p * 4 + mu);
#pragma unroll
    for (int k = 0; k < 9; k++) U64[(base * 9 + k) * g.Vh + cb] = make_double2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
    float r[12];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      r[2 * k] = (float)u.m[k / 3][k % 3].re;
      r[2 * k + 1] = (float)u.m[k / 3][k % 3].im;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
      U32[(base * 3 + k) * g.Vh + cb] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
      __half2 h0 = __floats2half2_rn(r[4 * k], r[4 * k + 1]);
      __half2 h1 = __floats2half2_rn(r[4 * k + 2], r[4 * k + 3]);
      U16[(base * 3 + k) * g.Vh + cb] = make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1));
    }
  }
  if (!(dev == dev)) dev = 1e300;  // NaN counts as non-unitary
  atomicMax(maxdev, (unsigned long long)__double_as_longlong(dev));
}

// ------------------------------------------------------------------ clover
LQ_DI su3<double> link_bc(const Geom& g, const double2* U, const int x[4], int mu) {
  if (g.bc_t == 0 && mu == 0 && x[0] == g.L[0] - 1) {
    su3<double> z;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) z.m[a][b] = {0, 0};
    return z;
  }
  return ld_nat(U, nat_index(g, x), mu);
}

LQ_DI void shift(const Geom& g, const int x[4], int mu, int d, int y[4]) {
#pragma unroll
  for (int k = 0; k < 4; k++) y[k] = x[k];
  y[mu] += d;
  if (y[mu] < 0) y[mu] += g.L[mu];
  if (y[mu] >= g.L[mu]) y[mu] -= g.L[mu];
}

// Fhat_mu_nu(x) = (Q - Q^dag)/8, Q = sum of the 4 leaves at x (mu -> nu).
LQ_DI su3<double> fhat(const Geom& g, const double2* U, const int x[4], int mu, int nu) {
  int xpm[4], xpn[4], xmm[4], xmn[4], xmmpn[4], xmmmn[4], xmnpm[4];
  shift(g, x, mu, 1, xpm);
  shift(g, x, nu, 1, xpn);
  shift(g, x, mu, -1, xmm);
  shift(g, x, nu, -1, xmn);
  shift(g, xmm, nu, 1, xmmpn);
  shift(g, xmm, nu, -1, xmmmn);
  shift(g, xmn, mu, 1, xmnpm);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  su3<double> q = mmd(mmd(mm(link_bc(g, U, x, mu), link_bc(g, U, xpm, nu)), link_bc(g, U, xpn, mu)), link_bc(g, U, x, nu));
  // leaf 2: U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  su3<double> l2 =
      mm(mmd(mmd(link_bc(g, U, x, nu), link_bc(g, U, xmmpn, mu)), link_bc(g, U, xmm, nu)), link_bc(g, U, xmm, mu));
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  //        = [U_nu(x-mu-nu) U_mu(x-mu)]^dag U_mu(x-mu-nu) U_nu(x-nu)
  su3<double> l3 = mm(mdm(mm(link_bc(g, U, xmmmn, nu), link_bc(g, U, xmm, mu)), link_bc(g, U, xmmmn, mu)),
                      link_bc(g, U, xmn, nu));
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
  su3<double> l4 = mmd(mm(mdm(link_bc(g, U, xmn, nu), link_bc(g, U, xmn, mu)), link_bc(g, U, xmnpm, nu)), link_bc(g, U, x, mu));
  su3<double> f;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      cd t = q.m[a][b] + l2.m[a][b] + l3.m[a][b] + l4.m[a][b];
      cd tt = q.m[b][a] + l2.m[b][a] + l3.m[b][a] + l4.m[b][a];
      f.m[a][b] = 0.125 * (t - conj(tt));
    }
  return f;
}


// Pack the 6x6 Hermitian block B into 36 reals: 6 diagonal, then the 15
// entries below the diagonal row by row.
LQ_DI void pack_herm6(const cd B[6][6], double out[36]) {
  for (int r = 0; r < 6; r++) out[r] = B[r][r].re;
  int q = 6;
  for (int r = 1; r < 6; r++)
    for (int c = 0; c < r; c++) {
      // Hermitian part of the pair (r,c), (c,r)
      out[q] = 0.5 * (B[r][c].re + B[c][r].re);
      out[q + 1] = 0.5 * (B[r][c].im - B[c][r].im);
      q += 2;
    }
}

// Gauss-Jordan inversion with partial pivoting (6x6 complex).  Returns
// false for a singular block.
LQ_DI bool invert6(const cd B[6][6], cd R[6][6]) {
  cd M[6][12];
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) {
      M[r][c] = B[r][c];
      M[r][6 + c] = {r == c ? 1.0 : 0.0, 0.0};
    }
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = norm2(M[col][col]);
    for (int r = col + 1; r < 6; r++) {
      double v = norm2(M[r][col]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 0.0)) return false;
    if (piv != col)
      for (int c = 0; c < 12; c++) {
        cd t = M[col][c];
        M[col][c] = M[piv][c];
        M[piv][c] = t;
      }
    cd d = M[col][col];
    double dn = norm2(d);
    cd inv = {d.re / dn, -d.im / dn};
    for (int c = 0; c < 12; c++) M[col][c] = M[col][c] * inv;
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      cd f = M[r][col];
      if (f.re == 0.0 && f.im == 0.0) continue;
      for (int c = 0; c < 12; c++) M[r][c] = M[r][c] - f * M[col][c];
    }
  }
  for (int r = 0; r < 6; r++)
    for (int c = 0; c < 6; c++) R[r][c] = M[r][6 + c];
  return true;
}

__global__ void k_clover(Geom g, const double2* U, double kappa, double csw, double2* A64, double2* Ai64, float4* A32,
                         float4* Ai32, int* fail) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  int x[4];
  nat_coords(g, i, x);
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long long cb = i >> 1;
  const long long Vh = g.Vh;
  const double d = 1.0 / (2.0 * kappa);
  su3<double> E[3], M[3];
  if (csw != 0.0) {
    for (int l = 0; l < 3; l++) E[l] = fhat(g, U, x, 0, l + 1);
    M[0] = fhat(g, U, x, 2, 3);
    M[1] = fhat(g, U, x, 3, 1);
    M[2] = fhat(g, U, x, 1, 2);
  }
  for (int blk = 0; blk < 2; blk++) {
    const double sg = blk == 0 ? 1.0 : -1.0;
    cd H[3][3][3];
    for (int l = 0; l < 3; l++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          if (csw == 0.0) {
            H[l][a][b] = {0.0, 0.0};
          } else {
            cd t = sg * E[l].m[a][b] - M[l].m[a][b];
            H[l][a][b] = (0.5 * csw) * ti(t);  // c_sw (i/2) (+-E_l - M_l)
          }
        }
    cd B[6][6];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        cd dd = {a == b ? d : 0.0, 0.0};
        B[a][b] = dd + H[2][a][b];
        B[3 + a][3 + b] = dd - H[2][a][b];
        B[a][3 + b] = H[0][a][b] - ti(H[1][a][b]);
        B[3 + a][b] = H[0][a][b] + ti(H[1][a][b]);
      }
    double pk[36];
    pack_herm6(B, pk);
    for (int k = 0; k < 18; k++) A64[((long long)p * 36 + blk * 18 + k) * Vh + cb] = make_double2(pk[2 * k], pk[2 * k + 1]);
    for (int k = 0; k < 9; k++)
      A32[((long long)p * 18 + blk * 9 + k) * Vh + cb] =
          make_float4((float)pk[4 * k], (float)pk[4 * k + 1], (float)pk[4 * k + 2], (float)pk[4 * k + 3]);
    if (p == 0) {
      cd R[6][6];
      if (!invert6(B, R)) {
        atomicExch(fail, 1);
        for (int r = 0; r < 6; r++)
          for (int c = 0; c < 6; c++) R[r][c] = {0.0, 0.0};
      }
      pack_herm6(R, pk);
      for (int k = 0; k < 18; k++) Ai64[((long long)blk * 18 + k) * Vh + cb] = make_double2(pk[2 * k], pk[2 * k + 1]);
      for (int k = 0; k < 9; k++)
        Ai32[((long long)blk * 9 + k) * Vh + cb] =
            make_float4((float)pk[4 * k], (float)pk[4 * k + 1], (float)pk[4 * k + 2], (float)pk[4 * k + 3]);
    }
  }
}

}  // namespace lq

// ------------------------------------------------------------------ launchers
int lq_launch_pack_links(const lq::Geom& g, const double2* U, double2* U64, float4* U32, uint2* U16,
                         unsigned long long* maxdev, cudaStream_t st) {
  const long long V = 2 * g.Vh;
  lq::k_pack_links<<<(unsigned)((V + 127) / 128), 128, 0, st>>>(g, U, U64, U32, U16, maxdev);
  lq_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int lq_launch_clover(const lq::Geom& g, const double2* U, double kappa, double csw, double2* A64, double2* Ai64,
                     float4* A32, float4* Ai32, int* fail, cudaStream_t st) {
  const long long V = 2 * g.Vh;
  lq::k_clover<<<(unsigned)((V + 63) / 64), 64, 0, st>>>(g, U, kappa, csw, A64, Ai64, A32, Ai32, fail);
  lq_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
