// Gauge-link force of the domain-local pseudofermion action
//   S = phi^dag (D_L^dag D_L)^{-1} phi,   X = (D_L^dag D_L)^{-1} phi,  Y = D_L X,
//   F^a_rho(x) = dS/domega  for U_rho(x) -> exp(i omega T_a) U_rho(x)
//              = -2 Re <Y, (dD_L/domega) X>,        T_a = lambda_a / 2.
//
// Hopping part (link l = U_rho(x), both ends in the slab, boundary sign f):
//   F^a = f Re tr[i T_a (l W1 - W2 l^dag)],
//   W1 = sum_s ((1 - g_rho) X(x+rho))_s (x) Y(x)_s^dag,
//   W2 = sum_s ((1 + g_rho) X(x))_s (x) Y(x+rho)_s^dag      (3x3 colour outer products).
// Clover part: with Xi_mn(z)[b][a] = sum_{s,t} sigma_mn[s][t] X(z)[t][b] conj(Y(z)[s][a])
// and K_mn = c_sw (i/4) (Xi_mn + Xi_mn^dag) (zero outside the slab),
//   F^a = -1/2 Re tr[i T_a G],  G = sum_{s != rho} ( l M_a + M_c ),
// where, for the plaquette above the link (corners x, x+rho, x+rho+s, x+s;
// b = U_s(x+rho), c = U_rho(x+s)^dag, d = U_s(x)^dag, K = K_{rho s}):
//   M_a = b c d K(x) + K(x+rho) b c d + b K(x+rho+s) c d + b c K(x+s) d,
// and for the plaquette below (w = x-s; a' = U_rho(w), b' = U_s(w+rho), d' = U_s(w)^dag):
//   M_c = -[d' K(w) a' b' + d' a' K(w+rho) b' + d' a' b' K(x+rho) + K(x) d' a' b'] l^dag.
// Each of the four leaves of the clover at z is one plaquette entered at a
// different corner, so summing over the link's two plaquettes per plane and
// their four corners covers every leaf that contains the link.  Under open
// time BC the link leaving the last time slice is absent (zero): every
// product through it vanishes and its own force is zero.
#include "dslash.cuh"
#include "internal.h"

namespace lq {

typedef cx<double> cd;
typedef su3<double> M3;

LQ_DI M3 zero3() {
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) r.m[a][b] = {0.0, 0.0};
  return r;
}
LQ_DI M3 mul(const M3& a, const M3& b) {
  M3 r;
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
LQ_DI M3 dagm(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i][j] = conj(a.m[j][i]);
  return r;
}
LQ_DI M3 add(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i][j] = a.m[i][j] + b.m[i][j];
  return r;
}
LQ_DI M3 scl(double s, const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i][j] = s * a.m[i][j];
  return r;
}

LQ_DI long long nidx(const Geom& g, const int x[4]) {
  return (((long long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}
LQ_DI void ncoords(const Geom& g, long long i, int x[4]) {
  x[3] = (int)(i % g.L[3]);
  i /= g.L[3];
  x[2] = (int)(i % g.L[2]);
  i /= g.L[2];
  x[1] = (int)(i % g.L[1]);
  x[0] = (int)(i / g.L[1]);
}
LQ_DI void shifted(const Geom& g, const int x[4], int mu, int d, int y[4]) {
#pragma unroll
  for (int k = 0; k < 4; k++) y[k] = x[k];
  y[mu] += d;
  if (y[mu] < 0) y[mu] += g.L[mu];
  if (y[mu] >= g.L[mu]) y[mu] -= g.L[mu];
}

// U_mu(x) from the even-odd FP64 link store; zero for the absent open-BC link.
LQ_DI M3 link(const Geom& g, const FieldPtrs& f, const int x[4], int mu) {
  if (g.bc_t == 0 && mu == 0 && x[0] == g.L[0] - 1) return zero3();
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  return LinkIO<64>::load(f, p, mu, g.Vh, nidx(g, x) >> 1);
}

// plane index of the unordered pair {mu, nu}: (0,1)(0,2)(0,3)(1,2)(1,3)(2,3)
LQ_DI int plane_of(int mu, int nu) {
  int a = mu < nu ? mu : nu, b = mu < nu ? nu : mu;
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// K_{mu nu}(z) (ordered pair; K_{nu mu} = -K_{mu nu}), stored for mu < nu.
LQ_DI M3 load_K(const Geom& g, const double2* K, const int z[4], int mu, int nu) {
  const long long i = nidx(g, z);
  const double2* b = K + (i * 6 + plane_of(mu, nu)) * 9;
  M3 r;
  const double s = mu < nu ? 1.0 : -1.0;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = b[k];
    r.m[k / 3][k % 3] = {s * v.x, s * v.y};
  }
  return r;
}

// Per site of the slab: K_mn = c_sw (i/4)(Xi + Xi^dag) for the 6 planes.
// sigma in the chiral basis: sigma_0k = diag(s_k, -s_k), sigma_jk = -eps_jkl diag(s_l, s_l).
__global__ void k_force_K(Geom g, int t0, int t1, double csw, const double2* X, const double2* Y, double2* K) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  const long long s3 = 2 * g.S3h;
  const int t = (int)(i / s3);
  double2* out = K + i * 54;
  if (t < t0 || t > t1 || csw == 0.0) {
    for (int k = 0; k < 54; k++) out[k] = make_double2(0.0, 0.0);
    return;
  }
  cd x[12], y[12];
  for (int k = 0; k < 12; k++) {
    double2 a = X[i * 12 + k], b = Y[i * 12 + k];
    x[k] = {a.x, a.y};
    y[k] = {b.x, b.y};
  }
  // O[chi][s][t][b][a] = X[2chi+t][b] conj(Y[2chi+s][a]), combined per Pauli matrix
  const int pl_l[6] = {1, 2, 3, 3, 2, 1};
  const double pl_up[6] = {1, 1, 1, -1, 1, -1};
  const double pl_dn[6] = {-1, -1, -1, -1, 1, -1};
  for (int pl = 0; pl < 6; pl++) {
    M3 xi = zero3();
    for (int chi = 0; chi < 2; chi++) {
      const double sg = chi == 0 ? pl_up[pl] : pl_dn[pl];
      const int o = 6 * chi;
      for (int b = 0; b < 3; b++)
        for (int a = 0; a < 3; a++) {
          // O_st = X[t][b] conj(Y[s][a]) within the chirality block
          cd O00 = cmulc(y[o + 0 + a], x[o + 0 + b]);
          cd O01 = cmulc(y[o + 0 + a], x[o + 3 + b]);
          cd O10 = cmulc(y[o + 3 + a], x[o + 0 + b]);
          cd O11 = cmulc(y[o + 3 + a], x[o + 3 + b]);
          cd v;
          if (pl_l[pl] == 1) v = O01 + O10;            // sigma_1 = [[0,1],[1,0]]
          else if (pl_l[pl] == 2) v = ti(O10 - O01);   // sigma_2 = [[0,-i],[i,0]]
          else v = O00 - O11;                          // sigma_3 = diag(1,-1)
          xi.m[b][a] = xi.m[b][a] + sg * v;
        }
    }
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        cd h = xi.m[a][b] + conj(xi.m[b][a]);
        cd kk = (0.25 * csw) * ti(h);
        out[pl * 9 + a * 3 + b] = make_double2(kk.re, kk.im);
      }
  }
}

LQ_DI cd tr_mul(const M3& a, const M3& b) {
  cd t = {0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int k = 0; k < 3; k++) t = t + a.m[i][k] * b.m[k][i];
  return t;
}

// F^a = Re tr[i T_a Z] = -Im tr[T_a Z] = -Im tr[lambda_a Z] / 2
LQ_DI void project_force(const M3& Z, double* out8) {
  const M3& z = Z;
  // tr[lambda_a Z] for the 8 Gell-Mann matrices
  cd t[8];
  t[0] = z.m[1][0] + z.m[0][1];
  t[1] = ti(z.m[1][0]) - ti(z.m[0][1]);  // lambda_2 = [[0,-i],[i,0]]: tr = -i Z10 + i Z01 ... see below
  // lambda_2[0][1] = -i, [1][0] = i  ->  tr(l Z) = l01 Z10 + l10 Z01 = -i Z10 + i Z01
  t[1] = ti(z.m[0][1]) - ti(z.m[1][0]);
  t[2] = z.m[0][0] - z.m[1][1];
  t[3] = z.m[2][0] + z.m[0][2];
  t[4] = ti(z.m[0][2]) - ti(z.m[2][0]);
  t[5] = z.m[2][1] + z.m[1][2];
  t[6] = ti(z.m[1][2]) - ti(z.m[2][1]);
  const double s3 = 0.57735026918962576451;
  t[7] = s3 * (z.m[0][0] + z.m[1][1]) - (2.0 * s3) * z.m[2][2];
#pragma unroll
  for (int a = 0; a < 8; a++) out8[a] = -0.5 * t[a].im;
}

// One thread per link (x, rho): hopping + clover force, natural order.
__global__ void k_force_link(Geom g, const FieldPtrs* fields, int field, int t0, int t1, double csw,
                             const double2* X, const double2* Y, const double2* K, double* F) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 8 * g.Vh) return;
  const long long i = gid >> 2;
  const int rho = (int)(gid & 3);
  double* out = F + gid * 8;
  int x[4];
  ncoords(g, i, x);
  const FieldPtrs f = fields[field];
  if (g.bc_t == 0 && rho == 0 && x[0] == g.L[0] - 1) {
    for (int a = 0; a < 8; a++) out[a] = 0.0;
    return;
  }
  const M3 l = link(g, f, x, rho);
  M3 Z = zero3();
  // ---- hopping part
  {
    int y[4];
    shifted(g, x, rho, 1, y);
    bool ok = x[0] >= t0 && x[0] <= t1 && y[0] >= t0 && y[0] <= t1;
    double fs = 1.0;
    if (rho == 0 && x[0] == g.L[0] - 1) {  // wraps in time: periodic / antiperiodic only
      fs = g.bc_t == 2 ? -1.0 : 1.0;
    }
    if (ok) {
      const long long iy = nidx(g, y);
      cd Xx[12], Xy[12], Yx[12], Yy[12];
      for (int k = 0; k < 12; k++) {
        double2 a = X[i * 12 + k], b = X[iy * 12 + k], c = Y[i * 12 + k], d = Y[iy * 12 + k];
        Xx[k] = {a.x, a.y};
        Xy[k] = {b.x, b.y};
        Yx[k] = {c.x, c.y};
        Yy[k] = {d.x, d.y};
      }
      // (1 - g_rho) X(x+rho) and (1 + g_rho) X(x), full spinors via project/expand
      cd h[6], P1[12], P2[12];
      for (int k = 0; k < 12; k++) P1[k] = P2[k] = {0.0, 0.0};
      switch (rho) {
        case 0: project<0, -1>(Xy, h); expand_add<0, -1>(P1, h); project<0, +1>(Xx, h); expand_add<0, +1>(P2, h); break;
        case 1: project<1, -1>(Xy, h); expand_add<1, -1>(P1, h); project<1, +1>(Xx, h); expand_add<1, +1>(P2, h); break;
        case 2: project<2, -1>(Xy, h); expand_add<2, -1>(P1, h); project<2, +1>(Xx, h); expand_add<2, +1>(P2, h); break;
        default: project<3, -1>(Xy, h); expand_add<3, -1>(P1, h); project<3, +1>(Xx, h); expand_add<3, +1>(P2, h); break;
      }
      M3 W1 = zero3(), W2 = zero3();
      for (int s = 0; s < 4; s++)
        for (int b = 0; b < 3; b++)
          for (int a = 0; a < 3; a++) {
            // W[b][a] = sum_s P[s][b] conj(Y[s][a])
            W1.m[b][a] = W1.m[b][a] + cmulc(Yx[3 * s + a], P1[3 * s + b]);
            W2.m[b][a] = W2.m[b][a] + cmulc(Yy[3 * s + a], P2[3 * s + b]);
          }
      M3 t1m = mul(l, W1), t2m = mul(W2, dagm(l));
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) Z.m[a][b] = fs * (t1m.m[a][b] - t2m.m[a][b]);
    }
  }
  // ---- clover part
  if (csw != 0.0) {
    M3 G = zero3();
    int xr[4];
    shifted(g, x, rho, 1, xr);
    for (int s = 0; s < 4; s++) {
      if (s == rho) continue;
      // plaquette above: corners x, x+rho, x+rho+s, x+s
      int xs[4], xrs[4];
      shifted(g, x, s, 1, xs);
      shifted(g, xr, s, 1, xrs);
      {
        const M3 b = link(g, f, xr, s);
        const M3 c = dagm(link(g, f, xs, rho));
        const M3 d = dagm(link(g, f, x, s));
        const M3 cd_ = mul(c, d);
        const M3 bcd = mul(b, cd_);
        M3 Ma = mul(bcd, load_K(g, K, x, rho, s));
        Ma = add(Ma, mul(load_K(g, K, xr, rho, s), bcd));
        Ma = add(Ma, mul(mul(b, load_K(g, K, xrs, rho, s)), cd_));
        Ma = add(Ma, mul(mul(mul(b, c), load_K(g, K, xs, rho, s)), d));
        G = add(G, mul(l, Ma));
      }
      // plaquette below: w = x - s, corners w, w+rho, x+rho, x
      int w[4], wr[4];
      shifted(g, x, s, -1, w);
      shifted(g, w, rho, 1, wr);
      {
        const M3 ap = link(g, f, w, rho);
        const M3 bp = link(g, f, wr, s);
        const M3 dp = dagm(link(g, f, w, s));
        const M3 apbp = mul(ap, bp);
        const M3 dpap = mul(dp, ap);
        M3 Mc = mul(mul(dp, load_K(g, K, w, rho, s)), apbp);
        Mc = add(Mc, mul(mul(dpap, load_K(g, K, wr, rho, s)), bp));
        Mc = add(Mc, mul(mul(dpap, bp), load_K(g, K, xr, rho, s)));
        Mc = add(Mc, mul(load_K(g, K, x, rho, s), mul(dp, apbp)));
        G = add(G, scl(-1.0, mul(Mc, dagm(l))));
      }
    }
    Z = add(Z, scl(-0.5, G));
  }
  project_force(Z, out);
}

}  // namespace lq

int lq_force(const lqcd_lattice* L, int field, const lqcd_slab& dom, const double2* X, const double2* Y, double* F,
             cudaStream_t st) {
  double2* K = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&K, sizeof(double2) * 54 * (size_t)L->V, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lq_set_error("link_force: allocation failed");
    return LQCD_ENOMEM;
  }
  lq::k_force_K<<<(unsigned)((L->V + 127) / 128), 128, 0, st>>>(L->g, dom.t0, dom.t1, L->csw, X, Y, K);
  lq_count_launch();
  lq::k_force_link<<<(unsigned)((4 * L->V + 127) / 128), 128, 0, st>>>(L->g, L->d_fields, field, dom.t0, dom.t1, L->csw,
                                                                        X, Y, K, F);
  lq_count_launch();
  cudaFreeAsync(K, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("link_force: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  return 0;
}
