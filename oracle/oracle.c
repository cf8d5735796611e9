/*
 * Plain FP64 CPU oracle for the Wilson(-clover) Dirac operator, its
 * domain-restricted (Dirichlet) blocks, Krylov solves and the gauge-link
 * force of phi^dag (D_L^dag D_L)^{-1} phi.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table
 * or helper with the CUDA path.  It is deliberately slow: natural site
 * order, no even-odd split, no link compression, every operator block built
 * as an explicit 12x12 matrix.
 *
 * Conventions (the paper fixes only the normalisation; the rest are the
 * standard Wilson choices, stated here so that every line can be checked):
 *  - site index i = ((x0*L1+x1)*L2+x2)*L3+x3, x0 is time (Sec. 5, x0 slices);
 *  - gauge field U[i][mu][a][b], spinor psi[i][s][c] (complex128);
 *  - D = 1/(2 kappa) - (1/2) D_hop + clover, i.e. 2 kappa D = 1 - kappa D_hop
 *    (Sec. 5, definition under eq. stochastic_estimator);
 *  - (D_hop psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
 *                          + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu);
 *  - chiral gamma basis, g5 = g0 g1 g2 g3 = diag(1,1,-1,-1);
 *  - time boundary: open (Sec. 5: no hop between x0=T-1 and x0=0, and every
 *    clover leaf through that missing link vanishes), periodic or
 *    antiperiodic (library option for the free-field test); space periodic;
 *  - clover: c_sw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu(x),
 *    sigma_mu_nu = (i/2)[g_mu, g_nu], Fhat = (Q_mu_nu - Q_mu_nu^dag)/8 with
 *    Q the sum of the four plaquette leaves at x;
 *  - a domain operator D_L on the time slab t0..t1 is the exact sub-block of
 *    D on the sites of L: every hop whose other end lies outside L is
 *    dropped (Dirichlet), and the clover term keeps the full-lattice links
 *    (Sec. 3, eq. block_inverse; Sec. 5, Dirichlet block operators).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { BC_OPEN = 0, BC_PERIODIC = 1, BC_ANTIPERIODIC = 2 };

typedef struct {
  int d[4];
  int bc;
  long V;
} geo;

static geo make_geo(const int dims[4], int bc) {
  geo g;
  for (int k = 0; k < 4; k++) g.d[k] = dims[k];
  g.bc = bc;
  g.V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  return g;
}

static void coords(const geo *g, long i, int x[4]) {
  for (int k = 3; k >= 0; k--) {
    x[k] = (int)(i % g->d[k]);
    i /= g->d[k];
  }
}

static long index_of(const geo *g, const int x[4]) {
  return ((long)(x[0] * g->d[1] + x[1]) * g->d[2] + x[2]) * g->d[3] + x[3];
}

/* Neighbour of x one step (+1 or -1) along mu.  *crossed_t is set when the
 * step wraps around the time boundary. */
static long neighbour(const geo *g, const int x[4], int mu, int step, int *crossed_t) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] += step;
  *crossed_t = 0;
  if (y[mu] < 0) {
    y[mu] += g->d[mu];
    if (mu == 0) *crossed_t = 1;
  } else if (y[mu] >= g->d[mu]) {
    y[mu] -= g->d[mu];
    if (mu == 0) *crossed_t = 1;
  }
  return index_of(g, y);
}

/* ---------------------------------------------------------------- gammas */

static cplx GAM[5][4][4];
static int gam_ready = 0;

static void init_gamma(void) {
  if (gam_ready) return;
  memset(GAM, 0, sizeof GAM);
  for (int i = 0; i < 2; i++) {
    GAM[0][i][i + 2] = -1;
    GAM[0][i + 2][i] = -1;
  }
  const cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  for (int k = 0; k < 3; k++)
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        GAM[k + 1][i][j + 2] = -I * sig[k][i][j];
        GAM[k + 1][i + 2][j] = I * sig[k][i][j];
      }
  cplx t1[4][4], t2[4][4];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      t1[i][j] = 0;
      for (int k = 0; k < 4; k++) t1[i][j] += GAM[0][i][k] * GAM[1][k][j];
    }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      t2[i][j] = 0;
      for (int k = 0; k < 4; k++) t2[i][j] += t1[i][k] * GAM[2][k][j];
    }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      GAM[4][i][j] = 0;
      for (int k = 0; k < 4; k++) GAM[4][i][j] += t2[i][k] * GAM[3][k][j];
    }
  gam_ready = 1;
}

void ora_gamma(int mu, double *out16c) {
  init_gamma();
  cplx *o = (cplx *)out16c;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) o[4 * i + j] = GAM[mu][i][j];
}

/* sigma_mu_nu = (i/2)[g_mu, g_nu] */
static void sigma(int mu, int nu, cplx s[4][4]) {
  init_gamma();
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      cplx c = 0;
      for (int k = 0; k < 4; k++) c += GAM[mu][i][k] * GAM[nu][k][j] - GAM[nu][i][k] * GAM[mu][k][j];
      s[i][j] = 0.5 * I * c;
    }
}

/* -------------------------------------------------------- colour algebra */

typedef struct {
  cplx m[3][3];
} su3;

static su3 link_of(const cplx *U, long i, int mu) {
  su3 r;
  memcpy(r.m, U + ((i * 4 + mu) * 9), sizeof r.m);
  return r;
}

static su3 mul(su3 a, su3 b) {
  su3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cplx c = 0;
      for (int k = 0; k < 3; k++) c += a.m[i][k] * b.m[k][j];
      r.m[i][j] = c;
    }
  return r;
}

static su3 dag(su3 a) {
  su3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i][j] = conj(a.m[j][i]);
  return r;
}

static su3 zero3(void) {
  su3 r;
  memset(r.m, 0, sizeof r.m);
  return r;
}

static su3 ident3(void) {
  su3 r = zero3();
  for (int i = 0; i < 3; i++) r.m[i][i] = 1;
  return r;
}

/* Link U_mu(x) as seen by the gauge part of D: the temporal link leaving the
 * last time slice is absent (zero) under open boundary conditions. */
static su3 gauge_link(const geo *g, const cplx *U, long i, int mu) {
  if (g->bc == BC_OPEN && mu == 0) {
    int x[4];
    coords(g, i, x);
    if (x[0] == g->d[0] - 1) return zero3();
  }
  return link_of(U, i, mu);
}

/* ------------------------------------------------------------- clover */

/* Shifted site: x + a*mu + b*nu (a, b in {-1,0,1}). */
static long shift2(const geo *g, long i, int mu, int a, int nu, int b) {
  int x[4], c;
  coords(g, i, x);
  long j = i;
  if (a) {
    j = neighbour(g, x, mu, a, &c);
    coords(g, j, x);
  }
  if (b) j = neighbour(g, x, nu, b, &c);
  return j;
}

/* One factor of a plaquette leaf: link U_dir(site), daggered or not. */
typedef struct {
  long site;
  int dir;
  int dagger;
} factor;

/* The four leaves of the clover at z in the (mu, nu) plane, each as four
 * ordered link factors (all leaves start and end at z, oriented mu -> nu). */
static void leaves(const geo *g, long z, int mu, int nu, factor f[4][4]) {
  long zpm = shift2(g, z, mu, 1, nu, 0), zpn = shift2(g, z, mu, 0, nu, 1);
  long zmm = shift2(g, z, mu, -1, nu, 0), zmn = shift2(g, z, mu, 0, nu, -1);
  long zmm_pn = shift2(g, z, mu, -1, nu, 1), zmm_mn = shift2(g, z, mu, -1, nu, -1);
  long zpm_mn = shift2(g, z, mu, 1, nu, -1);
  (void)zpm_mn;
  /* leaf 1: U_mu(z) U_nu(z+mu) U_mu(z+nu)^dag U_nu(z)^dag */
  f[0][0] = (factor){z, mu, 0};
  f[0][1] = (factor){zpm, nu, 0};
  f[0][2] = (factor){zpn, mu, 1};
  f[0][3] = (factor){z, nu, 1};
  /* leaf 2: U_nu(z) U_mu(z+nu-mu)^dag U_nu(z-mu)^dag U_mu(z-mu) */
  f[1][0] = (factor){z, nu, 0};
  f[1][1] = (factor){zmm_pn, mu, 1};
  f[1][2] = (factor){zmm, nu, 1};
  f[1][3] = (factor){zmm, mu, 0};
  /* leaf 3: U_mu(z-mu)^dag U_nu(z-mu-nu)^dag U_mu(z-mu-nu) U_nu(z-nu) */
  f[2][0] = (factor){zmm, mu, 1};
  f[2][1] = (factor){zmm_mn, nu, 1};
  f[2][2] = (factor){zmm_mn, mu, 0};
  f[2][3] = (factor){zmn, nu, 0};
  /* leaf 4: U_nu(z-nu)^dag U_mu(z-nu) U_nu(z-nu+mu) U_mu(z)^dag */
  f[3][0] = (factor){zmn, nu, 1};
  f[3][1] = (factor){zmn, mu, 0};
  f[3][2] = (factor){shift2(g, z, mu, 1, nu, -1), nu, 0};
  f[3][3] = (factor){z, mu, 1};
}

static su3 factor_value(const geo *g, const cplx *U, factor f) {
  su3 u = gauge_link(g, U, f.site, f.dir);
  return f.dagger ? dag(u) : u;
}

/* Fhat_mu_nu(z) = (Q - Q^dag)/8, Q = sum of the four leaves. */
static su3 fhat(const geo *g, const cplx *U, long z, int mu, int nu) {
  factor f[4][4];
  leaves(g, z, mu, nu, f);
  su3 Q = zero3();
  for (int l = 0; l < 4; l++) {
    su3 p = ident3();
    for (int k = 0; k < 4; k++) p = mul(p, factor_value(g, U, f[l][k]));
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) Q.m[a][b] += p.m[a][b];
  }
  su3 F;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) F.m[a][b] = (Q.m[a][b] - conj(Q.m[b][a])) / 8.0;
  return F;
}

/* A[V][12][12]: the site-diagonal part of D,
 *   A(x) = 1/(2 kappa) + c_sw (i/4) sum_{mu != nu} sigma_mu_nu Fhat_mu_nu(x),
 * with row/column index 3*s + c. */
/* The 12x12 site-diagonal block of D at site z. */
static void clover_site(const geo *g, const cplx *U, long z, double kappa, double csw, cplx *M) {
  static cplx sg[4][4][4][4];
  static int sg_ready = 0;
  if (!sg_ready) {
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) sigma(mu, nu, sg[mu][nu]);
    sg_ready = 1;
  }
  memset(M, 0, 144 * sizeof(cplx));
  for (int r = 0; r < 12; r++) M[r * 12 + r] = 1.0 / (2.0 * kappa);
  if (csw == 0.0) return;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = 0; nu < 4; nu++) {
      if (mu == nu) continue;
      su3 F = fhat(g, U, z, mu, nu);
      for (int s = 0; s < 4; s++)
        for (int t = 0; t < 4; t++)
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) M[(3 * s + a) * 12 + 3 * t + b] += csw * 0.25 * I * sg[mu][nu][s][t] * F.m[a][b];
    }
}

void ora_clover(const int dims[4], int bc, const double *Ud, double kappa, double csw, double *Ad) {
  geo g = make_geo(dims, bc);
  const cplx *U = (const cplx *)Ud;
  cplx *A = (cplx *)Ad;
  for (long z = 0; z < g.V; z++) clover_site(&g, U, z, kappa, csw, A + z * 144);
}

/* ------------------------------------------------------- Dirac operator */

/* Explicit 12x12 block of D coupling row site x to column site y = x +/- mu:
 *   forward  (y = x+mu): -(1/2) f (1 - g_mu) (x) U_mu(x)
 *   backward (y = x-mu): -(1/2) f (1 + g_mu) (x) U_mu(x-mu)^dag
 * f is the boundary factor (0 dropped, -1 antiperiodic wrap, 1 otherwise). */
static void hop_block(const su3 *W, int mu, int fwd, double f, cplx B[12][12]) {
  init_gamma();
  for (int s = 0; s < 4; s++)
    for (int t = 0; t < 4; t++) {
      cplx P = (s == t ? 1.0 : 0.0) + (fwd ? -1.0 : 1.0) * GAM[mu][s][t];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) B[3 * s + a][3 * t + b] = -0.5 * f * P * W->m[a][b];
    }
}

/* Boundary factor of the hop from x (time x0) to its neighbour along mu,
 * for the domain operator on t0..t1. */
static double hop_factor(const geo *g, int mu, int crossed, int y0, int t0, int t1) {
  if (y0 < t0 || y0 > t1) return 0.0;
  if (mu == 0 && crossed) {
    if (g->bc == BC_OPEN) return 0.0;
    if (g->bc == BC_ANTIPERIODIC) return -1.0;
  }
  return 1.0;
}

static int in_slab(const geo *g, long i, int t0, int t1) {
  long s3 = (long)g->d[1] * g->d[2] * g->d[3];
  int t = (int)(i / s3);
  return t >= t0 && t <= t1;
}

static void blk_apply(cplx B[12][12], const cplx *v, cplx *o, int adjoint) {
  for (int r = 0; r < 12; r++) {
    cplx c = 0;
    for (int k = 0; k < 12; k++) c += (adjoint ? conj(B[k][r]) : B[r][k]) * v[k];
    o[r] += c;
  }
}

/* out = D_L in (dagger = 0) or D_L^dag in (dagger = 1) on the slab t0..t1.
 * The adjoint is formed term by term: every block D(x,y) is applied as
 * D(x,y)^dag from x to y.  out is zero outside the slab. */
void ora_dirac(const int dims[4], int bc, const double *Ud, const double *Ad, int t0, int t1,
               int dagger, const double *ind, double *outd) {
  geo g = make_geo(dims, bc);
  const cplx *U = (const cplx *)Ud, *A = (const cplx *)Ad, *in = (const cplx *)ind;
  cplx *out = (cplx *)outd;
  memset(out, 0, g.V * 12 * sizeof(cplx));
  cplx B[12][12];
  for (long x = 0; x < g.V; x++) {
    if (!in_slab(&g, x, t0, t1)) continue;
    int xc[4];
    coords(&g, x, xc);
    /* site-diagonal block */
    for (int r = 0; r < 12; r++)
      for (int k = 0; k < 12; k++) B[r][k] = A[x * 144 + r * 12 + k];
    blk_apply(B, in + x * 12, out + x * 12, dagger);
    for (int mu = 0; mu < 4; mu++)
      for (int fwd = 1; fwd >= 0; fwd--) {
        int crossed;
        long y = neighbour(&g, xc, mu, fwd ? 1 : -1, &crossed);
        int yc[4];
        coords(&g, y, yc);
        double f = hop_factor(&g, mu, crossed, yc[0], t0, t1);
        if (f == 0.0) continue;
        su3 W = fwd ? link_of(U, x, mu) : dag(link_of(U, y, mu));
        hop_block(&W, mu, fwd, f, B);
        if (!dagger)
          blk_apply(B, in + y * 12, out + x * 12, 0);
        else
          blk_apply(B, in + x * 12, out + y * 12, 1);
      }
  }
}

/* ---------------------------------------------------------------- solver */

static cplx dotc(long n, const cplx *a, const cplx *b) {
  cplx s = 0;
  for (long i = 0; i < n; i++) s += conj(a[i]) * b[i];
  return s;
}

static double nrm2(long n, const cplx *a) { return creal(dotc(n, a, a)); }

typedef struct {
  const int *dims;
  int bc;
  const double *U, *A;
  int t0, t1, dagger;
} opctx;

static void op(const opctx *c, const cplx *in, cplx *out) {
  ora_dirac(c->dims, c->bc, c->U, c->A, c->t0, c->t1, c->dagger, (const double *)in, (double *)out);
}

static void op_adj(const opctx *c, const cplx *in, cplx *out) {
  ora_dirac(c->dims, c->bc, c->U, c->A, c->t0, c->t1, !c->dagger, (const double *)in, (double *)out);
}

/* BiCGStab (van der Vorst 1992) on M x = b, restarted from the true residual;
 * returns 0 on success. */
static int bicgstab(const opctx *c, long n, const cplx *b, cplx *x, double tol, int maxit, int *its) {
  cplx *r = malloc(n * sizeof(cplx)), *r0 = malloc(n * sizeof(cplx)), *p = malloc(n * sizeof(cplx));
  cplx *v = malloc(n * sizeof(cplx)), *s = malloc(n * sizeof(cplx)), *t = malloc(n * sizeof(cplx));
  double bn = sqrt(nrm2(n, b));
  int k = 0, ok = 0;
  while (k < maxit) {
    op(c, x, t);
    for (long i = 0; i < n; i++) r[i] = b[i] - t[i];
    double rn = sqrt(nrm2(n, r));
    if (rn <= tol * bn) {
      ok = 1;
      break;
    }
    memcpy(r0, r, n * sizeof(cplx));
    memcpy(p, r, n * sizeof(cplx));
    cplx rho = dotc(n, r0, r);
    int inner = 0;
    while (k < maxit && inner < 2000) {
      op(c, p, v);
      cplx r0v = dotc(n, r0, v);
      if (cabs(r0v) == 0.0) break;
      cplx alpha = rho / r0v;
      for (long i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
      op(c, s, t);
      double tt = nrm2(n, t);
      if (tt == 0.0) {
        for (long i = 0; i < n; i++) x[i] += alpha * p[i];
        k++;
        break;
      }
      cplx omega = dotc(n, t, s) / tt;
      for (long i = 0; i < n; i++) {
        x[i] += alpha * p[i] + omega * s[i];
        r[i] = s[i] - omega * t[i];
      }
      k++;
      inner++;
      double rr = sqrt(nrm2(n, r));
      if (rr <= 0.1 * tol * bn) break;
      cplx rho1 = dotc(n, r0, r);
      if (cabs(rho1) < 1e-30 * bn * bn || cabs(omega) == 0.0) break;
      cplx beta = (rho1 / rho) * (alpha / omega);
      for (long i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      rho = rho1;
    }
  }
  *its = k;
  free(r); free(r0); free(p); free(v); free(s); free(t);
  return ok ? 0 : -1;
}

/* CG on M^dag M x = M^dag b (CGNR), the fallback when BiCGStab stalls. */
static int cgnr(const opctx *c, long n, const cplx *b, cplx *x, double tol, int maxit, int *its) {
  cplx *r = malloc(n * sizeof(cplx)), *z = malloc(n * sizeof(cplx)), *p = malloc(n * sizeof(cplx));
  cplx *q = malloc(n * sizeof(cplx)), *w = malloc(n * sizeof(cplx));
  double bn = sqrt(nrm2(n, b));
  int k = 0, ok = 0;
  op(c, x, w);
  for (long i = 0; i < n; i++) r[i] = b[i] - w[i];
  op_adj(c, r, z);
  memcpy(p, z, n * sizeof(cplx));
  double zz = nrm2(n, z);
  while (k < maxit) {
    if (k % 100 == 0) {
      op(c, x, w);
      for (long i = 0; i < n; i++) r[i] = b[i] - w[i];
      if (sqrt(nrm2(n, r)) <= tol * bn) {
        ok = 1;
        break;
      }
    }
    op(c, p, q);
    double qq = nrm2(n, q);
    if (qq == 0.0) break;
    double alpha = zz / qq;
    for (long i = 0; i < n; i++) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    op_adj(c, r, z);
    double zz1 = nrm2(n, z);
    double beta = zz1 / zz;
    for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    zz = zz1;
    k++;
    if (sqrt(nrm2(n, r)) <= 0.5 * tol * bn) {
      op(c, x, w);
      for (long i = 0; i < n; i++) r[i] = b[i] - w[i];
      if (sqrt(nrm2(n, r)) <= tol * bn) {
        ok = 1;
        break;
      }
    }
  }
  *its = k;
  free(r); free(z); free(p); free(q); free(w);
  return ok ? 0 : -1;
}

/* Solve D_L x = b (dagger = 0) or D_L^dag x = b (dagger = 1) on t0..t1 to
 * relative true residual tol.  b is masked to the slab first; x starts at 0.
 * Returns 0 on success, -1 if neither BiCGStab nor CGNR converged. */
int ora_solve(const int dims[4], int bc, const double *Ud, const double *Ad, int t0, int t1, int dagger,
              const double *bd, double *xd, double tol, int maxit, int *iters, double *relres) {
  geo g = make_geo(dims, bc);
  long n = g.V * 12;
  opctx c = {dims, bc, Ud, Ad, t0, t1, dagger};
  cplx *b = malloc(n * sizeof(cplx));
  cplx *x = (cplx *)xd;
  memcpy(b, bd, n * sizeof(cplx));
  for (long i = 0; i < g.V; i++)
    if (!in_slab(&g, i, t0, t1))
      for (int k = 0; k < 12; k++) b[i * 12 + k] = 0;
  memset(x, 0, n * sizeof(cplx));
  int its1 = 0, its2 = 0;
  int rc = bicgstab(&c, n, b, x, tol, maxit, &its1);
  if (rc != 0) rc = cgnr(&c, n, b, x, tol, maxit, &its2);
  cplx *w = malloc(n * sizeof(cplx));
  op(&c, x, w);
  for (long i = 0; i < n; i++) w[i] = b[i] - w[i];
  double bn = sqrt(nrm2(n, b));
  *relres = bn > 0 ? sqrt(nrm2(n, w)) / bn : 0.0;
  *iters = its1 + its2;
  free(w);
  free(b);
  return rc;
}

/* ----------------------------------------------------------------- force */

/* i T_a = i lambda_a / 2 */
static void gen(int a, su3 *out) {
  static const double s3 = 0.57735026918962576451;
  su3 l = zero3();
  switch (a) {
    case 0: l.m[0][1] = l.m[1][0] = 1; break;
    case 1: l.m[0][1] = -I; l.m[1][0] = I; break;
    case 2: l.m[0][0] = 1; l.m[1][1] = -1; break;
    case 3: l.m[0][2] = l.m[2][0] = 1; break;
    case 4: l.m[0][2] = -I; l.m[2][0] = I; break;
    case 5: l.m[1][2] = l.m[2][1] = 1; break;
    case 6: l.m[1][2] = -I; l.m[2][1] = I; break;
    case 7: l.m[0][0] = l.m[1][1] = s3; l.m[2][2] = -2 * s3; break;
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) out->m[i][j] = 0.5 * I * l.m[i][j];
}

/* d/d omega of the link U_dir(site) (or its adjoint) under
 * U -> exp(i omega T_a) U at omega = 0. */
static su3 dlink(const geo *g, const cplx *U, factor f, const su3 *iT) {
  su3 u = gauge_link(g, U, f.site, f.dir);
  if (!f.dagger) return mul(*iT, u);
  su3 r = mul(dag(u), *iT);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i][j] = -r.m[i][j];
  return r;
}

static void force_add(double *F, long site, int dir, int a, double val) { F[(site * 4 + dir) * 8 + a] += val; }

/* F[V][4][8]: F^a_mu(x) = dS/d omega for U_mu(x) -> exp(i omega T_a) U_mu(x),
 * S = phi^dag (D_L^dag D_L)^{-1} phi, given X = (D_L^dag D_L)^{-1} phi and
 * Y = D_L X:  F = -2 Re <Y, (dD_L/d omega) X>.  Hopping and clover terms
 * are both differentiated by the product rule, link by link. */
void ora_force(const int dims[4], int bc, const double *Ud, double csw, int t0, int t1, const double *Xd,
               const double *Yd, double *F) {
  geo g = make_geo(dims, bc);
  const cplx *U = (const cplx *)Ud, *X = (const cplx *)Xd, *Y = (const cplx *)Yd;
  memset(F, 0, g.V * 32 * sizeof(double));
  su3 iT[8];
  for (int a = 0; a < 8; a++) gen(a, &iT[a]);
  cplx B[12][12];
  /* hopping part: the link U_mu(x) appears in D(x, x+mu) and D(x+mu, x) */
  for (long x = 0; x < g.V; x++) {
    if (!in_slab(&g, x, t0, t1)) continue;
    int xc[4];
    coords(&g, x, xc);
    for (int mu = 0; mu < 4; mu++) {
      int crossed;
      long y = neighbour(&g, xc, mu, 1, &crossed);
      int yc[4];
      coords(&g, y, yc);
      double f = hop_factor(&g, mu, crossed, yc[0], t0, t1);
      if (f == 0.0) continue;
      su3 u = link_of(U, x, mu);
      for (int a = 0; a < 8; a++) {
        su3 du = mul(iT[a], u);              /* d U      */
        su3 dud = dag(du);                    /* d U^dag  */
        cplx acc = 0;
        cplx o[12];
        hop_block(&du, mu, 1, f, B);          /* row x, column y */
        memset(o, 0, sizeof o);
        blk_apply(B, X + y * 12, o, 0);
        for (int k = 0; k < 12; k++) acc += conj(Y[x * 12 + k]) * o[k];
        hop_block(&dud, mu, 0, f, B);         /* row y, column x */
        memset(o, 0, sizeof o);
        blk_apply(B, X + x * 12, o, 0);
        for (int k = 0; k < 12; k++) acc += conj(Y[y * 12 + k]) * o[k];
        force_add(F, x, mu, a, -2.0 * creal(acc));
      }
    }
  }
  if (csw == 0.0) return;
  /* clover part: <Y(z), dA(z) X(z)> for every z in the slab */
  cplx sg[4][4][4][4];
  for (int mu = 0; mu < 4; mu++)
    for (int nu = 0; nu < 4; nu++) sigma(mu, nu, sg[mu][nu]);
  for (long z = 0; z < g.V; z++) {
    if (!in_slab(&g, z, t0, t1)) continue;
    const cplx *xz = X + z * 12, *yz = Y + z * 12;
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (mu == nu) continue;
        /* Xi[b][a] = sum_{s,t} X[t][b] sigma[s][t] conj(Y[s][a]):
         * Y^dag (sigma x G) X = tr(G Xi) */
        su3 Xi = zero3();
        for (int s = 0; s < 4; s++)
          for (int t = 0; t < 4; t++)
            for (int a = 0; a < 3; a++)
              for (int b = 0; b < 3; b++) Xi.m[b][a] += xz[3 * t + b] * sg[mu][nu][s][t] * conj(yz[3 * s + a]);
        factor f[4][4];
        leaves(&g, z, mu, nu, f);
        for (int l = 0; l < 4; l++)
          for (int k = 0; k < 4; k++) {
            factor fk = f[l][k];
            if (g.bc == BC_OPEN && fk.dir == 0) {
              int wc[4];
              coords(&g, fk.site, wc);
              if (wc[0] == g.d[0] - 1) continue; /* absent link: no force */
            }
            for (int a = 0; a < 8; a++) {
              su3 p = ident3();
              for (int m = 0; m < 4; m++) p = mul(p, m == k ? dlink(&g, U, f[l][m], &iT[a]) : factor_value(&g, U, f[l][m]));
              /* dFhat = (dQ - dQ^dag)/8 ; clover term c_sw (i/4) sigma dFhat */
              cplx tr = 0;
              for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) tr += (p.m[i][j] - conj(p.m[j][i])) / 8.0 * Xi.m[j][i];
              force_add(F, fk.site, fk.dir, a, -2.0 * creal(csw * 0.25 * I * tr));
            }
          }
      }
  }
}

/* (D_L in)(x) at the listed sites x only (natural indices, inside the slab
 * t0..t1): out[k][12] for sites[k].  Same terms as ora_dirac (dagger = 0),
 * with the site-diagonal block built from the links at each listed site, so
 * no full-lattice clover array is needed on very large lattices. */
void ora_dirac_sites(const int dims[4], int bc, const double *Ud, double kappa, double csw, int t0, int t1,
                     const long *sites, int nsites, const double *ind, double *outd) {
  geo g = make_geo(dims, bc);
  const cplx *U = (const cplx *)Ud, *in = (const cplx *)ind;
  cplx *out = (cplx *)outd;
  cplx B[12][12], M[144];
  for (int k = 0; k < nsites; k++) {
    const long x = sites[k];
    cplx *o = out + (long)k * 12;
    memset(o, 0, 12 * sizeof(cplx));
    if (!in_slab(&g, x, t0, t1)) continue;
    int xc[4];
    coords(&g, x, xc);
    clover_site(&g, U, x, kappa, csw, M);
    for (int r = 0; r < 12; r++)
      for (int c = 0; c < 12; c++) B[r][c] = M[r * 12 + c];
    blk_apply(B, in + x * 12, o, 0);
    for (int mu = 0; mu < 4; mu++)
      for (int fwd = 1; fwd >= 0; fwd--) {
        int crossed;
        long y = neighbour(&g, xc, mu, fwd ? 1 : -1, &crossed);
        int yc[4];
        coords(&g, y, yc);
        double f = hop_factor(&g, mu, crossed, yc[0], t0, t1);
        if (f == 0.0) continue;
        su3 W = fwd ? link_of(U, x, mu) : dag(link_of(U, y, mu));
        hop_block(&W, mu, fwd, f, B);
        blk_apply(B, in + y * 12, o, 0);
      }
  }
}
