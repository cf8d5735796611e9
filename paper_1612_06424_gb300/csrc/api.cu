// C-ABI entry points (include/lqcd.h) and the host side of the batched
// solver: the FP64 defect-correction loop around even-odd preconditioned
// BiCGStab in FP64, FP32 or FP16, the factorized-propagator pipeline of
// Sec. 3 and the link-force driver.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <string>
#include <functional>
#include <vector>

#include "internal.h"

static thread_local std::string g_err;
static bool verbose() {
  static int v = -1;
  if (v < 0) v = getenv("LQCD_VERBOSE") ? 1 : 0;
  return v == 1;
}
void lq_set_error(const std::string& m) { g_err = m; }
extern "C" const char* lqcd_last_error(void) { return g_err.c_str(); }

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      lq_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));              \
      return e_ == cudaErrorMemoryAllocation ? LQCD_ENOMEM : LQCD_ECUDA;             \
    }                                                                                \
  } while (0)

#define RC(call)               \
  do {                         \
    int r_ = (call);           \
    if (r_ != 0) return r_;    \
  } while (0)

namespace {

// Stream-ordered device buffer (freed on scope exit).
struct DBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  int alloc(size_t bytes, cudaStream_t s) {
    st = s;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
      // The pool keeps the blocks of earlier waves mapped; when they are too
      // small for this request they only block it.  Wait for every pending
      // free, hand the pool's unused memory back to the CUDA driver and retry.
      cudaGetLastError();
      int dev = 0;
      cudaMemPool_t pool;
      if (cudaDeviceSynchronize() == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
        e = cudaMallocAsync(&p, bytes, s);
    }
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      lq_set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
      return LQCD_ENOMEM;
    }
    return 0;
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

struct PinnedInt {
  int* h = nullptr;
  PinnedInt() { cudaHostAlloc((void**)&h, sizeof(int) * 4, cudaHostAllocDefault); }
  ~PinnedInt() {
    if (h) cudaFreeHost(h);
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int check_lat(const lqcd_lattice* L) {
  if (!L) {
    lq_set_error("null lattice");
    return LQCD_EBADARG;
  }
  return 0;
}

// A batch with its own descriptor / flag / scalar / partial storage.
struct BatchStore {
  Batch b;
  DBuf sys, active, sc, partial;
  std::vector<lq::SysDesc> h_sys;
  std::vector<lq::SolverScal> h_sc;
  std::vector<int> h_active;

  int build(const lqcd_lattice* L, int n, const lqcd_slab* doms, const int* fields, cudaStream_t st) {
    h_sys.resize(n);
    long long off = 0, maxn = 0;  // maxn: sites per parity of the largest system
    for (int k = 0; k < n; k++) {
      const lqcd_slab d = doms[k];
      if (d.t0 < 0 || d.t1 >= L->dims[0] || d.t0 > d.t1) {
        lq_set_error("slab out of range: " + std::to_string(d.t0) + ".." + std::to_string(d.t1));
        return LQCD_EBADARG;
      }
      if (fields[k] < 0 || fields[k] >= (int)L->fields.size()) {
        lq_set_error("field index " + std::to_string(fields[k]) + " not loaded");
        return LQCD_ENOFIELD;
      }
      lq::SysDesc s{};
      s.field = fields[k];
      s.t0 = d.t0;
      s.t1 = d.t1;
      s.wrap = (d.t0 == 0 && d.t1 == L->dims[0] - 1 && L->bc != LQCD_BC_OPEN) ? 1 : 0;
      s.tsign = L->bc == LQCD_BC_ANTIPERIODIC ? -1.f : 1.f;
      s.n = (int)((d.t1 - d.t0 + 1) * L->S3h);
      s.cb0 = (int)(d.t0 * L->S3h);
      s.off = off;
      off += s.n;
      maxn = std::max(maxn, (long long)s.n);
      h_sys[k] = s;
    }
    b.nsys = n;
    b.max_n = maxn;
    b.total = off;
    b.tblk_ok = L->S3h % 32 == 0 ? 1 : 0;
    for (int k = 0; k < n; k++)
      if ((doms[k].t1 - doms[k].t0 + 1) % 4 != 0) b.tblk_ok = 0;
    b.nby = (int)((maxn + LQ_BLOCK - 1) / LQ_BLOCK);
    b.pstride = (int)((12 * maxn + LQ_BLOCK - 1) / LQ_BLOCK);
    if ((long long)n * b.pstride >= (1LL << 31)) {
      lq_set_error("batch too large for one grid (systems x blocks per system >= 2^31)");
      return LQCD_EBADARG;
    }
    RC(sys.alloc(sizeof(lq::SysDesc) * n, st));
    RC(active.alloc(sizeof(int) * n, st));
    RC(sc.alloc(sizeof(lq::SolverScal) * n, st));
    RC(partial.alloc(sizeof(double) * 4 * (size_t)n * b.pstride, st));
    CK(cudaMemcpyAsync(sys.p, h_sys.data(), sizeof(lq::SysDesc) * n, cudaMemcpyHostToDevice, st));
    b.sys = sys.as<lq::SysDesc>();
    b.active = active.as<int>();
    b.sc = sc.as<lq::SolverScal>();
    b.partial = partial.as<double>();
    h_sc.assign(n, lq::SolverScal{});
    h_active.assign(n, 1);
    CK(cudaMemcpyAsync(sc.p, h_sc.data(), sizeof(lq::SolverScal) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(active.p, h_active.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    return 0;
  }
  int push_active(cudaStream_t st) {
    CK(cudaMemcpyAsync(active.p, h_active.data(), sizeof(int) * b.nsys, cudaMemcpyHostToDevice, st));
    return 0;
  }
  int pull_sc(cudaStream_t st) {
    CK(cudaMemcpyAsync(h_sc.data(), sc.p, sizeof(lq::SolverScal) * b.nsys, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return 0;
  }
  int push_sc(cudaStream_t st) {
    CK(cudaMemcpyAsync(sc.p, h_sc.data(), sizeof(lq::SolverScal) * b.nsys, cudaMemcpyHostToDevice, st));
    return 0;
  }
};

// FP64 pool of `count` vectors of a batch (each total*12 double2).
struct Pool64 {
  DBuf buf;
  long long words = 0;
  int alloc(const Batch& b, int count, cudaStream_t st) {
    words = b.total * 12;
    return buf.alloc(sizeof(double2) * (size_t)words * count, st);
  }
  double2* v(int k) const { return buf.as<double2>() + (size_t)k * words; }
};

// Pool of `count` vectors in precision P (norm pool for FP16).
struct PoolP {
  DBuf buf, nrm;
  long long bytes = 0;
  long long total = 0;
  int P = 64;
  int alloc(const Batch& b, int prec, int count, cudaStream_t st) {
    P = prec;
    total = b.total;
    bytes = b.total * (P == 64 ? 192 : P == 32 ? 96 : 48);
    RC(buf.alloc((size_t)bytes * count, st));
    if (P == 16) RC(nrm.alloc(sizeof(float) * (size_t)total * count, st));
    return 0;
  }
  VecP v(int k) const {
    VecP r;
    r.d = (char*)buf.p + (size_t)bytes * k;
    r.nrm = P == 16 ? nrm.as<float>() + (size_t)total * k : nullptr;
    return r;
  }
};

VecP v64(double2* p) {
  VecP r;
  r.d = p;
  return r;
}

struct SolveOut {
  std::vector<int> iters, cycles, status;
  std::vector<double> res;
};

// Solve D_L x = b (dag: D_L^dag x = b) for every system of the batch.
// b_e, b_o, x_e, x_o: FP64 even / odd pools of the batch.  With guess, x_o
// holds a starting iterate of the odd half on entry (the even half is always
// reconstructed from it at the end); else the solve starts from x = 0.
int solve_core(lqcd_lattice* L, BatchStore& B, bool dag, const lqcd_solver_params& prm, double2* b_e, double2* b_o,
               double2* x_e, double2* x_o, SolveOut& out, cudaStream_t st, bool guess = false) {
  Batch& b = B.b;
  const int n = b.nsys;
  const int P = prm.precision == 16 ? 16 : prm.precision == 32 ? 32 : 64;
  const bool clov = L->csw != 0.0;
  const double tol = prm.tol > 0 ? prm.tol : 1e-10;
  const int max_iter = prm.max_iter > 0 ? prm.max_iter : 100000;
  const int check_every = prm.check_every > 0 ? prm.check_every : 8;
  // the inner iterations run as a captured CUDA graph unless LQCD_NO_GRAPH is set
  static const bool use_graph = getenv("LQCD_NO_GRAPH") == nullptr;
  double inner_tol = prm.inner_tol;
  // FP32: 3e-6 measured 1.7% faster than 1e-5 on the 48^3 x 96 factorized propagator (fewer
  // iterations over the two cycles); FP16 cannot go deeper than a few 1e-2
  if (!(inner_tol > 0)) inner_tol = P == 64 ? 0.0 : P == 32 ? 3e-6 : 2e-2;
  // iterations of one inner cycle: a reduced-precision BiCGStab that has not
  // reached inner_tol by then is restarted from the true FP64 residual
  const int cycle_cap = P == 64 ? max_iter : P == 32 ? 2000 : 500;
  if (P == 64) inner_tol = 0.0;
  out.iters.assign(n, 0);
  out.cycles.assign(n, 0);
  out.status.assign(n, 0);
  out.res.assign(n, 0.0);

  Pool64 f64;
  RC(f64.alloc(b, 3, st));
  double2* bh_o = f64.v(0);
  double2* r64 = f64.v(1);
  double2* t64 = f64.v(2);
  PoolP ps;
  RC(ps.alloc(b, P, 8, st));
  VecP r = ps.v(0), r0 = ps.v(1), p = ps.v(2), v = ps.v(3), s = ps.v(4), t = ps.v(5), xs = ps.v(6), te = ps.v(7);
  PinnedInt cnt;
  DBuf dcnt;
  RC(dcnt.alloc(sizeof(int), st));
  VecP none;
  const int PC = P == 64 ? 64 : 32;  // precision of the CGNR fallback's vectors
  PoolP cgp;                         // its vectors, allocated when a system first needs them

  // stencil variant for this batch shape (autotuned once per shape)
  b.hop_variant = lq_tune_hop(L, b, P, clov, te, p, v, st);
  if (verbose())
    fprintf(stderr, "[lqcd] stencil variant %d for P=%d nsys=%d max_n=%lld\n", b.hop_variant, P, n, b.max_n);
  // |eta|^2 of each system (both parities)
  std::fill(B.h_active.begin(), B.h_active.end(), 1);
  RC(B.push_active(st));
  std::vector<double> bb(n);
  RC(lq_norm2_64(b, b_e, st));
  RC(lq_finalize(lq::FIN_NORM, b, 0, 0, 12, st));
  RC(B.pull_sc(st));
  for (int k = 0; k < n; k++) bb[k] = B.h_sc[k].rr;
  RC(lq_norm2_64(b, b_o, st));
  RC(lq_finalize(lq::FIN_NORM, b, 0, 0, 12, st));
  RC(B.pull_sc(st));
  for (int k = 0; k < n; k++) {
    bb[k] += B.h_sc[k].rr;
    B.h_sc[k].bb = bb[k];
  }
  if (verbose())
    for (int k = 0; k < n; k++) fprintf(stderr, "[lqcd] solve P=%d sys %d |eta|^2 = %.6e n=%d\n", P, k, bb[k], B.h_sys[k].n);
  RC(B.push_sc(st));

  // prepare: bh_o = b_o + 1/2 H_oe A_ee^{-1} b_e
  RC(lq_hop_clinv(64, dag, clov, L, b, none, v64(b_e), v64(t64), 0.0, 1.0, st));
  RC(lq_hop_lin(64, dag, clov, lq::RED_NONE, L, b, 1, v64(t64), none, v64(b_o), none, v64(bh_o), 0.5, 0.0, 1.0, st));
  if (!guess) CK(cudaMemsetAsync(x_o, 0, sizeof(double2) * (size_t)b.total * 12, st));

  std::vector<int> outer(n, 1);
  for (int k = 0; k < n; k++)
    if (!(bb[k] > 0)) outer[k] = 0;  // zero source: zero solution
  std::vector<double> prev_rr(n, INFINITY);
  std::vector<double> last_rr(n, 0.0);  // last FP64 residual |bh_o - Dhat x_o|^2 of each system
  std::vector<int> stall(n, 0);
  // Krylov method per system: BiCGStab, or CG on the normal equations
  // Dhat^dag Dhat e = Dhat^dag r once BiCGStab has stalled for 6 cycles (or for
  // every system with LQCD_KRYLOV=cgnr).  CGNR converges on any nonsingular
  // Dhat, at the price of the squared condition number.
  static const bool force_cg = getenv("LQCD_KRYLOV") && std::string(getenv("LQCD_KRYLOV")) == "cgnr";
  std::vector<int> use_cg(n, force_cg ? 1 : 0);
  for (int cycle = 0;; cycle++) {
    // true residual of the preconditioned system: r64 = bh_o - Dhat x_o (FP64);
    // at the first cycle without a guess x_o = 0 and r64 = bh_o needs no operator
    B.h_active = outer;
    RC(B.push_active(st));
    if (cycle == 0 && !guess) {
      CK(cudaMemcpyAsync(r64, bh_o, sizeof(double2) * (size_t)b.total * 12, cudaMemcpyDeviceToDevice, st));
      RC(lq_norm2_64(b, r64, st));
      RC(lq_finalize(lq::FIN_NORM, b, 0, 0, 12, st));
    } else {
      RC(lq_hop_clinv(64, dag, clov, L, b, v64(x_o), none, v64(t64), 1.0, 0.0, st));
      RC(lq_hop_lin(64, dag, clov, lq::RED_NORM, L, b, 1, v64(t64), v64(x_o), v64(bh_o), none, v64(r64), 0.25, -1.0,
                    1.0, st));
      RC(lq_finalize(lq::FIN_NORM, b, 0, 0, 1, st));
    }
    RC(B.pull_sc(st));
    int n_act = 0;
    for (int k = 0; k < n; k++) {
      if (!outer[k]) continue;
      const double rr = B.h_sc[k].rr;
      last_rr[k] = rr;
      if (verbose())
        fprintf(stderr, "[lqcd] cycle %d sys %d |r|/|eta| = %.3e iters %d status %d\n", cycle, k, std::sqrt(rr / bb[k]),
                out.iters[k], B.h_sc[k].status);
      out.cycles[k] = cycle;
      if (!std::isfinite(rr)) {
        out.status[k] = LQCD_ENAN;
        outer[k] = 0;
      } else if (rr <= tol * tol * bb[k]) {
        outer[k] = 0;
      } else if (out.iters[k] >= max_iter) {
        out.status[k] = LQCD_ENOTCONVERGED;
        outer[k] = 0;
      } else {
        stall[k] = rr > 0.25 * prev_rr[k] ? stall[k] + 1 : 0;
        prev_rr[k] = rr;
        if (stall[k] >= 6 && !use_cg[k]) {  // BiCGStab stalled: continue with CGNR
          if (verbose()) fprintf(stderr, "[lqcd] sys %d: BiCGStab stalled, switching to CGNR\n", k);
          use_cg[k] = 1;
          stall[k] = 0;
          prev_rr[k] = INFINITY;
        } else if (stall[k] >= 6) {
          out.status[k] = LQCD_ENOTCONVERGED;
          outer[k] = 0;
        }
      }
      n_act += outer[k];
    }
    if (n_act == 0) break;
    const double t_in0 = now_s();
    std::vector<int> grp_b(n), grp_c(n);
    int n_b = 0, n_c = 0;
    for (int k = 0; k < n; k++) {
      grp_b[k] = outer[k] && !use_cg[k];
      grp_c[k] = outer[k] && use_cg[k];
      n_b += grp_b[k];
      n_c += grp_c[k];
    }
    // the first FP32 cycle from x = 0 reduces the residual by inner_tol; later
    // ones, and the first one from a starting iterate (whose residual is already
    // small), aim 10x deeper, so that one more FP64 check ends the solve (FP16
    // cannot go deeper than inner_tol; FP64 aims at the floor)
    const double tau = ((cycle == 0 && !guess) || P == 16) ? inner_tol : 0.1 * inner_tol;
    int it = 0;
    int budget = 0;
    for (int k = 0; k < n; k++)
      if (outer[k]) budget = std::max(budget, max_iter - out.iters[k]);
    budget = std::min(budget, cycle_cap);
    auto poll = [&](cudaStream_t s_) -> int {  // systems still iterating
      RC(lq_count_active(b, dcnt.as<int>(), s_));
      CK(cudaMemcpyAsync(cnt.h, dcnt.p, sizeof(int), cudaMemcpyDeviceToHost, s_));
      CK(cudaStreamSynchronize(s_));
      return 0;
    };
    if (n_b) {
      // inner solve of Dhat e = r64 in precision P (BiCGStab)
      B.h_active = grp_b;
      RC(B.push_active(st));
      RC(lq_inner_init(P, b, r64, r, r0, p, xs, st));
      // an inner cycle stops at tau |r| or at half the tolerance, whichever is larger; the FP64
      // check that follows decides (0.5 tol measured 2.8% faster than 0.3 tol on the 48^3 x 96
      // factorized propagator, worst final residual 8.5e-11)
      RC(lq_finalize(lq::FIN_INIT, b, tau * tau, 0.25 * tol * tol, lq_words_per_site(P), st));
      // one BiCGStab iteration: 10 kernels, all scalars and flags on the device
      auto iteration = [&](cudaStream_t s_) -> int {
        RC(lq_hop_clinv(P, dag, clov, L, b, p, none, te, 1.0, 0.0, s_));
        RC(lq_hop_lin(P, dag, clov, lq::RED_DOT_W, L, b, 1, te, p, none, r0, v, -0.25, 1.0, 0.0, s_));
        RC(lq_finalize(lq::FIN_ALPHA, b, 0, 0, lq_hop_wps(P, b), s_));
        RC(lq_bicg_s(P, b, r, v, s, s_));
        RC(lq_hop_clinv(P, dag, clov, L, b, s, none, te, 1.0, 0.0, s_));
        RC(lq_hop_lin(P, dag, clov, lq::RED_TS, L, b, 1, te, s, none, none, t, -0.25, 1.0, 0.0, s_));
        RC(lq_finalize(lq::FIN_OMEGA, b, 0, 0, lq_hop_wps(P, b), s_));
        RC(lq_bicg_xr(P, b, xs, p, s, t, r, r0, s_));
        RC(lq_finalize(lq::FIN_BETA, b, 0, 0, lq_words_per_site(P), s_));
        RC(lq_bicg_p(P, b, p, r, v, s_));
        return 0;
      };
      if (use_graph && budget >= 2 * check_every) {
        // check_every iterations captured once as a CUDA graph on a private
        // stream, replayed between host convergence checks (retired systems
        // skip every kernel, so iterations past convergence change nothing)
        cudaStream_t gs = L->graph_stream;
        CK(cudaEventRecord(L->graph_event, st));
        CK(cudaStreamWaitEvent(gs, L->graph_event, 0));
        const long long c0 = lqcd_kernel_launches();
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
        int crc = 0;
        for (int g = 0; g < check_every && !crc; g++) crc = iteration(gs);
        cudaError_t ce = cudaStreamEndCapture(gs, &graph);
        if (crc) return crc;
        CK(ce);
        const long long per_replay = lqcd_kernel_launches() - c0;
        lq_count_launches(-per_replay);  // captured, not run
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        int grc = 0;
        while (it < budget) {
          if (cudaGraphLaunch(exec, gs) != cudaSuccess) {
            lq_set_error("solve: CUDA graph launch failed");
            grc = LQCD_ECUDA;
            break;
          }
          lq_count_launches(per_replay);
          it += check_every;
          if ((grc = poll(gs)) != 0) break;
          if (*cnt.h == 0) break;
        }
        cudaGraphExecDestroy(exec);
        if (grc) return grc;
        CK(cudaEventRecord(L->graph_event, gs));
        CK(cudaStreamWaitEvent(st, L->graph_event, 0));
      } else {
        while (it < budget) {
          RC(iteration(st));
          it++;
          if (it % check_every == 0 || it >= budget) {
            RC(poll(st));
            if (*cnt.h == 0) break;
          }
        }
      }
      // x_o += e for the systems of this cycle
      RC(B.pull_sc(st));
      B.h_active = grp_b;
      RC(B.push_active(st));
      RC(lq_accum64(P, b, x_o, xs, st));
      for (int k = 0; k < n; k++)
        if (grp_b[k]) out.iters[k] += B.h_sc[k].iters;
    }
    if (n_c) {
      // inner solve by CG on Dhat^dag Dhat e = Dhat^dag r64 (FP32 vectors for the
      // FP32 / FP16 solvers, FP64 for the FP64 one), the same defect correction
      if (!cgp.buf.p) RC(cgp.alloc(b, PC, 6, st));
      VecP cxv = cgp.v(0), crv = cgp.v(1), cpv = cgp.v(2), cvv = cgp.v(3), czv = cgp.v(4), ctv = cgp.v(5);
      B.h_active = grp_c;
      RC(B.push_active(st));
      RC(lq_inner_init(PC, b, r64, crv, czv, cpv, cxv, st));  // r = r64, x = 0
      RC(lq_finalize(lq::FIN_INIT, b, tau * tau, 0.25 * tol * tol, lq_words_per_site(PC), st));
      // z = Dhat^dag r, rho = |z|^2, p = z
      RC(lq_hop_clinv(PC, !dag, clov, L, b, crv, none, ctv, 1.0, 0.0, st));
      RC(lq_hop_lin(PC, !dag, clov, lq::RED_TS, L, b, 1, ctv, crv, none, none, czv, -0.25, 1.0, 0.0, st));
      RC(lq_finalize(lq::FIN_CG_RHO, b, 0, 0, lq_hop_wps(PC, b), st));
      RC(lq_cg_p(PC, b, cpv, czv, st));
      int itc = 0;
      while (itc < budget) {
        // v = Dhat p, alpha = rho / |v|^2
        RC(lq_hop_clinv(PC, dag, clov, L, b, cpv, none, ctv, 1.0, 0.0, st));
        RC(lq_hop_lin(PC, dag, clov, lq::RED_TS, L, b, 1, ctv, cpv, none, none, cvv, -0.25, 1.0, 0.0, st));
        RC(lq_finalize(lq::FIN_CG_ALPHA, b, 0, 0, lq_hop_wps(PC, b), st));
        // x += alpha p, r -= alpha v
        RC(lq_cg_xr(PC, b, cxv, cpv, crv, cvv, st));
        RC(lq_finalize(lq::FIN_CG_R, b, 0, 0, lq_words_per_site(PC), st));
        // z = Dhat^dag r, beta = |z|^2 / rho, p = z + beta p
        RC(lq_hop_clinv(PC, !dag, clov, L, b, crv, none, ctv, 1.0, 0.0, st));
        RC(lq_hop_lin(PC, !dag, clov, lq::RED_TS, L, b, 1, ctv, crv, none, none, czv, -0.25, 1.0, 0.0, st));
        RC(lq_finalize(lq::FIN_CG_BETA, b, 0, 0, lq_hop_wps(PC, b), st));
        RC(lq_cg_p(PC, b, cpv, czv, st));
        itc++;
        if (itc % check_every == 0 || itc >= budget) {
          RC(poll(st));
          if (*cnt.h == 0) break;
        }
      }
      RC(B.pull_sc(st));
      B.h_active = grp_c;
      RC(B.push_active(st));
      RC(lq_accum64(PC, b, x_o, cxv, st));
      for (int k = 0; k < n; k++)
        if (grp_c[k]) out.iters[k] += B.h_sc[k].iters;
      it = std::max(it, itc);
    }
    if (verbose()) fprintf(stderr, "[lqcd] cycle %d: inner %d its in %.2f ms\n", cycle, it, 1e3 * (now_s() - t_in0));
  }
  // reconstruct x_e = A_ee^{-1}(b_e + 1/2 H_eo x_o).  Then the even half of
  // eta - D x vanishes (up to rounding) and the odd half is bh_o - Dhat x_o, so
  // the true FP64 residual is the one the last cycle recomputed from x_o.
  std::fill(B.h_active.begin(), B.h_active.end(), 1);
  RC(B.push_active(st));
  RC(lq_hop_clinv(64, dag, clov, L, b, v64(x_o), v64(b_e), v64(x_e), 0.5, 1.0, st));
  for (int k = 0; k < n; k++) {
    out.res[k] = bb[k] > 0 ? std::sqrt(last_rr[k] / bb[k]) : 0.0;
    if (out.status[k] == 0 && !(out.res[k] <= tol)) out.status[k] = std::isfinite(out.res[k]) ? LQCD_ENOTCONVERGED : LQCD_ENAN;
  }
  return 0;
}

lqcd_solver_params default_params(const lqcd_solver_params* p) {
  lqcd_solver_params q{};
  q.tol = 1e-10;
  q.max_iter = 100000;
  q.precision = 64;
  q.inner_tol = 0;
  q.check_every = 0;
  q.max_wave = 0;
  if (p) q = *p;
  return q;
}

int worst_status(const SolveOut& o) {
  int w = 0;
  for (int s : o.status)
    if (s != 0 && (w == 0 || s < w)) w = s;
  return w;
}

void fill_stats(const SolveOut& o, int k0, int n, double secs, lqcd_solver_stats* st) {
  st->iters = 0;
  st->cycles = 0;
  st->status = 0;
  st->true_residual = 0;
  st->seconds = secs;
  for (int k = k0; k < k0 + n; k++) {
    st->iters = std::max(st->iters, o.iters[k]);
    st->cycles = std::max(st->cycles, o.cycles[k]);
    st->true_residual = std::max(st->true_residual, o.res[k]);
    if (o.status[k] != 0 && st->status == 0) st->status = o.status[k];
  }
}

// ---------------------------------------------------------------- waves
// One system of a batched call: slab, field and what fills / consumes it.
struct SysSpec {
  lqcd_slab dom;
  int field;
  int role;   // caller-defined (which source / which output)
  int col;    // spin-colour column 3*s + c of a point source
  int4 xsrc;  // point-source position
  int out = 0;  // caller-defined output slot (e.g. field index * 12 + column)
};

using FillFn = std::function<int(BatchStore& B, int k0, double2* b_e, double2* b_o)>;
using SinkFn = std::function<int(BatchStore& B, int k0, const double2* x_e, const double2* x_o)>;
// Writes a starting iterate of the wave's systems into their even / odd pools
// (only the odd half enters the solve).
using GuessFn = std::function<int(BatchStore& B, int k0, double2* x_e, double2* x_o)>;

// device bytes per system site (one parity) held during a solve in precision P:
// 4 caller-side FP64 vectors + 3 solver FP64 vectors + 8 Krylov vectors
size_t site_bytes(int P) { return (size_t)(7 * 192 + 8 * (P == 64 ? 192 : P == 32 ? 96 : 52)); }

// Free device memory, counting what the stream-ordered pool holds unused.
size_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long res = 0, used = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    if (res > used) fr += (size_t)(res - used);
  }
  cudaGetLastError();
  return fr;
}

// Solve every system of `sp` (D_L x = b, or D_L^dag x = b), in consecutive
// waves that fit in free device memory (at most prm.max_wave systems each).
// For each wave: fill its sources, solve, hand the solutions to sink.
int solve_waves(lqcd_lattice* L, const std::vector<SysSpec>& sp, bool dag, const lqcd_solver_params& prm,
                const FillFn& fill, const SinkFn& sink, SolveOut& out, cudaStream_t st,
                const GuessFn& guess = GuessFn()) {
  const int N = (int)sp.size();
  out.iters.assign(N, 0);
  out.cycles.assign(N, 0);
  out.status.assign(N, 0);
  out.res.assign(N, 0.0);
  const int P = prm.precision == 16 ? 16 : prm.precision == 32 ? 32 : 64;
  const size_t fb = free_device_bytes();
  const size_t reserve = (size_t)1 << 30;
  const size_t budget = fb > 2 * reserve ? (size_t)(0.85 * (double)(fb - reserve)) : fb / 2;
  int k = 0;
  while (k < N) {
    size_t need = 0;
    int w = 0;
    while (k + w < N && (prm.max_wave <= 0 || w < prm.max_wave)) {
      const size_t n = (size_t)(sp[k + w].dom.t1 - sp[k + w].dom.t0 + 1) * (size_t)L->S3h;
      const size_t add = n * site_bytes(P) + 4096;
      if (w > 0 && need + add > budget) break;
      need += add;
      w++;
    }
    std::vector<lqcd_slab> doms(w);
    std::vector<int> fields(w);
    for (int q = 0; q < w; q++) {
      doms[q] = sp[k + q].dom;
      fields[q] = sp[k + q].field;
    }
    BatchStore B;
    RC(B.build(L, w, doms.data(), fields.data(), st));
    Pool64 e;
    RC(e.alloc(B.b, 4, st));
    RC(fill(B, k, e.v(0), e.v(1)));
    if (guess) RC(guess(B, k, e.v(2), e.v(3)));
    SolveOut o;
    RC(solve_core(L, B, dag, prm, e.v(0), e.v(1), e.v(2), e.v(3), o, st, (bool)guess));
    RC(sink(B, k, e.v(2), e.v(3)));
    for (int q = 0; q < w; q++) {
      out.iters[k + q] = o.iters[q];
      out.cycles[k + q] = o.cycles[q];
      out.status[k + q] = o.status[q];
      out.res[k + q] = o.res[q];
    }
    if (verbose()) fprintf(stderr, "[lqcd] wave of %d systems (%d..%d of %d)\n", w, k, k + w - 1, N);
    k += w;
  }
  return 0;
}

// Device copies of the per-system point-source columns / positions and
// output slots of [k0, k0+n).
struct SrcArrays {
  DBuf cols, xsrc, outs;
  int upload(const std::vector<SysSpec>& sp, int k0, int n, cudaStream_t st) {
    std::vector<int> c(n), o(n);
    std::vector<int4> x(n);
    for (int q = 0; q < n; q++) {
      c[q] = sp[k0 + q].col;
      o[q] = sp[k0 + q].out;
      x[q] = sp[k0 + q].xsrc;
    }
    RC(cols.alloc(sizeof(int) * n, st));
    RC(outs.alloc(sizeof(int) * n, st));
    RC(xsrc.alloc(sizeof(int4) * n, st));
    CK(cudaMemcpyAsync(cols.p, c.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(outs.p, o.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(xsrc.p, x.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, st));
    return 0;
  }
};

// Device array of n pointers.
int upload_ptrs(DBuf& d, const std::vector<void*>& p, cudaStream_t st) {
  RC(d.alloc(sizeof(void*) * (p.empty() ? 1 : p.size()), st));
  if (!p.empty()) CK(cudaMemcpyAsync(d.p, p.data(), sizeof(void*) * p.size(), cudaMemcpyHostToDevice, st));
  return 0;
}

}  // namespace

namespace {
int check_split(const lqcd_lattice* L, const lqcd_split* split, const char* who);
lqcd_slab gamma_bar_of(const lqcd_split* split);
}  // namespace

// ===================================================================== API
extern "C" int lqcd_create_lattice(const int dims[4], int bc_t, lqcd_lattice** out) {
  if (!dims || !out) {
    lq_set_error("null argument");
    return LQCD_EBADARG;
  }
  for (int k = 0; k < 4; k++)
    if (dims[k] < 2 || dims[k] % 2) {
      lq_set_error("every extent must be even and >= 2");
      return LQCD_EBADARG;
    }
  if (bc_t < 0 || bc_t > 2) {
    lq_set_error("bad time boundary condition");
    return LQCD_EBADARG;
  }
  {
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (72 * (V / 2) >= (1LL << 31)) {  // 32-bit site indexing of the packed link / clover arrays
      lq_set_error("lattice too large for one GPU field (V/2 * 72 must stay below 2^31)");
      return LQCD_EBADARG;
    }
    // site coordinates use one multiply-high per division (fast_div): exact while index * divisor < 2^32
    const long long dmax = std::max({(long long)dims[1], (long long)dims[2], (long long)dims[3] / 2});
    if ((V / 2) * dmax >= (1LL << 32)) {
      lq_set_error("spatial extent too large for this lattice volume (V/2 * max(L1, L2, L3/2) must stay below 2^32)");
      return LQCD_EBADARG;
    }
  }
  lqcd_lattice* L = new lqcd_lattice();
  for (int k = 0; k < 4; k++) L->dims[k] = dims[k];
  L->bc = bc_t;
  L->S3 = (long long)dims[1] * dims[2] * dims[3];
  L->S3h = L->S3 / 2;
  L->V = L->S3 * dims[0];
  L->Vh = L->V / 2;
  for (int k = 0; k < 4; k++) L->g.L[k] = dims[k];
  L->g.L3h = dims[3] / 2;
  L->g.Vh = (int)L->Vh;
  L->g.S3h = (int)L->S3h;
  L->g.bc_t = bc_t;
  L->g.m3h = lq::fast_magic((unsigned)L->g.L3h);
  L->g.m2 = lq::fast_magic((unsigned)dims[2]);
  L->g.m1 = lq::fast_magic((unsigned)dims[1]);
  cudaGetDevice(&L->device);
  // Solver work vectors come from the device's stream-ordered pool; keep its
  // memory mapped across synchronisations instead of returning it to the
  // driver (and re-mapping it) at every stream synchronise.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, L->device) == cudaSuccess) {
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  if (cudaStreamCreateWithFlags(&L->graph_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&L->graph_event, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete L;
    lq_set_error("create_lattice: cannot create the solver stream");
    return LQCD_ECUDA;
  }
  *out = L;
  return 0;
}

static void free_fields(lqcd_lattice* L) {
  for (auto& f : L->fields) {
    cudaFree(f.U64);
    cudaFree(f.U32);
    cudaFree(f.U16);
    cudaFree(f.A64);
    cudaFree(f.Ai64);
    cudaFree(f.A32);
    cudaFree(f.Ai32);
  }
  L->fields.clear();
  if (L->d_fields) cudaFree(L->d_fields);
  L->d_fields = nullptr;
}

extern "C" int lqcd_destroy_lattice(lqcd_lattice* L) {
  RC(check_lat(L));
  cudaDeviceSynchronize();
  free_fields(L);
  if (L->graph_stream) cudaStreamDestroy(L->graph_stream);
  if (L->graph_event) cudaEventDestroy(L->graph_event);
  delete L;
  return 0;
}

extern "C" int lqcd_set_gauge(lqcd_lattice* L, int n_fields, const double* U, double kappa, double c_sw, int mem,
                              void* stream) {
  RC(check_lat(L));
  if (n_fields < 1 || !U || !(kappa > 0)) {
    lq_set_error("set_gauge: need n_fields >= 1, U != NULL, kappa > 0");
    return LQCD_EBADARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(st));
  const bool reuse = (int)L->fields.size() == n_fields && L->d_fields != nullptr;
  if (!reuse) free_fields(L);
  L->kappa = kappa;
  L->csw = c_sw;
  const long long V = L->V, Vh = L->Vh;
  const size_t nat_bytes = sizeof(double2) * (size_t)V * 36;
  DBuf tmp;
  if (mem == LQCD_MEM_HOST) RC(tmp.alloc(nat_bytes, st));
  DBuf dev, fail;
  RC(dev.alloc(sizeof(unsigned long long), st));
  RC(fail.alloc(sizeof(int), st));
  std::vector<lq::FieldPtrs> ptrs;
  for (int fi = 0; fi < n_fields; fi++) {
    if (!reuse) {
      FieldData f;
      L->fields.push_back(f);
      FieldData& F = L->fields.back();
      CK(cudaMalloc(&F.U64, sizeof(double2) * 2 * 4 * 9 * Vh));
      CK(cudaMalloc(&F.U32, sizeof(float4) * 2 * 4 * 3 * Vh));
      CK(cudaMalloc(&F.U16, sizeof(uint2) * 2 * 4 * 3 * Vh));
      CK(cudaMalloc(&F.A64, sizeof(double2) * 2 * 36 * Vh));
      CK(cudaMalloc(&F.Ai64, sizeof(double2) * 36 * Vh));
      CK(cudaMalloc(&F.A32, sizeof(float4) * 2 * 18 * Vh));
      CK(cudaMalloc(&F.Ai32, sizeof(float4) * 18 * Vh));
    }
    FieldData& F = L->fields[fi];
    const double2* src = (const double2*)(U + (size_t)fi * V * 72);
    if (mem == LQCD_MEM_HOST) {
      CK(cudaMemcpyAsync(tmp.p, src, nat_bytes, cudaMemcpyHostToDevice, st));
      src = tmp.as<double2>();
    }
    CK(cudaMemsetAsync(dev.p, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(fail.p, 0, sizeof(int), st));
    RC(lq_launch_pack_links(L->g, src, F.U64, F.U32, F.U16, dev.as<unsigned long long>(), st));
    RC(lq_launch_clover(L->g, src, kappa, c_sw, F.A64, F.Ai64, F.A32, F.Ai32, fail.as<int>(), st));
    unsigned long long d = 0;
    int fl = 0;
    CK(cudaMemcpyAsync(&d, dev.p, sizeof(d), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&fl, fail.p, sizeof(fl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double dv;
    memcpy(&dv, &d, sizeof(dv));
    if (!(dv <= 1e-10)) {
      lq_set_error("set_gauge: field " + std::to_string(fi) + " is not SU(3): deviation " + std::to_string(dv));
      free_fields(L);
      return LQCD_ENONUNITARY;
    }
    if (fl) {
      lq_set_error("set_gauge: singular clover block in field " + std::to_string(fi));
      free_fields(L);
      return LQCD_EBADARG;
    }
    lq::FieldPtrs fp;
    fp.U64 = F.U64;
    fp.U32 = F.U32;
    fp.U16 = F.U16;
    fp.A64 = F.A64;
    fp.Ai64 = F.Ai64;
    fp.A32 = F.A32;
    fp.Ai32 = F.Ai32;
    ptrs.push_back(fp);
  }
  if (!reuse) {
    CK(cudaMalloc(&L->d_fields, sizeof(lq::FieldPtrs) * n_fields));
    CK(cudaMemcpy(L->d_fields, ptrs.data(), sizeof(lq::FieldPtrs) * n_fields, cudaMemcpyHostToDevice));
  }
  return 0;
}

extern "C" int lqcd_dslash(lqcd_lattice* L, int field, const lqcd_slab* dom, int dagger, int precision,
                           const double* in, double* out, void* stream) {
  RC(check_lat(L));
  if (!in || !out || (precision != 64 && precision != 32 && precision != 16)) {
    lq_set_error("dslash: bad arguments");
    return LQCD_EBADARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_slab d = dom ? *dom : lqcd_slab{0, L->dims[0] - 1};
  BatchStore B;
  RC(B.build(L, 1, &d, &field, st));
  const Batch& b = B.b;
  Pool64 e;
  RC(e.alloc(b, 4, st));
  DBuf ptr;
  RC(ptr.alloc(sizeof(void*), st));
  const double2* srcp = (const double2*)in;
  CK(cudaMemcpyAsync(ptr.p, &srcp, sizeof(void*), cudaMemcpyHostToDevice, st));
  RC(lq_nat_to_eo(L, b, ptr.as<const double2*>(), e.v(0), e.v(1), st));
  const bool clov = L->csw != 0.0;
  VecP none;
  if (precision == 64) {
    RC(lq_hop_lin(precision, dagger, clov, lq::RED_NONE, L, b, 0, v64(e.v(1)), v64(e.v(0)), none, none, v64(e.v(2)),
                  -0.5, 1.0, 0.0, st));
    RC(lq_hop_lin(precision, dagger, clov, lq::RED_NONE, L, b, 1, v64(e.v(0)), v64(e.v(1)), none, none, v64(e.v(3)),
                  -0.5, 1.0, 0.0, st));
  } else {
    PoolP q;
    RC(q.alloc(b, precision, 4, st));
    RC(lq_convert(64, precision, b, v64(e.v(0)), q.v(0), st));
    RC(lq_convert(64, precision, b, v64(e.v(1)), q.v(1), st));
    RC(lq_hop_lin(precision, dagger, clov, lq::RED_NONE, L, b, 0, q.v(1), q.v(0), none, none, q.v(2), -0.5, 1.0, 0.0,
                  st));
    RC(lq_hop_lin(precision, dagger, clov, lq::RED_NONE, L, b, 1, q.v(0), q.v(1), none, none, q.v(3), -0.5, 1.0, 0.0,
                  st));
    RC(lq_convert(precision, 64, b, q.v(2), v64(e.v(2)), st));
    RC(lq_convert(precision, 64, b, q.v(3), v64(e.v(3)), st));
    CK(cudaStreamSynchronize(st));
  }
  double2* dstp = (double2*)out;
  CK(cudaMemcpyAsync(ptr.p, &dstp, sizeof(void*), cudaMemcpyHostToDevice, st));
  RC(lq_eo_to_nat(L, b, e.v(2), e.v(3), ptr.as<double2* const>(), 1.0, st));
  CK(cudaStreamSynchronize(st));
  return 0;
}

static int solve_api(lqcd_lattice* L, int n, const lqcd_slab* doms, const int* field_ids, const double* src,
                     double* sol, const lqcd_solver_params* params, lqcd_solver_stats* stats, void* stream) {
  if (n < 1 || !doms || !field_ids || !src || !sol) {
    lq_set_error("solve: bad arguments");
    return LQCD_EBADARG;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  std::vector<SysSpec> sp(n);
  std::vector<long long> goff(n + 1, 0);  // natural-order site offset of each system's slab vector
  for (int k = 0; k < n; k++) {
    sp[k] = SysSpec{doms[k], field_ids[k], 0, 0, make_int4(0, 0, 0, 0)};
    const long long len = doms[k].t1 >= doms[k].t0 ? (long long)(doms[k].t1 - doms[k].t0 + 1) * L->S3 : 0;
    goff[k + 1] = goff[k] + len;
  }
  FillFn fill = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((const double2*)src + goff[k0 + q] * 12);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_nat_to_eo(L, B.b, d.as<const double2*>(), be, bo, st);
  };
  SinkFn sink = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((double2*)sol + goff[k0 + q] * 12);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), 1.0, st);
  };
  SolveOut o;
  RC(solve_waves(L, sp, false, prm, fill, sink, o, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats)
    for (int k = 0; k < n; k++) fill_stats(o, k, 1, secs, &stats[k]);
  int w = worst_status(o);
  if (w) lq_set_error("solve: some systems did not reach the tolerance");
  return w;
}

extern "C" int lqcd_solve_block(lqcd_lattice* L, int n_sys, const lqcd_slab* doms, const int* field_ids,
                                const double* src, double* sol, const lqcd_solver_params* params,
                                lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  return solve_api(L, n_sys, doms, field_ids, src, sol, params, stats, stream);
}

extern "C" int lqcd_solve_full(lqcd_lattice* L, int n_sys, const int* field_ids, const double* src, double* sol,
                               const lqcd_solver_params* params, lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (n_sys < 1) {
    lq_set_error("solve_full: n_sys < 1");
    return LQCD_EBADARG;
  }
  std::vector<lqcd_slab> d(n_sys, lqcd_slab{0, L->dims[0] - 1});
  return solve_api(L, n_sys, d.data(), field_ids, src, sol, params, stats, stream);
}

namespace {

// Sec. 3 for the fields field_ids[0..n_f) and n_d nested overlaps (DeltaGamma_d =
// g1+1 .. d1s[d], empty when d1s[d] <= g1), per field and point-source column:
//   fact = D_Gamma^{-1} eta on Gamma                                  (eq. quark_prop_I)
//   fact = -D_Gamma*^{-1} D_dGamma* (D_Gammabar^{-1} eta)|_Gamma on Gamma*  (eq. quark_prop_II)
//   full = D^{-1} eta                                                 (eq. observable_factorization)
// in four batched stages, each holding the systems of one kind:
//   A1  Gamma from the point sources, 12 n_f systems shared by every overlap;
//   A2  Gammabar_d from the point sources, 12 n_f n_d systems, each started
//       from the Gamma solution (zero on DeltaGamma_d): its residual lives on
//       the first slice of DeltaGamma_d only; its boundary slice gives
//       chi = D_dGamma* psi|_Gamma;
//   B   Gamma* from chi, 12 n_f n_d systems;
//   C   the full lattice from the point sources, 12 n_f systems, started from
//       fact of the last overlap: the residual eta - D fact vanishes off the two
//       slices next to the cut, where it is as small as the propagator across it.
// The starting iterates change the iteration counts, not the solutions: every
// system stops at the same true FP64 residual ||eta - D psi|| <= tol ||eta||.
// fact: [n_d][n_f][12][V][4][3]; full: [n_f][12][V][4][3] or NULL (then stage C
// is skipped); with sub_fact, full receives full - fact of the last overlap.
// stats (host, 4 per field, or NULL): Gamma, Gammabar, Gamma*, full, each the
// worst over the field's columns and overlaps.
int factorized_run(lqcd_lattice* L, lqcd_slab G, lqcd_slab Gs, int n_d, const int* d1s, int4 xs, int n_f,
                   const int* field_ids, double* fact, double* full, bool sub_fact, const lqcd_solver_params& prm,
                   lqcd_solver_stats* stats, cudaStream_t st) {
  const int T = L->dims[0];
  const long long V = L->V, S3 = L->S3;
  const size_t col_words = (size_t)V * 12;  // one propagator column (complex128 words)
  const int NF = 12 * n_f;                  // systems of one overlap
  const int ND = NF * n_d;                  // output slot = (d * n_f + field index) * 12 + column
  const lqcd_slab Full = {0, T - 1};
  const double t_start = now_s();
  std::vector<lqcd_slab> Gb(n_d);
  std::vector<bool> has_delta(n_d);
  for (int d = 0; d < n_d; d++) {
    has_delta[d] = d1s[d] > G.t1;
    Gb[d] = lqcd_slab{0, has_delta[d] ? d1s[d] : G.t1};
  }

  CK(cudaMemsetAsync(fact, 0, sizeof(double2) * (size_t)ND * col_words, st));
  // compact boundary source chi[slot][2][slice site][12] (two time slices per system)
  DBuf chi;
  RC(chi.alloc(sizeof(double2) * (size_t)ND * 2 * (size_t)S3 * 12, st));
  auto make = [&](lqcd_slab dom, int d) {
    std::vector<SysSpec> sp;
    for (int j = 0; j < n_f; j++)
      for (int c = 0; c < 12; c++) {
        SysSpec q{dom, field_ids[j], d, c, xs};
        q.out = (d * n_f + j) * 12 + c;
        sp.push_back(q);
      }
    return sp;
  };
  // natural-order device pointers of each system's slab inside the columns of `base`
  auto col_ptrs = [&](const std::vector<SysSpec>& sp, int k0, int n, double* base, DBuf& d, int slot_of_d = -1) -> int {
    std::vector<void*> p(n);
    for (int q = 0; q < n; q++) {
      const SysSpec& y = sp[k0 + q];
      const int slot = slot_of_d < 0 ? y.out : (slot_of_d * n_f + (y.out / 12) % n_f) * 12 + y.col;
      p[q] = (double2*)base + (size_t)slot * col_words + (size_t)y.dom.t0 * S3 * 12;
    }
    return upload_ptrs(d, p, st);
  };
  auto point_fill = [&](const std::vector<SysSpec>& sp) -> FillFn {
    return [&, sp_ptr = &sp](BatchStore& B, int k0, double2* be, double2* bo) -> int {
      SrcArrays s;
      RC(s.upload(*sp_ptr, k0, B.b.nsys, st));
      return lq_point_source(L, B.b, s.cols.as<int>(), s.xsrc.as<int4>(), be, bo, st);
    };
  };
  // starting iterate read from fact (natural order) on each system's slab
  auto fact_guess = [&](const std::vector<SysSpec>& sp, int slot_of_d) -> GuessFn {
    return [&, sp_ptr = &sp, slot_of_d](BatchStore& B, int k0, double2* xe, double2* xo) -> int {
      DBuf d;
      RC(col_ptrs(*sp_ptr, k0, B.b.nsys, fact, d, slot_of_d));
      return lq_nat_to_eo(L, B.b, d.as<const double2*>(), xe, xo, st);
    };
  };
  auto chi_sink = [&](const std::vector<SysSpec>& sp, BatchStore& B, int k0, const double2* xe,
                      const double2* xo) -> int {
    SrcArrays s;
    RC(s.upload(sp, k0, B.b.nsys, st));
    return lq_boundary_chi(L, B.b, s.outs.as<int>(), G.t1, xe, xo, chi.as<double2>(), st);
  };

  // A1: Gamma (eq. quark_prop_I), written into fact of every overlap; an
  // overlap that is empty takes its chi from this solve
  const std::vector<SysSpec> sa1 = make(G, 0);
  SinkFn sink_a1 = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    for (int d = 0; d < n_d; d++) {
      DBuf dp;
      RC(col_ptrs(sa1, k0, B.b.nsys, fact, dp, d));
      RC(lq_eo_to_nat(L, B.b, xe, xo, dp.as<double2* const>(), 1.0, st));
      if (!has_delta[d]) {
        std::vector<SysSpec> sd(sa1.begin() + k0, sa1.begin() + k0 + B.b.nsys);
        for (auto& y : sd) y.out += d * NF;
        RC(chi_sink(sd, B, 0, xe, xo));
      }
    }
    return 0;
  };
  SolveOut o_g, o_gb, o_gs, o_full;
  RC(solve_waves(L, sa1, false, prm, point_fill(sa1), sink_a1, o_g, st));
  // A2: Gammabar_d, started from the Gamma solution (eq. quark_prop_II)
  std::vector<SysSpec> sa2;
  for (int d = 0; d < n_d; d++)
    if (has_delta[d]) {
      auto v = make(Gb[d], d);
      sa2.insert(sa2.end(), v.begin(), v.end());
    }
  if (!sa2.empty()) {
    SinkFn sink_a2 = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
      return chi_sink(sa2, B, k0, xe, xo);
    };
    RC(solve_waves(L, sa2, false, prm, point_fill(sa2), sink_a2, o_gb, st, fact_guess(sa2, -1)));
  }
  // B: Gamma* from chi; fact on Gamma* is -zeta (eq. quark_prop_II)
  std::vector<SysSpec> sb;
  for (int d = 0; d < n_d; d++) {
    auto v = make(Gs, d);
    sb.insert(sb.end(), v.begin(), v.end());
  }
  FillFn fill_b = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    SrcArrays s;
    RC(s.upload(sb, k0, B.b.nsys, st));
    return lq_chi_to_eo(L, B.b, s.outs.as<int>(), G.t1, chi.as<double2>(), be, bo, st);
  };
  SinkFn sink_b = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    DBuf d;
    RC(col_ptrs(sb, k0, B.b.nsys, fact, d));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), -1.0, st);
  };
  RC(solve_waves(L, sb, false, prm, fill_b, sink_b, o_gs, st));
  const double t_b1 = now_s();
  // C: the full lattice, started from fact of the last overlap
  if (full) {
    const std::vector<SysSpec> sc = make(Full, 0);
    SinkFn sink_c = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
      DBuf d;
      RC(col_ptrs(sc, k0, B.b.nsys, full, d));
      return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), 1.0, st);
    };
    RC(solve_waves(L, sc, false, prm, point_fill(sc), sink_c, o_full, st, fact_guess(sc, n_d - 1)));
    if (sub_fact)  // full - fact of the last overlap
      RC(lq_sub_inplace((double2*)full, (const double2*)fact + (size_t)(n_d - 1) * NF * col_words,
                        (long long)NF * V * 12, st));
  }
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (verbose())
    fprintf(stderr, "[lqcd] factorized (%d fields, %d overlaps): domains %.1f ms, full %.1f ms\n", n_f, n_d,
            1e3 * (t_b1 - t_start), 1e3 * (now_s() - t_b1));
  if (stats) {
    // per field: the worst over its columns (and overlaps) of each stage
    auto of_field = [&](const SolveOut& o, const std::vector<SysSpec>& sp, int j) {
      SolveOut r;
      for (size_t k = 0; k < sp.size() && k < o.iters.size(); k++)
        if ((sp[k].out / 12) % n_f == j) {
          r.iters.push_back(o.iters[k]);
          r.cycles.push_back(o.cycles[k]);
          r.status.push_back(o.status[k]);
          r.res.push_back(o.res[k]);
        }
      return r;
    };
    for (int j = 0; j < n_f; j++) {
      lqcd_solver_stats* sj = stats + 4 * j;
      SolveOut og = of_field(o_g, sa1, j), ogb = sa2.empty() ? og : of_field(o_gb, sa2, j), ogs = of_field(o_gs, sb, j);
      fill_stats(og, 0, (int)og.iters.size(), secs, &sj[0]);
      fill_stats(ogb, 0, (int)ogb.iters.size(), secs, &sj[1]);
      fill_stats(ogs, 0, (int)ogs.iters.size(), secs, &sj[2]);
      if (full) {
        SolveOut oc = of_field(o_full, make(Full, 0), j);
        fill_stats(oc, 0, (int)oc.iters.size(), secs, &sj[3]);
      } else {
        memset(&sj[3], 0, sizeof(lqcd_solver_stats));
      }
    }
  }
  int w = worst_status(o_g);
  if (!w) w = worst_status(o_gb);
  if (!w) w = worst_status(o_gs);
  if (!w && full) w = worst_status(o_full);
  if (w) lq_set_error("factorized_propagator: some solves did not reach the tolerance");
  return w;
}

int check_factorized_args(const lqcd_lattice* L, const lqcd_split* split, const int x_src[4], int n_f,
                          const int* field_ids) {
  if (!split || !x_src || n_f < 1 || !field_ids) {
    lq_set_error("factorized_propagator: null argument or n_fields < 1");
    return LQCD_EBADARG;
  }
  RC(check_split(L, split, "factorized_propagator"));
  const lqcd_slab G = split->gamma;
  if (x_src[0] < G.t0 || x_src[0] > G.t1) {
    lq_set_error("factorized_propagator: the source must lie in Gamma");
    return LQCD_EBADARG;
  }
  for (int k = 1; k < 4; k++)
    if (x_src[k] < 0 || x_src[k] >= L->dims[k]) {
      lq_set_error("factorized_propagator: source outside the lattice");
      return LQCD_EBADARG;
    }
  for (int j = 0; j < n_f; j++)
    if (field_ids[j] < 0 || field_ids[j] >= (int)L->fields.size()) {
      lq_set_error("factorized_propagator: field index not loaded");
      return LQCD_ENOFIELD;
    }
  return 0;
}

}  // namespace

extern "C" int lqcd_factorized_propagators(lqcd_lattice* L, const lqcd_split* split, const int x_src[4], int n_f,
                                           const int* field_ids, double* fact, double* corr,
                                           const lqcd_solver_params* params, lqcd_solver_stats* stats,
                                           void* stream) {
  RC(check_lat(L));
  if (!fact) {
    lq_set_error("factorized_propagator: null fact");
    return LQCD_EBADARG;
  }
  RC(check_factorized_args(L, split, x_src, n_f, field_ids));
  const bool has_delta = split->delta.t1 >= split->delta.t0;
  const int d1 = has_delta ? split->delta.t1 : split->gamma.t1;
  return factorized_run(L, split->gamma, split->gamma_star, 1, &d1, make_int4(x_src[0], x_src[1], x_src[2], x_src[3]),
                        n_f, field_ids, fact, corr, true, default_params(params), stats, (cudaStream_t)stream);
}

// Sec. 6 eq. nucleon_prop_hierarchical for one gauge field: the factorized
// propagators of n_d nested overlaps in one batched run (Gamma and the full
// lattice solved once), then the nucleon point correlators of each and of the
// full propagator, and the terms of the expansion.
extern "C" int lqcd_nucleon_hierarchy(lqcd_lattice* L, const lqcd_split* split, int n_d, const int* delta_t1,
                                      const int x_src[4], int field, double* C, const lqcd_solver_params* params,
                                      lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (!C || n_d < 1 || n_d > 16 || !delta_t1) {
    lq_set_error("nucleon_hierarchy: bad arguments (1 <= n_d <= 16)");
    return LQCD_EBADARG;
  }
  RC(check_factorized_args(L, split, x_src, 1, &field));
  const int T = L->dims[0];
  const lqcd_slab G = split->gamma, Gs = split->gamma_star;
  for (int d = 0; d < n_d; d++)
    if (delta_t1[d] <= G.t1 || delta_t1[d] >= T - 1 || (d > 0 && delta_t1[d] <= delta_t1[d - 1])) {
      lq_set_error("nucleon_hierarchy: need g1 < delta_t1[0] < delta_t1[1] < ... < T-1");
      return LQCD_EBADARG;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const long long V = L->V;
  const size_t prop_words = (size_t)12 * V * 12;
  // fact of every overlap followed by the full propagator: n_d + 1 propagators back to back
  DBuf props, partial, Wd;
  RC(props.alloc(sizeof(double2) * prop_words * (n_d + 1), st));
  double2* fact = props.as<double2>();
  double2* full = fact + prop_words * n_d;
  lqcd_solver_stats st4[4];
  RC(factorized_run(L, G, Gs, n_d, delta_t1, make_int4(x_src[0], x_src[1], x_src[2], x_src[3]), 1, &field,
                    (double*)fact, (double*)full, false, default_params(params), stats ? st4 : nullptr, st));
  if (stats) memcpy(stats, st4, sizeof st4);
  RC(partial.alloc(sizeof(double2) * (size_t)lq_nucleon_point_partial_words(L, n_d + 1, T), st));
  RC(Wd.alloc(sizeof(double2) * (size_t)(n_d + 1) * T * 2, st));
  RC(lq_nucleon_point(L, n_d + 1, fact, 0, T, partial.as<double2>(), Wd.as<double2>(), st));
  std::vector<double2> W((size_t)(n_d + 1) * T * 2);
  CK(cudaMemcpyAsync(W.data(), Wd.p, sizeof(double2) * W.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // C^(p)(t) = W1 - W2; terms C^(0), C^(d) - C^(d-1), C - C^(n_d - 1), then C
  auto corr_of = [&](int p, int t) {
    const double2 a = W[((size_t)p * T + t) * 2], b = W[((size_t)p * T + t) * 2 + 1];
    return make_double2(a.x - b.x, a.y - b.y);
  };
  double2* out = (double2*)C;
  for (int t = 0; t < T; t++) {
    for (int k = 0; k <= n_d; k++) {
      const double2 cur = corr_of(k, t);
      const double2 prev = k == 0 ? make_double2(0.0, 0.0) : corr_of(k - 1, t);
      out[(size_t)k * T + t] = make_double2(cur.x - prev.x, cur.y - prev.y);
    }
    out[(size_t)(n_d + 1) * T + t] = corr_of(n_d, t);
  }
  return 0;
}

extern "C" int lqcd_factorized_propagator(lqcd_lattice* L, const lqcd_split* split, const int x_src[4], int field,
                                          double* fact, double* corr, const lqcd_solver_params* params,
                                          lqcd_solver_stats* stats, void* stream) {
  return lqcd_factorized_propagators(L, split, x_src, 1, &field, fact, corr, params, stats, stream);
}

// The two halves of eq. quark_prop_II on their own, so that the systems of a
// factorized propagator can be split between processes that exchange only chi.
extern "C" int lqcd_schur_boundary(lqcd_lattice* L, const lqcd_split* split, int n, const int* field_ids,
                                   const double* psi, double* chi, void* stream) {
  RC(check_lat(L));
  if (!split || n < 1 || !field_ids || !psi || !chi) {
    lq_set_error("schur_boundary: bad arguments");
    return LQCD_EBADARG;
  }
  RC(check_split(L, split, "schur_boundary"));
  for (int k = 0; k < n; k++)
    if (field_ids[k] < 0 || field_ids[k] >= (int)L->fields.size()) {
      lq_set_error("schur_boundary: field index not loaded");
      return LQCD_ENOFIELD;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const lqcd_slab Gb = gamma_bar_of(split);
  std::vector<lqcd_slab> doms(n, Gb);
  BatchStore B;
  RC(B.build(L, n, doms.data(), field_ids, st));
  Pool64 e;
  RC(e.alloc(B.b, 2, st));
  const long long len = (long long)(Gb.t1 - Gb.t0 + 1) * L->S3 * 12;
  std::vector<void*> p(n);
  std::vector<int> ids(n);
  for (int k = 0; k < n; k++) {
    p[k] = (void*)((const double2*)psi + k * len);
    ids[k] = k;
  }
  DBuf d, di;
  RC(upload_ptrs(d, p, st));
  RC(di.alloc(sizeof(int) * n, st));
  CK(cudaMemcpyAsync(di.p, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  RC(lq_nat_to_eo(L, B.b, d.as<const double2*>(), e.v(0), e.v(1), st));
  RC(lq_boundary_chi(L, B.b, di.as<int>(), split->gamma.t1, e.v(0), e.v(1), (double2*)chi, st));
  CK(cudaStreamSynchronize(st));
  return 0;
}

extern "C" int lqcd_schur_solve(lqcd_lattice* L, const lqcd_split* split, int n, const int* field_ids,
                                const double* chi, double* fact_gs, const lqcd_solver_params* params,
                                lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (!split || n < 1 || !field_ids || !chi || !fact_gs) {
    lq_set_error("schur_solve: bad arguments");
    return LQCD_EBADARG;
  }
  RC(check_split(L, split, "schur_solve"));
  for (int k = 0; k < n; k++)
    if (field_ids[k] < 0 || field_ids[k] >= (int)L->fields.size()) {
      lq_set_error("schur_solve: field index not loaded");
      return LQCD_ENOFIELD;
    }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  const lqcd_slab Gs = split->gamma_star;
  const int g1 = split->gamma.t1;
  const long long len = (long long)(Gs.t1 - Gs.t0 + 1) * L->S3 * 12;
  std::vector<SysSpec> sp(n);
  for (int k = 0; k < n; k++) {
    sp[k] = SysSpec{Gs, field_ids[k], 0, 0, make_int4(0, 0, 0, 0)};
    sp[k].out = k;
  }
  FillFn fill = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    SrcArrays s;
    RC(s.upload(sp, k0, B.b.nsys, st));
    return lq_chi_to_eo(L, B.b, s.outs.as<int>(), g1, (const double2*)chi, be, bo, st);
  };
  SinkFn sink = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((double2*)fact_gs + (k0 + q) * len);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), -1.0, st);
  };
  SolveOut o;
  RC(solve_waves(L, sp, false, prm, fill, sink, o, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats)
    for (int k = 0; k < n; k++) fill_stats(o, k, 1, secs, &stats[k]);
  int w = worst_status(o);
  if (w) lq_set_error("schur_solve: some systems did not reach the tolerance");
  return w;
}

extern "C" int lqcd_point_propagators(lqcd_lattice* L, int n_sys, const lqcd_slab* doms, const int* field_ids,
                                      const int* x_src, const int* cols, double* sol,
                                      const lqcd_solver_params* params, lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (n_sys < 1 || !doms || !field_ids || !x_src || !cols || !sol) {
    lq_set_error("point_propagators: bad arguments");
    return LQCD_EBADARG;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  std::vector<SysSpec> sp(n_sys);
  std::vector<long long> goff(n_sys + 1, 0);
  for (int k = 0; k < n_sys; k++) {
    const int* x = x_src + 4 * k;
    if (cols[k] < 0 || cols[k] > 11 || x[0] < doms[k].t0 || x[0] > doms[k].t1 || x[1] < 0 || x[1] >= L->dims[1] ||
        x[2] < 0 || x[2] >= L->dims[2] || x[3] < 0 || x[3] >= L->dims[3]) {
      lq_set_error("point_propagators: source " + std::to_string(k) + " outside its slab or bad column");
      return LQCD_EBADARG;
    }
    sp[k] = SysSpec{doms[k], field_ids[k], 0, cols[k], make_int4(x[0], x[1], x[2], x[3])};
    const long long len = doms[k].t1 >= doms[k].t0 ? (long long)(doms[k].t1 - doms[k].t0 + 1) * L->S3 : 0;
    goff[k + 1] = goff[k] + len;
  }
  FillFn fill = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    SrcArrays s;
    RC(s.upload(sp, k0, B.b.nsys, st));
    return lq_point_source(L, B.b, s.cols.as<int>(), s.xsrc.as<int4>(), be, bo, st);
  };
  SinkFn sink = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((double2*)sol + goff[k0 + q] * 12);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), 1.0, st);
  };
  SolveOut o;
  RC(solve_waves(L, sp, false, prm, fill, sink, o, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats)
    for (int k = 0; k < n_sys; k++) fill_stats(o, k, 1, secs, &stats[k]);
  int w = worst_status(o);
  if (w) lq_set_error("point_propagators: some systems did not reach the tolerance");
  return w;
}

extern "C" int lqcd_link_force(lqcd_lattice* L, const lqcd_slab* dom, int field, const double* phi, double* force,
                               double* action, const lqcd_solver_params* params, lqcd_solver_stats* stats,
                               void* stream) {
  RC(check_lat(L));
  if (!phi) {
    lq_set_error("link_force: null argument");
    return LQCD_EBADARG;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_slab d = dom ? *dom : lqcd_slab{0, L->dims[0] - 1};
  lqcd_solver_params prm = default_params(params);
  BatchStore B;
  RC(B.build(L, 1, &d, &field, st));
  const Batch& b = B.b;
  Pool64 e;
  RC(e.alloc(b, 6, st));  // phi_e, phi_o, Y_e, Y_o, X_e, X_o
  DBuf ptr;
  RC(ptr.alloc(sizeof(void*), st));
  const double2* srcp = (const double2*)phi;
  CK(cudaMemcpyAsync(ptr.p, &srcp, sizeof(void*), cudaMemcpyHostToDevice, st));
  RC(lq_nat_to_eo(L, b, ptr.as<const double2*>(), e.v(0), e.v(1), st));
  SolveOut oy, ox;
  RC(solve_core(L, B, true, prm, e.v(0), e.v(1), e.v(2), e.v(3), oy, st));   // D^dag Y = phi
  if (force) RC(solve_core(L, B, false, prm, e.v(2), e.v(3), e.v(4), e.v(5), ox, st));  // D X = Y
  // S = |Y|^2
  std::fill(B.h_active.begin(), B.h_active.end(), 1);
  RC(B.push_active(st));
  double S = 0;
  for (int par = 0; par < 2; par++) {
    RC(lq_norm2_64(b, e.v(2 + par), st));
    RC(lq_finalize(lq::FIN_NORM, b, 0, 0, 12, st));
    RC(B.pull_sc(st));
    S += B.h_sc[0].rr;
  }
  if (action) *action = S;
  if (!force) {  // action only: S = |Y|^2 needs the D^dag solve alone
    CK(cudaStreamSynchronize(st));
    if (stats) {
      fill_stats(oy, 0, 1, now_s() - t_start, &stats[0]);
      memset(&stats[1], 0, sizeof(lqcd_solver_stats));
    }
    int w = worst_status(oy);
    if (w) lq_set_error("link_force: the D^dag solve did not reach the tolerance");
    return w;
  }
  // natural full-lattice X, Y (zero outside the slab)
  const long long V = L->V;
  DBuf Xn, Yn;
  RC(Xn.alloc(sizeof(double2) * (size_t)V * 12, st));
  RC(Yn.alloc(sizeof(double2) * (size_t)V * 12, st));
  CK(cudaMemsetAsync(Xn.p, 0, sizeof(double2) * (size_t)V * 12, st));
  CK(cudaMemsetAsync(Yn.p, 0, sizeof(double2) * (size_t)V * 12, st));
  double2* dx = Xn.as<double2>() + (size_t)d.t0 * L->S3 * 12;
  CK(cudaMemcpyAsync(ptr.p, &dx, sizeof(void*), cudaMemcpyHostToDevice, st));
  RC(lq_eo_to_nat(L, b, e.v(4), e.v(5), ptr.as<double2* const>(), 1.0, st));
  DBuf ptr2;
  RC(ptr2.alloc(sizeof(void*), st));
  double2* dy = Yn.as<double2>() + (size_t)d.t0 * L->S3 * 12;
  CK(cudaMemcpyAsync(ptr2.p, &dy, sizeof(void*), cudaMemcpyHostToDevice, st));
  RC(lq_eo_to_nat(L, b, e.v(2), e.v(3), ptr2.as<double2* const>(), 1.0, st));
  RC(lq_force(L, field, d, Xn.as<double2>(), Yn.as<double2>(), force, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats) {
    fill_stats(oy, 0, 1, secs, &stats[0]);
    fill_stats(ox, 0, 1, secs, &stats[1]);
  }
  int w = worst_status(oy);
  if (!w) w = worst_status(ox);
  if (w) lq_set_error("link_force: a solve did not reach the tolerance");
  return w;
}

// Sec. 5 eq. stochastic_estimator: per source i and slab d, solve
// D_L psi = g5 eta_i, apply (kappa D_hop)^8 on the slab and contract with
// eta_i per time slice.  Systems are ordered source-major (k = i * n_doms + d).
extern "C" int lqcd_disconnected_trace(lqcd_lattice* L, int n_doms, const lqcd_slab* doms, int field, int n_src,
                                       const double* eta, double* trace, double* mean,
                                       const lqcd_solver_params* params, lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  const int T = L->dims[0];
  if (n_doms < 1 || n_src < 1 || !doms || !eta || !trace) {
    lq_set_error("disconnected_trace: bad arguments");
    return LQCD_EBADARG;
  }
  if (L->csw != 0.0) {
    lq_set_error("disconnected_trace: the (kappa D_hop)^8 estimator needs the Wilson operator (c_sw = 0)");
    return LQCD_EBADARG;
  }
  for (int d = 0; d < n_doms; d++)
    if (doms[d].t0 < 0 || doms[d].t1 < doms[d].t0 || doms[d].t1 >= T) {
      lq_set_error("disconnected_trace: slab " + std::to_string(d) + " outside the lattice or empty");
      return LQCD_EBADARG;
    }
  if (field < 0 || field >= (int)L->fields.size()) {
    lq_set_error("disconnected_trace: field index not loaded");
    return LQCD_ENOFIELD;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  const long long V = L->V, S3 = L->S3;
  const long long per_src = (long long)n_doms * T;
  CK(cudaMemsetAsync(trace, 0, sizeof(double2) * (size_t)(n_src * per_src), st));
  std::vector<SysSpec> sp;
  for (int i = 0; i < n_src; i++)
    for (int d = 0; d < n_doms; d++) sp.push_back(SysSpec{doms[d], field, d, i, make_int4(0, 0, 0, 0)});
  const double2* eta2 = (const double2*)eta;
  FillFn fill = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++)
      p[q] = (void*)(eta2 + (size_t)sp[k0 + q].col * V * 12 + (size_t)sp[k0 + q].dom.t0 * S3 * 12);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_nat_to_eo_g5(L, B.b, d.as<const double2*>(), be, bo, st);
  };
  SinkFn sink = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    Batch b = B.b;
    b.active = nullptr;  // every system, converged or not
    Pool64 h;
    RC(h.alloc(b, 4, st));
    // ping-pong (x -> a -> b -> a ...): eight applications of kappa D_hop
    const double2* ie = xe;
    const double2* io = xo;
    for (int n = 0; n < 8; n++) {
      double2* oe = h.v(n & 1 ? 2 : 0);
      double2* oo = h.v(n & 1 ? 3 : 1);
      RC(lq_hop_kappa(L, b, 0, io, oe, st));
      RC(lq_hop_kappa(L, b, 1, ie, oo, st));
      ie = oe;
      io = oo;
    }
    std::vector<void*> p(b.nsys);
    std::vector<int> slot(b.nsys);
    for (int q = 0; q < b.nsys; q++) {
      p[q] = (void*)(eta2 + (size_t)sp[k0 + q].col * V * 12);
      slot[q] = sp[k0 + q].col * n_doms + sp[k0 + q].role;
    }
    DBuf d, ds;
    RC(upload_ptrs(d, p, st));
    RC(ds.alloc(sizeof(int) * slot.size(), st));
    CK(cudaMemcpyAsync(ds.p, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice, st));
    return lq_slice_dot(L, b, d.as<const double2*>(), ie, io, ds.as<int>(), (double2*)trace, st);
  };
  SolveOut o;
  RC(solve_waves(L, sp, false, prm, fill, sink, o, st));
  if (mean) RC(lq_mean_sources((const double2*)trace, n_src, per_src, (double2*)mean, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats)
    for (int d = 0; d < n_doms; d++) {
      SolveOut od;
      for (int i = 0; i < n_src; i++) {
        const int k = i * n_doms + d;
        od.iters.push_back(o.iters[k]);
        od.cycles.push_back(o.cycles[k]);
        od.status.push_back(o.status[k]);
        od.res.push_back(o.res[k]);
      }
      fill_stats(od, 0, n_src, secs, &stats[d]);
    }
  int w = worst_status(o);
  if (w) lq_set_error("disconnected_trace: some solves did not reach the tolerance");
  return w;
}

// ------------------------------------------------ quark-line projection
namespace {

// Gamma = 0..g1, Gamma* = g1+1..T-1, DeltaGamma = g1+1..d1 (d1 < T-1) or empty.
int check_split(const lqcd_lattice* L, const lqcd_split* split, const char* who) {
  const int T = L->dims[0];
  const lqcd_slab G = split->gamma, Gs = split->gamma_star, Dl = split->delta;
  const bool has_delta = Dl.t1 >= Dl.t0;
  if (G.t0 != 0 || G.t1 < 0 || Gs.t0 != G.t1 + 1 || Gs.t1 != T - 1 ||
      (has_delta && (Dl.t0 != G.t1 + 1 || Dl.t1 >= T - 1))) {
    lq_set_error(std::string(who) + ": need Gamma = 0..g1, Gamma* = g1+1..T-1, DeltaGamma = g1+1..d1 (d1 < T-1)");
    return LQCD_EBADARG;
  }
  return 0;
}

lqcd_slab gamma_bar_of(const lqcd_split* split) {
  const bool has_delta = split->delta.t1 >= split->delta.t0;
  return lqcd_slab{0, has_delta ? split->delta.t1 : split->gamma.t1};
}

void merge_stats(const SolveOut& o, double secs, lqcd_solver_stats* acc, bool first) {
  lqcd_solver_stats s;
  fill_stats(o, 0, (int)o.iters.size(), secs, &s);
  if (first) {
    *acc = s;
    return;
  }
  acc->iters = std::max(acc->iters, s.iters);
  acc->cycles = std::max(acc->cycles, s.cycles);
  acc->true_residual = std::max(acc->true_residual, s.true_residual);
  if (acc->status == 0) acc->status = s.status;
  acc->seconds = secs;
}

}  // namespace

// Sec. 6: projection vectors on the time slice g1 from n_iter inverse
// iterations of D_L, L = dom, each followed by an orthonormalisation; then
// phi = orthonormalise(P_+ V|_{g1}).
extern "C" int lqcd_boundary_modes(lqcd_lattice* L, const lqcd_slab* dom, int g1, int field, int n_modes, int n_iter,
                                   const double* v0, double* phi, const lqcd_solver_params* params,
                                   lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (!dom || !v0 || !phi || n_iter < 0 || dom->t0 < 0 || dom->t1 < dom->t0 || dom->t1 >= L->dims[0] ||
      g1 < dom->t0 || g1 > dom->t1) {
    lq_set_error("boundary_modes: bad arguments (need a slab inside the lattice containing slice g1)");
    return LQCD_EBADARG;
  }
  if (n_modes < 1 || n_modes > 1024 || (long long)n_modes > 6 * L->S3) {
    lq_set_error("boundary_modes: need 1 <= n_modes <= min(1024, 6 L1 L2 L3)");
    return LQCD_EBADARG;
  }
  if (field < 0 || field >= (int)L->fields.size()) {
    lq_set_error("boundary_modes: field index not loaded");
    return LQCD_ENOFIELD;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  const int N = n_modes;
  std::vector<lqcd_slab> doms(N, *dom);
  std::vector<int> fields(N, field);
  BatchStore A;
  RC(A.build(L, N, doms.data(), fields.data(), st));
  const long long n = A.h_sys[0].n;  // sites per parity of one system
  const long long words = 12 * n;    // one system's block in an even or odd pool
  Pool64 P;
  RC(P.alloc(A.b, 4, st));  // V_e, V_o, T_e, T_o
  double2 *Ve = P.v(0), *Vo = P.v(1), *Te = P.v(2), *To = P.v(3);
  {
    const long long len = (long long)(dom->t1 - dom->t0 + 1) * L->S3 * 12;
    std::vector<void*> p(N);
    for (int k = 0; k < N; k++) p[k] = (void*)((const double2*)v0 + k * len);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    RC(lq_nat_to_eo(L, A.b, d.as<const double2*>(), Ve, Vo, st));
  }
  ColMat V, Tm;
  V.nseg = Tm.nseg = 2;
  V.ncol = Tm.ncol = N;
  V.p[0] = Ve;
  V.p[1] = Vo;
  Tm.p[0] = Te;
  Tm.p[1] = To;
  for (int s = 0; s < 2; s++) V.ld[s] = V.rows[s] = Tm.ld[s] = Tm.rows[s] = words;
  std::vector<SysSpec> sp(N);
  for (int k = 0; k < N; k++) sp[k] = SysSpec{*dom, field, 0, k, make_int4(0, 0, 0, 0)};
  // a wave's pools hold its systems back to back, as V does: plain copies
  FillFn fill = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    const size_t bytes = sizeof(double2) * (size_t)(B.b.nsys * words);
    CK(cudaMemcpyAsync(be, Ve + k0 * words, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(bo, Vo + k0 * words, bytes, cudaMemcpyDeviceToDevice, st));
    return 0;
  };
  SinkFn sink = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    const size_t bytes = sizeof(double2) * (size_t)(B.b.nsys * words);
    CK(cudaMemcpyAsync(Ve + k0 * words, xe, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Vo + k0 * words, xo, bytes, cudaMemcpyDeviceToDevice, st));
    return 0;
  };
  lqcd_solver_stats acc{};
  int worst = 0;
  for (int it = 0; it < n_iter; it++) {
    SolveOut o;
    RC(solve_waves(L, sp, false, prm, fill, sink, o, st));
    merge_stats(o, now_s() - t_start, &acc, it == 0);
    if (!worst) worst = worst_status(o);
    RC(lq_orthonormalize(V, Tm, st));
  }
  RC(lq_slice_plus(L, A.b, g1, Ve, Vo, (double2*)phi, st));
  ColMat F, Ft;
  F.nseg = Ft.nseg = 1;
  F.ncol = Ft.ncol = N;
  F.p[0] = (double2*)phi;
  Ft.p[0] = Te;  // T_e and T_o are adjacent: 2 N 12 n = N 12 S3 (t1 - t0 + 1) entries
  F.ld[0] = F.rows[0] = Ft.ld[0] = Ft.rows[0] = 12 * L->S3;
  RC(lq_orthonormalize(F, Ft, st));
  CK(cudaStreamSynchronize(st));
  if (stats) {
    *stats = acc;
    stats->seconds = now_s() - t_start;
  }
  if (worst) lq_set_error("boundary_modes: some solves did not reach the tolerance");
  return worst;
}

// Sec. 3.3 eq. quark_prop_II_proj: xi_i = D_Gammabar^{-dag} phi_i and
// eta_i = D_Gamma*^{-1} D_dGamma* phi_i for phi_i on the last slice of Gamma.
extern "C" int lqcd_projected_factors(lqcd_lattice* L, const lqcd_split* split, int field, int n_modes,
                                      const double* phi, double* xi, double* eta, const lqcd_solver_params* params,
                                      lqcd_solver_stats* stats, void* stream) {
  RC(check_lat(L));
  if (!split || !phi || !xi || !eta || n_modes < 1) {
    lq_set_error("projected_factors: bad arguments");
    return LQCD_EBADARG;
  }
  RC(check_split(L, split, "projected_factors"));
  if (L->bc != LQCD_BC_OPEN) {
    lq_set_error("projected_factors: needs the open time boundary (the boundary block is one time hop)");
    return LQCD_EBADARG;
  }
  if (field < 0 || field >= (int)L->fields.size()) {
    lq_set_error("projected_factors: field index not loaded");
    return LQCD_ENOFIELD;
  }
  const double t_start = now_s();
  cudaStream_t st = (cudaStream_t)stream;
  lqcd_solver_params prm = default_params(params);
  const int N = n_modes;
  const int g1 = split->gamma.t1;
  const lqcd_slab Gb = gamma_bar_of(split), Gs = split->gamma_star;
  const long long S3 = L->S3;
  const long long len_gb = (long long)(Gb.t1 - Gb.t0 + 1) * S3 * 12, len_gs = (long long)(Gs.t1 - Gs.t0 + 1) * S3 * 12;
  DBuf ids;
  {
    std::vector<int> h(N);
    for (int k = 0; k < N; k++) h[k] = k;
    RC(ids.alloc(sizeof(int) * N, st));
    CK(cudaMemcpyAsync(ids.p, h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  }
  const double2* phi2 = (const double2*)phi;
  // xi: dagger solves on Gammabar from phi on slice g1
  std::vector<SysSpec> sa(N), sb(N);
  for (int k = 0; k < N; k++) {
    sa[k] = SysSpec{Gb, field, 0, k, make_int4(0, 0, 0, 0)};
    sb[k] = SysSpec{Gs, field, 0, k, make_int4(0, 0, 0, 0)};
  }
  FillFn fill_a = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    return lq_slice_source(L, B.b, ids.as<int>() + k0, g1, phi2, be, bo, st);
  };
  SinkFn sink_a = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((double2*)xi + (k0 + q) * len_gb);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), 1.0, st);
  };
  SolveOut oa;
  RC(solve_waves(L, sa, true, prm, fill_a, sink_a, oa, st));
  const double t_a = now_s() - t_start;
  // chi_i = D_dGamma* phi_i (slot 0: the time hop from slice g1 to g1+1)
  DBuf chi;
  RC(chi.alloc(sizeof(double2) * (size_t)N * 2 * S3 * 12, st));
  {
    std::vector<lqcd_slab> d1(N, lqcd_slab{g1, g1});
    std::vector<int> f1(N, field);
    BatchStore P;
    RC(P.build(L, N, d1.data(), f1.data(), st));
    Pool64 pv;
    RC(pv.alloc(P.b, 2, st));
    RC(lq_slice_source(L, P.b, ids.as<int>(), g1, phi2, pv.v(0), pv.v(1), st));
    RC(lq_boundary_chi(L, P.b, ids.as<int>(), g1, pv.v(0), pv.v(1), chi.as<double2>(), st));
  }
  FillFn fill_b = [&](BatchStore& B, int k0, double2* be, double2* bo) -> int {
    return lq_chi_to_eo(L, B.b, ids.as<int>() + k0, g1, chi.as<double2>(), be, bo, st);
  };
  SinkFn sink_b = [&](BatchStore& B, int k0, const double2* xe, const double2* xo) -> int {
    std::vector<void*> p(B.b.nsys);
    for (int q = 0; q < B.b.nsys; q++) p[q] = (void*)((double2*)eta + (k0 + q) * len_gs);
    DBuf d;
    RC(upload_ptrs(d, p, st));
    return lq_eo_to_nat(L, B.b, xe, xo, d.as<double2* const>(), 1.0, st);
  };
  SolveOut ob;
  RC(solve_waves(L, sb, false, prm, fill_b, sink_b, ob, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  if (stats) {
    fill_stats(oa, 0, N, t_a, &stats[0]);
    fill_stats(ob, 0, N, secs, &stats[1]);
  }
  int w = worst_status(oa);
  if (!w) w = worst_status(ob);
  if (w) lq_set_error("projected_factors: some solves did not reach the tolerance");
  return w;
}

// Case II of eq. quark_prop_II_proj on Gamma* for the 12 point sources at x:
// fact[b][y][a] = -sum_i eta_i(y)[a] conj(xi_i(x)[b]).
extern "C" int lqcd_projected_propagator(lqcd_lattice* L, const lqcd_split* split, int n_modes, const double* xi,
                                         const double* eta, const int x_src[4], double* fact, void* stream) {
  RC(check_lat(L));
  if (!split || !xi || !eta || !x_src || !fact || n_modes < 1 || n_modes > 1024) {
    lq_set_error("projected_propagator: bad arguments (1 <= n_modes <= 1024)");
    return LQCD_EBADARG;
  }
  RC(check_split(L, split, "projected_propagator"));
  if (x_src[0] < split->gamma.t0 || x_src[0] > split->gamma.t1) {
    lq_set_error("projected_propagator: the source must lie in Gamma");
    return LQCD_EBADARG;
  }
  for (int k = 1; k < 4; k++)
    if (x_src[k] < 0 || x_src[k] >= L->dims[k]) {
      lq_set_error("projected_propagator: source outside the lattice");
      return LQCD_EBADARG;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const lqcd_slab Gb = gamma_bar_of(split), Gs = split->gamma_star;
  const long long S3 = L->S3;
  const long long xnat = (((long long)x_src[0] * L->dims[1] + x_src[1]) * L->dims[2] + x_src[2]) * L->dims[3] + x_src[3];
  RC(lq_proj_prop(L, n_modes, (long long)(Gb.t1 - Gb.t0 + 1) * S3, xnat - (long long)Gb.t0 * S3,
                  (const double2*)xi, (long long)(Gs.t1 - Gs.t0 + 1) * S3, (long long)Gs.t0 * S3,
                  (const double2*)eta, (double2*)fact, st));
  CK(cudaStreamSynchronize(st));
  return 0;
}

// Timing hook: one kernel of the solver's BiCGStab iteration on a batch.
extern "C" int lqcd_stencil_bench(lqcd_lattice* L, int n_sys, const lqcd_slab* doms, const int* field_ids,
                                  int precision, int kernel, int reps, double* ms_per_launch,
                                  double* bytes_per_launch, double* flops_per_launch, void* stream) {
  RC(check_lat(L));
  if (n_sys < 1 || !doms || !field_ids || reps < 1 || (precision != 64 && precision != 32 && precision != 16) ||
      kernel < 0 || kernel > 6) {
    lq_set_error("stencil_bench: bad arguments");
    return LQCD_EBADARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  BatchStore B;
  RC(B.build(L, n_sys, doms, field_ids, st));
  const Batch& b = B.b;
  Pool64 tmp;
  RC(tmp.alloc(b, 2, st));
  RC(lq_fill64(tmp.v(0), b.total * 12, 12345u, st));
  RC(lq_fill64(tmp.v(1), b.total * 12, 67890u, st));
  PoolP q;
  RC(q.alloc(b, precision, kernel >= 4 ? 6 : 4, st));
  RC(lq_convert(64, precision, b, v64(tmp.v(0)), q.v(0), st));
  RC(lq_convert(64, precision, b, v64(tmp.v(1)), q.v(1), st));
  RC(lq_convert(64, precision, b, v64(tmp.v(1)), q.v(3), st));
  if (kernel >= 4) {
    RC(lq_convert(64, precision, b, v64(tmp.v(0)), q.v(4), st));
    RC(lq_convert(64, precision, b, v64(tmp.v(1)), q.v(5), st));
  }
  const bool clov = L->csw != 0.0;
  VecP none;
  B.b.hop_variant = lq_tune_hop(L, B.b, precision, clov, q.v(0), q.v(1), q.v(2), st);
  // the iteration's kernels on the pools q0..q5 (x, y, out, w, and two more for the BLAS passes)
  auto launch = [&]() -> int {
    switch (kernel) {
      case 0:  // out_o = A_oo y_o - 1/4 D_hop x_e
        return lq_hop_lin(precision, false, clov, lq::RED_NONE, L, b, 1, q.v(0), q.v(1), none, none, q.v(2), -0.25,
                          1.0, 0.0, st);
      case 1:  // out_e = A_ee^{-1} D_hop x_o
        return lq_hop_clinv(precision, false, clov, L, b, q.v(0), none, q.v(2), 1.0, 0.0, st);
      case 2:  // v = A_oo p - 1/4 D_hop te, with <r0, v>
        return lq_hop_lin(precision, false, clov, lq::RED_DOT_W, L, b, 1, q.v(0), q.v(1), none, q.v(3), q.v(2),
                          -0.25, 1.0, 0.0, st);
      case 3:  // t = A_oo s - 1/4 D_hop te, with <t, s> and |t|^2
        return lq_hop_lin(precision, false, clov, lq::RED_TS, L, b, 1, q.v(0), q.v(1), none, none, q.v(2), -0.25,
                          1.0, 0.0, st);
      case 4:  // s = r - alpha v
        return lq_bicg_s(precision, b, q.v(0), q.v(1), q.v(2), st);
      case 5:  // x += alpha p + omega s, r = s - omega t, <r0, r>, |r|^2
        return lq_bicg_xr(precision, b, q.v(2), q.v(0), q.v(1), q.v(4), q.v(5), q.v(3), st);
      default:  // p = r + beta (p - omega v)
        return lq_bicg_p(precision, b, q.v(2), q.v(0), q.v(1), st);
    }
  };
  for (int w = 0; w < 3; w++) RC(launch());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; r++) RC(launch());
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // algorithmic bytes: the spinor passes per system site (each vector read or
  // written once), plus 8 links + the clover block per distinct site of each
  // field's slabs for the hop kernels
  const double S = precision == 64 ? 192.0 : precision == 32 ? 96.0 : 52.0;
  const double Lk = precision == 64 ? 144.0 : precision == 32 ? 48.0 : 24.0;
  const double C = clov ? (precision == 64 ? 576.0 : 288.0) : 0.0;
  static const double passes[7] = {3, 2, 4, 3, 3, 7, 4};
  double bytes = 0.0, sites = 0.0;
  std::vector<std::vector<char>> used(L->fields.size(), std::vector<char>(L->dims[0], 0));
  for (int k = 0; k < n_sys; k++) {
    bytes += passes[kernel] * S * (double)B.h_sys[k].n;
    sites += (double)B.h_sys[k].n;
    for (int t = doms[k].t0; t <= doms[k].t1; t++) used[field_ids[k]][t] = 1;
  }
  if (kernel <= 3)
    for (auto& u : used)
      for (char c : u)
        if (c) bytes += (8.0 * Lk + C) * (double)L->S3h;
  // flop per system site: hop 1320, site-diagonal block 504 (clover) or 24, epilogue and reductions
  const double diag = clov ? 504.0 : 24.0;
  const double flop[7] = {1320.0 + diag + 72.0, 1320.0 + diag + 24.0, 1320.0 + diag + 72.0 + 96.0,
                          1320.0 + diag + 72.0 + 144.0, 96.0, 432.0, 192.0};
  const double fl = sites * flop[kernel];
  if (ms_per_launch) *ms_per_launch = ms / reps;
  if (bytes_per_launch) *bytes_per_launch = bytes;
  if (flops_per_launch) *flops_per_launch = fl;
  return 0;
}

extern "C" int lqcd_dslash_bench(lqcd_lattice* L, int n_sys, const lqcd_slab* doms, const int* field_ids,
                                 int precision, int reps, double* ms_per_launch, double* bytes_per_launch,
                                 double* flops_per_launch, void* stream) {
  return lqcd_stencil_bench(L, n_sys, doms, field_ids, precision, 0, reps, ms_per_launch, bytes_per_launch,
                            flops_per_launch, stream);
}
