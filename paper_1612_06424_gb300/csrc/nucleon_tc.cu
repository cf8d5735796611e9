// Nucleon blocks (Sec. 4.2 eq. nucleon_prop_factorized) on the 5th-generation
// tensor cores: the same product as k_nucleon_block in nucleon.cu,
//   B[(i,j)][(k,alpha)] = sum_{x in slice, c} D[(i,j)][(x,c)] S[(x,c)][(k,alpha)],
// D the diquark eps^{abc} s_i^a(x)^T C g5 s_j^b(x), S[(x,c)][(k,alpha)] = s_k(x)[alpha][c],
// written as one real GEMM per tile with tcgen05.mma (kind::tf32, accumulator in TMEM).
//
// Complex to real: with kappa = 2 (x,c) + p (p: real / imaginary part),
//   A[m][kappa]      = (Re D, Im D)[m][(x,c)]                      (D stored as complex pairs),
//   Bt[2n][kappa]    = (Re S, -Im S)[(x,c)][n],  Bt[2n+1][kappa] = (Im S, Re S)[(x,c)][n],
// so that C[m][2n] = Re B and C[m][2n+1] = Im B for C = A Bt^T (both operands K-major).
//
// FP32 accuracy from TF32 tensor cores (three-pass split, Markidis et al. 2018, "NVIDIA
// tensor core programmability, performance & precision"): each FP32 operand value v is split
// into hi = v rounded to the 11 significant bits of TF32 and lo = v - hi (exact in FP32);
// C accumulates hi*hi + hi*lo + lo*hi in FP32, which drops lo*lo (<= 2^-22 |A||B|) and the
// truncation of lo to TF32 by the tensor core (<= 2^-21 |A||B| per product).
//
// Two-level sum, as in k_nucleon_block: the tensor core accumulates 64 sites (16 chunks of 4)
// into one TMEM accumulator, which is then added into FP32 running sums held in a second TMEM
// region; the result is written in FP64.
//
// The fields of the requested slices are first converted once to FP32 (conjugated for the xi
// side) by k_slices_f32, a group of slices at a time (at most about 2 GB of scratch), into an
// array [slice][field][site][12] whose sites are padded to a multiple of 4 with zeros.
//
// One CTA per SM (512 threads, 16 warps): 128 rows (i, j) = 8 i x 16 j of one slice and 128
// complex columns (32 k x 4 alpha) = 256 real columns, so the accumulator fills the 512 TMEM
// columns (256 inner + 256 running sums).  Per chunk of 4 sites (24 real K values, three MMA
// K-steps of 8) all threads stage the 56 spinors of the chunk (FP32, 16-byte loads prefetched
// one chunk ahead) in shared memory; warps 0-7 build the split diquark operand A (128 rows) and
// warps 8-15 the split operand Bt (256 rows) into one of two operand buffers in the canonical
// K-major layout without swizzle, and one thread issues 9 MMAs (3 K-steps x 3 products, each
// M 128 x N 256 x K 8) and commits them to the buffer's mbarrier.  The building of chunk c+1
// overlaps the MMAs of chunk c.
//
// Operand layout (no swizzle, K-major): a core matrix is 8 rows x 16 bytes (4 TF32).  One
// R-row x 8-value operand of one K-step is R/8 row groups x 2 core matrices:
//   byte offset of (row r, value q) = ((r / 8) * 2 + q / 4) * 128 + (r % 8) * 16 + (q % 4) * 4,
// i.e. leading-dimension byte offset (between the two core matrices along K) 128 and
// stride-dimension byte offset (between row groups) 256.  Each operand occupies its own block
// of R * 32 bytes, so every address the descriptor can form lies inside that block.
//
// Every wait on an mbarrier is bounded (about one second of clock cycles); on expiry the CTA
// records the failure in `status`, stops issuing, and still frees its TMEM.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tc_layout.cuh"

using namespace lq;

namespace {

constexpr int TI = TC_TI, TJ = TC_TJ, TK = TC_TK;  // tile: 8 x 16 (i, j) rows, 32 k (128 complex columns)
constexpr int NSLOT = TI + TJ + TK;      // spinors per site of a tile
constexpr int XS = 4;                    // sites per chunk
constexpr int NSTEP = XS * 6 / 8;        // MMA K-steps per chunk (K = 8 TF32 per step)
constexpr int GROUP = 16;                // chunks per inner accumulation (64 sites)
constexpr int NT = 512;
constexpr int MAT_A = 4096;                   // bytes of the 128-row x 8 operand A of one step
constexpr int MAT_B = 8192;                   // bytes of the 256-row x 8 operand Bt of one step
constexpr int STEP = 2 * MAT_A + 2 * MAT_B;   // one K-step: A hi, A lo, Bt hi, Bt lo
constexpr int BUF = NSTEP * STEP;             // one chunk
// FP32 staging per site (tc_stage_index): the 24 (i, j) spinors at a stride of 14 float2
// (16-byte aligned; the 16-byte reads of 8 consecutive j by a quarter warp's A rows on distinct
// banks), then the 32 k spinors at a stride of 12 (16-byte aligned; the (k, alpha) reads of a
// warp's Bt rows on distinct banks)
constexpr int SITE_STG = TC_SITE_STG;  // float2 per site
constexpr int STG = XS * SITE_STG * 8;
constexpr int SMEM = 2 * BUF + STG + 64;      // + 2 mbarriers, the TMEM address and a flag
constexpr int TMEM_COLS = 512;                // inner accumulator (0..255) + running sums (256..511)
constexpr int NPRE = 4;                       // 16-byte staging loads per thread and chunk

// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

LQ_DI uint64_t smem_desc(uint32_t addr) {
  // start address >> 4 (bits 0-13), leading byte offset 128 >> 4 (16-29), stride byte offset
  // 256 >> 4 (32-45), descriptor version 1 (bit 46), base offset 0, no swizzle (61-63 = 0)
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
         (1ull << 46);
}

LQ_DI void split_tf32(float v, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
  lo = v - hi;
}

LQ_DI void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

LQ_DI void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// bounded wait for the completion of the phase with the given parity; false on expiry
LQ_DI bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

LQ_DI void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
LQ_DI void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

LQ_DI void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

LQ_DI void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// s^T C g5 t for colour a of s and b of t (C g5 entries as in nucleon.cu)
LQ_DI float2 cg5_pair_tc(const float2* si, const float2* tj, int a, int b) {
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

// store the hi / lo split of four consecutive K values of row r into K-block beta (0..5) of
// the operand at byte offset `hi_off` of a step (lo at hi_off + mat)
LQ_DI void put4(unsigned char* buf, int hi_off, int mat, int r, int beta, float4 v) {
  float4 h, l;
  split_tf32(v.x, h.x, l.x);
  split_tf32(v.y, h.y, l.y);
  split_tf32(v.z, h.z, l.z);
  split_tf32(v.w, h.w, l.w);
  const int off = (beta >> 1) * STEP + hi_off + tc_operand_offset(r, 4 * (beta & 1));
  *reinterpret_cast<float4*>(buf + off) = h;
  *reinterpret_cast<float4*>(buf + off + mat) = l;
}

// TMEM readout: warp w reads lanes 32 (w % 4) .. + 31 and real columns 64 (w / 4) .. + 63 of
// the inner accumulator and adds them into the running sums (columns + 256).
LQ_DI void fold_group(uint32_t tmem, int warp, bool first) {
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int c0 = 64 * (warp >> 2);
#pragma unroll 1
  for (int q = 0; q < 4; q++) {
    float a[16], s[16];
    tmem_ld16(tmem + lane_base + (uint32_t)(c0 + 16 * q), a);
    if (!first) {
      tmem_ld16(tmem + lane_base + (uint32_t)(256 + c0 + 16 * q), s);
#pragma unroll
      for (int e = 0; e < 16; e++) a[e] += s[e];
    }
    tmem_st16(tmem + lane_base + (uint32_t)(256 + c0 + 16 * q), a);
  }
}

// sf[((ts * n + f) * S3p + x) * 12 + comp] = s[(f * nsite + lo + ts * S3 + x) * 12 + comp] in FP32
// (imaginary part negated for conj), zero for the padding sites x >= S3
__global__ void k_slices_f32(int n, long long nsite, const double2* s, int conj, int S3, int S3p, long long lo,
                             int nts, float2* sf) {
  const long long total = (long long)nts * n * S3p * 12;
  const float cs = conj ? -1.f : 1.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)(e % 12);
    const long long r = e / 12;
    const int x = (int)(r % S3p);
    const long long q = r / S3p;
    const int f = (int)(q % n), ts = (int)(q / n);
    float2 v = make_float2(0.f, 0.f);
    if (x < S3) {
      const double2 d = s[((long long)f * nsite + lo + (long long)ts * S3 + x) * 12 + comp];
      v = make_float2((float)d.x, cs * (float)d.y);
    }
    sf[e] = v;
  }
}

__global__ void __launch_bounds__(NT, 1) k_nucleon_block_tc(int n, int S3p, const float2* sf, int t_base,
                                                             double2* B, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* buf0 = smem;
  float2* stg = reinterpret_cast<float2*>(smem + 2 * BUF);  // [XS][SITE_STG]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * BUF + STG);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + 2 * BUF + STG + 16);
  int* fail = reinterpret_cast<int*>(smem + 2 * BUF + STG + 20);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntj = (n + TJ - 1) / TJ;
  const int i0 = (int)(blockIdx.x / ntj) * TI, j0 = (int)(blockIdx.x % ntj) * TJ;
  const int k0 = blockIdx.y * TK;
  const int ts = blockIdx.z;  // slice within this launch's scratch array
  const int t = t_base + ts;  // slice within the output

  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&bars[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail = 0;
  }
  if (warp == 0) {
    const uint32_t h = (uint32_t)__cvta_generic_to_shared(tmem_holder);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(h), "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_holder;

  // staging loads: thread t moves float4 q = t % 8 (two complex components; q < 6) of site
  // x = (t / 8) % 4 of slots (t / 32) + 16 r, r < NPRE
  const int pq = tid & 7, px = (tid >> 3) & 3, pslot0 = tid >> 5;
  const float4* sf4 = reinterpret_cast<const float4*>(sf);
  long long gbase[NPRE];  // float4 index of (slot, site 0 of the slice), or -1
#pragma unroll
  for (int r = 0; r < NPRE; r++) {
    const int slot = pslot0 + 16 * r;
    const int f = slot < TI ? i0 + slot : (slot < TI + TJ ? j0 + slot - TI : k0 + slot - TI - TJ);
    gbase[r] = (pq < 6 && slot < NSLOT && f < n) ? (((long long)ts * n + f) * S3p + px) * 6 + pq : -1;
  }
  float4 pre[NPRE];
  auto prefetch = [&](int x0) {
#pragma unroll
    for (int r = 0; r < NPRE; r++)
      pre[r] = gbase[r] >= 0 ? sf4[gbase[r] + (long long)x0 * 6] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  const int nchunk = S3p / XS;
  prefetch(0);
  bool ok = true;
  int issued = -1;  // last chunk whose MMAs were committed
  for (int c = 0; c < nchunk; c++) {
    const int b = c & 1;
    unsigned char* buf = buf0 + b * BUF;
    // staging <- chunk c; then prefetch chunk c + 1
#pragma unroll
    for (int r = 0; r < NPRE; r++) {
      const int slot = pslot0 + 16 * r;
      if (pq < 6 && slot < NSLOT) {
        *reinterpret_cast<float4*>(&stg[tc_stage_index(px, slot, 2 * pq)]) = pre[r];
      }
    }
    if (c + 1 < nchunk) prefetch((c + 1) * XS);
    // the MMAs of chunk c - 2 read this operand buffer: wait for them
    if (c >= 2 && !mbar_wait(b ? bar1 : bar0, (uint32_t)(((c - 2) >> 1) & 1))) *fail = 1;
    __syncthreads();
    if (*fail) {
      ok = false;
      break;
    }
    if (warp < 8) {
      // A: row m = 16 ii + jj, sites 2h, 2h + 1 (h = tid / 128): K values 12h .. 12h + 11
      const int m = tid & 127, h = tid >> 7;
      const int ii = m >> 4, jj = m & 15;
      float v[12];
#pragma unroll
      for (int q = 0; q < 2; q++) {
        const int x = 2 * h + q;
        const float4* u = reinterpret_cast<const float4*>(&stg[tc_stage_index(x, ii, 0)]);
        const float4* w = reinterpret_cast<const float4*>(&stg[tc_stage_index(x, TI + jj, 0)]);
        float2 uu[12], ww[12];
#pragma unroll
        for (int e = 0; e < 6; e++) {
          const float4 a4 = u[e], b4 = w[e];
          uu[2 * e] = make_float2(a4.x, a4.y);
          uu[2 * e + 1] = make_float2(a4.z, a4.w);
          ww[2 * e] = make_float2(b4.x, b4.y);
          ww[2 * e + 1] = make_float2(b4.z, b4.w);
        }
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {
          const int a = (cc + 1) % 3, bb = (cc + 2) % 3;
          const float2 p = cg5_pair_tc(uu, ww, a, bb), mm = cg5_pair_tc(uu, ww, bb, a);
          v[6 * q + 2 * cc] = p.x - mm.x;
          v[6 * q + 2 * cc + 1] = p.y - mm.y;
        }
      }
#pragma unroll
      for (int q = 0; q < 3; q++)
        put4(buf, 0, MAT_A, m, 3 * h + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    } else {
      // Bt: rows 2 nc (Re S, -Im S) and 2 nc + 1 (Im S, Re S), nc = 4 kk + alpha; K-block
      // beta holds the (x, c) pairs 2 beta and 2 beta + 1 (x = pair / 3, c = pair % 3)
      const int u0 = tid - 256;
#pragma unroll
      for (int r = 0; r < 6; r++) {
        const int e = u0 + 256 * r;
        const int row = e & 255, beta = e >> 8;
        const int nc = row >> 1, q = row & 1;
        const int kk = nc >> 2, al = nc & 3;
        float vv[4];
#pragma unroll
        for (int uu = 0; uu < 2; uu++) {
          const int pr = 2 * beta + uu;
          const int x = pr / 3, cc = pr % 3;
          const float2 sv = stg[tc_stage_index(x, TI + TJ + kk, al * 3 + cc)];
          vv[2 * uu] = q ? sv.y : sv.x;
          vv[2 * uu + 1] = q ? sv.x : -sv.y;
        }
        put4(buf, 2 * MAT_A, MAT_B, row, beta, make_float4(vv[0], vv[1], vv[2], vv[3]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
      for (int st = 0; st < NSTEP; st++) {
        const uint32_t sb = base + st * STEP;
        const uint64_t ah = smem_desc(sb), al = smem_desc(sb + MAT_A);
        const uint64_t bh = smem_desc(sb + 2 * MAT_A), bl = smem_desc(sb + 2 * MAT_A + MAT_B);
        const uint32_t acc = (c % GROUP != 0 || st > 0) ? 1u : 0u;
        mma_tf32(tmem, ah, bh, acc);
        mma_tf32(tmem, ah, bl, 1u);
        mma_tf32(tmem, al, bh, 1u);
      }
      mma_commit(b ? bar1 : bar0);
    }
    issued = c;
    // end of an inner group: wait for its MMAs, fold the accumulator into the running sums
    if (c % GROUP == GROUP - 1 || c == nchunk - 1) {
      if (!mbar_wait(b ? bar1 : bar0, (uint32_t)((c >> 1) & 1))) *fail = 1;
      __syncthreads();
      if (*fail) {
        ok = false;
        break;
      }
      fence_after();
      fold_group(tmem, warp, c < GROUP);
      fence_before();
      __syncthreads();
    }
  }

  if (ok) {
    // running sums -> B (FP64): thread row m = 32 (warp % 4) + lane, complex columns
    // 32 (warp / 4) .. + 31 of the tile
    const int m = 32 * (warp & 3) + (tid & 31);
    const int i = i0 + (m >> 4), j = j0 + (m & 15);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    fence_after();
#pragma unroll 1
    for (int q = 0; q < 4; q++) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)(256 + 64 * (warp >> 2) + 16 * q), v);
      if (i < n && j < n) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int nc = 32 * (warp >> 2) + 8 * q + e;
          const int k = k0 + (nc >> 2), al = nc & 3;
          if (k < n)
            B[((((long long)t * n + i) * n + j) * n + k) * 4 + al] = make_double2((double)v[2 * e], (double)v[2 * e + 1]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(status, 1);
    // give the MMAs still in flight a bounded chance to finish before the TMEM is freed
    if (issued >= 0) mbar_wait((issued & 1) ? bar1 : bar0, (uint32_t)((issued >> 1) & 1));
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

int lq_nucleon_blocks_tc(int n, long long nsite, const double2* s, int conj, int S3, long long lo0, int n_t,
                         double2* B, cudaStream_t st) {
  static std::mutex mu;
  static std::vector<int> opted;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    lq_set_error("nucleon_blocks: no current device");
    return LQCD_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(opted.begin(), opted.end(), dev) == opted.end()) {
      if (cudaFuncSetAttribute(k_nucleon_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess) {
        cudaGetLastError();
        lq_set_error("nucleon_blocks: shared-memory opt-in failed");
        return LQCD_ECUDA;
      }
      opted.push_back(dev);
    }
  }
  // FP32 scratch of the fields on a group of slices (at most about 2 GB)
  const int S3p = (S3 + XS - 1) / XS * XS;
  const long long slice_words = (long long)n * S3p * 12;  // float2 per slice
  const int g = (int)std::max(1LL, std::min((long long)n_t, (2LL << 30) / (slice_words * 8)));
  int* status = nullptr;
  float2* sf = nullptr;
  if (cudaMallocAsync(&status, sizeof(int), st) != cudaSuccess ||
      cudaMallocAsync(&sf, sizeof(float2) * slice_words * g, st) != cudaSuccess) {
    cudaGetLastError();
    if (status) cudaFreeAsync(status, st);
    lq_set_error("nucleon_blocks: device allocation failed");
    return LQCD_ENOMEM;
  }
  cudaMemsetAsync(status, 0, sizeof(int), st);
  const int nti = (n + TI - 1) / TI, ntj = (n + TJ - 1) / TJ, ntk = (n + TK - 1) / TK;
  for (int t0 = 0; t0 < n_t; t0 += g) {
    const int nts = std::min(g, n_t - t0);
    k_slices_f32<<<152 * 8, 256, 0, st>>>(n, nsite, s, conj, S3, S3p, lo0 + (long long)t0 * S3, nts, sf);
    lq_count_launch();
    k_nucleon_block_tc<<<dim3((unsigned)(nti * ntj), (unsigned)ntk, (unsigned)nts), NT, SMEM, st>>>(n, S3p, sf, t0,
                                                                                                   B, status);
    lq_count_launch();
  }
  cudaError_t e = cudaGetLastError();
  int h_status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(sf, st);
  cudaFreeAsync(status, st);
  if (e != cudaSuccess) {
    lq_set_error(std::string("nucleon_blocks (tensor cores): ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  if (h_status != 0) {
    lq_set_error("nucleon_blocks (tensor cores): a wait for the tensor-core pipeline timed out");
    return LQCD_ECUDA;
  }
  return 0;
}
