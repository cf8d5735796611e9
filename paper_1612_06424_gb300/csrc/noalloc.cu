// lqcd_dslash_noalloc: the FP64 Dirac operator of lqcd_dslash without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: an application
// that hands this library a share of a GPU whose memory is owned by its own
// allocator (so a cudaMalloc outside that allocator fails or fragments the
// pool), or code on a latency-critical path where an allocation's cost or
// possible failure is not acceptable.  For them this entry point keeps its
// scratch -- the even / odd copies of the input and output and the small
// descriptor tables the kernels read -- in one file-scope device array of
// LQCD_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that
// array until the process exits.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LQCD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    lq_set_error("dslash_noalloc: no usable current CUDA device");
    return LQCD_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      lq_set_error(std::string("dslash_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return LQCD_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return 0;
}

// Writes the system descriptor and the in / out pointer table into the
// scratch array.  They arrive as by-value kernel arguments, which the launch
// copies, so no host buffer has to outlive the call.
__global__ void k_noalloc_setup(lq::SysDesc s, const void* in, void* out, lq::SysDesc* d_sys, void** d_ptr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *d_sys = s;
    d_ptr[0] = const_cast<void*>(in);
    d_ptr[1] = out;
  }
}

}  // namespace

extern "C" int lqcd_dslash_noalloc(lqcd_lattice* L, int field, const lqcd_slab* dom, int dagger, const double* in,
                                   double* out, void* stream) {
  if (!L || !in || !out) {
    lq_set_error("dslash_noalloc: null argument");
    return LQCD_EBADARG;
  }
  const lqcd_slab d = dom ? *dom : lqcd_slab{0, L->dims[0] - 1};
  if (d.t0 < 0 || d.t1 >= L->dims[0] || d.t0 > d.t1) {
    lq_set_error("dslash_noalloc: slab out of range");
    return LQCD_EBADARG;
  }
  if (field < 0 || field >= (int)L->fields.size()) {
    lq_set_error("dslash_noalloc: field index not loaded");
    return LQCD_ENOFIELD;
  }
  // scratch layout: [descriptor 256 B][pointer table 256 B][in_e][in_o][out_e][out_o]
  const long long n = (long long)(d.t1 - d.t0 + 1) * L->S3h;  // sites per parity
  const size_t vec_bytes = (size_t)n * 12 * sizeof(double2);
  const size_t need = 512 + 4 * vec_bytes;
  if (need > (size_t)LQCD_NOALLOC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "dslash_noalloc: slab of %lld sites needs %zu bytes of scratch, more than the %d-byte maximum "
             "(use lqcd_dslash)",
             2 * n, need, (int)LQCD_NOALLOC_SCRATCH_BYTES);
    lq_set_error(msg);
    return LQCD_EBADARG;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* b8 = (unsigned char*)base;
  lq::SysDesc* d_sys = (lq::SysDesc*)b8;
  void** d_ptr = (void**)(b8 + 256);
  double2* in_e = (double2*)(b8 + 512);
  double2* in_o = in_e + n * 12;
  double2* out_e = in_o + n * 12;
  double2* out_o = out_e + n * 12;

  lq::SysDesc s{};
  s.field = field;
  s.t0 = d.t0;
  s.t1 = d.t1;
  s.wrap = (d.t0 == 0 && d.t1 == L->dims[0] - 1 && L->bc != LQCD_BC_OPEN) ? 1 : 0;
  s.tsign = L->bc == LQCD_BC_ANTIPERIODIC ? -1.f : 1.f;
  s.n = (int)n;
  s.cb0 = (int)(d.t0 * L->S3h);
  s.off = 0;
  k_noalloc_setup<<<1, 32, 0, st>>>(s, in, out, d_sys, d_ptr);
  lq_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lq_set_error(std::string("dslash_noalloc: ") + cudaGetErrorString(e));
    return LQCD_ECUDA;
  }
  Batch b;
  b.nsys = 1;
  b.max_n = n;
  b.total = n;
  b.nby = (int)((n + LQ_BLOCK - 1) / LQ_BLOCK);
  b.pstride = b.nby;
  b.sys = d_sys;
  // the conversion writes every site of both parities and the operator every
  // output site, so no part of the scratch needs to start at zero
  rc = lq_nat_to_eo(L, b, (const double2* const*)d_ptr, in_e, in_o, st);
  if (rc) return rc;
  const bool clov = L->csw != 0.0;
  VecP none, ie, io, oe, oo;
  ie.d = in_e;
  io.d = in_o;
  oe.d = out_e;
  oo.d = out_o;
  rc = lq_hop_lin(64, dagger != 0, clov, lq::RED_NONE, L, b, 0, io, ie, none, none, oe, -0.5, 1.0, 0.0, st);
  if (rc) return rc;
  rc = lq_hop_lin(64, dagger != 0, clov, lq::RED_NONE, L, b, 1, ie, io, none, none, oo, -0.5, 1.0, 0.0, st);
  if (rc) return rc;
  rc = lq_eo_to_nat(L, b, out_e, out_o, (double2* const*)(d_ptr + 1), 1.0, st);
  if (rc) return rc;
  return 0;
}
