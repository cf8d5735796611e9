// Shared-memory layouts of the tensor-core nucleon-block kernel (nucleon_tc.cu), host and device.
//
// Operands (tcgen05.mma, K-major, no swizzle): a core matrix is 8 rows x 16 bytes (4 TF32).  The
// R-row x 8-value operand of one K-step is R/8 row groups x 2 core matrices, and element (r, q)
// lies at  tc_operand_offset(r, q)  =  ((r / 8) * 2 + q / 4) * 128 + (r % 8) * 16 + (q % 4) * 4.
// The matrix descriptor describes it by the leading-dimension byte offset TC_LBO (between the two
// core matrices along K) and the stride-dimension byte offset TC_SBO (between row groups):
// tc_desc_offset(r, q, TC_LBO, TC_SBO) is the same address.  Each operand has its own block of
// R * 32 bytes, and the offsets formed with the two byte offsets exchanged stay inside it too.
//
// Staging of one chunk's spinors (FP32 complex, float2 units): per site TC_SITE_STG words; the
// 24 (i, j) spinors at a stride of 14 from 0, then the 32 k spinors at a stride of 12.
#pragma once

namespace lq {

constexpr int TC_LBO = 128, TC_SBO = 256;
constexpr int TC_TI = 8, TC_TJ = 16, TC_TK = 32;
constexpr int TC_SITE_STG = (TC_TI + TC_TJ) * 14 + TC_TK * 12;

__host__ __device__ __forceinline__ int tc_operand_offset(int r, int q) {
  return ((r >> 3) * 2 + (q >> 2)) * 128 + (r & 7) * 16 + (q & 3) * 4;
}

// the byte address, relative to the descriptor's start, of element (r, q) of a K-major
// no-swizzle operand with the given leading / stride byte offsets
__host__ __device__ __forceinline__ int tc_desc_offset(int r, int q, int lbo, int sbo) {
  return (r >> 3) * sbo + (q >> 2) * lbo + (r & 7) * 16 + (q & 3) * 4;
}

// float2 index of component comp (0..11) of staging slot `slot` (0..55) of site x
__host__ __device__ __forceinline__ int tc_stage_index(int x, int slot, int comp) {
  const int off = slot < TC_TI + TC_TJ ? slot * 14 : (TC_TI + TC_TJ) * 14 + (slot - TC_TI - TC_TJ) * 12;
  return x * TC_SITE_STG + off + comp;
}

}  // namespace lq
