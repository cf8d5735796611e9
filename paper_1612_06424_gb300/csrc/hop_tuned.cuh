// Launchers of the alternative launch configurations (HopCfg 1 and 2) of the
// one-thread-per-site stencil kernels, for the forward operator (the
// solver's D^; dagger solves keep the default configuration).  Each
// precision's instantiations live in a translation unit of their own
// (hop_tuned32.cu, hop_tuned16.cu) so that they compile in parallel with the
// rest of the library.
#pragma once

#include "dslash.cuh"

namespace lq {

template <int P, int CFG, bool CLOV>
int hop_lin_cfg(int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  constexpr int XY = EPI_X | EPI_Y, XZ = EPI_X | EPI_Z, XYZ = EPI_X | EPI_Y | EPI_Z;
  if (red == RED_NONE && epi == XY) k_hop_lin<P, false, CLOV, RED_NONE, XY, CFG><<<gr, 128, 0, st>>>(a);
  else if (red == RED_NONE && epi == XZ) k_hop_lin<P, false, CLOV, RED_NONE, XZ, CFG><<<gr, 128, 0, st>>>(a);
  else if (red == RED_DOT_W && epi == XY) k_hop_lin<P, false, CLOV, RED_DOT_W, XY, CFG><<<gr, 128, 0, st>>>(a);
  else if (red == RED_TS && epi == XY) k_hop_lin<P, false, CLOV, RED_TS, XY, CFG><<<gr, 128, 0, st>>>(a);
  else if (red == RED_NORM && epi == XYZ) k_hop_lin<P, false, CLOV, RED_NORM, XYZ, CFG><<<gr, 128, 0, st>>>(a);
  else return -1;
  return 0;
}

template <int P, int CFG, bool CLOV>
int hop_clinv_cfg(int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (epi == EPI_X) k_hop_clinv<P, false, CLOV, EPI_X, CFG><<<gr, 128, 0, st>>>(a);
  else if (epi == EPI_Y) k_hop_clinv<P, false, CLOV, EPI_Y, CFG><<<gr, 128, 0, st>>>(a);
  else if (epi == (EPI_X | EPI_Y)) k_hop_clinv<P, false, CLOV, EPI_X | EPI_Y, CFG><<<gr, 128, 0, st>>>(a);
  else return -1;
  return 0;
}

// cfg 1 or 2; returns -1 for an unsupported (reduction, epilogue) pair
template <int P>
int hop_lin_tuned(int cfg, bool clov, int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (cfg == 1) return clov ? hop_lin_cfg<P, 1, true>(red, epi, gr, a, st) : hop_lin_cfg<P, 1, false>(red, epi, gr, a, st);
  return clov ? hop_lin_cfg<P, 2, true>(red, epi, gr, a, st) : hop_lin_cfg<P, 2, false>(red, epi, gr, a, st);
}

template <int P>
int hop_clinv_tuned(int cfg, bool clov, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (cfg == 1) return clov ? hop_clinv_cfg<P, 1, true>(epi, gr, a, st) : hop_clinv_cfg<P, 1, false>(epi, gr, a, st);
  return clov ? hop_clinv_cfg<P, 2, true>(epi, gr, a, st) : hop_clinv_cfg<P, 2, false>(epi, gr, a, st);
}

}  // namespace lq
