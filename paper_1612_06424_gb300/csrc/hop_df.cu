// Instantiations of the stencil kernels in double-float arithmetic (P = 65:
// FP64 data, arithmetic on the FP32 pipes through dfloat.h), the operator of
// the mixed-precision solvers' FP64-accuracy steps; a translation unit of its
// own so that it compiles in parallel with the rest of the library.
#include "dslash.cuh"

namespace lq {

namespace {

template <bool DAG, bool CLOV>
int lin_df(int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  constexpr int XY = EPI_X | EPI_Y, XZ = EPI_X | EPI_Z, XYZ = EPI_X | EPI_Y | EPI_Z;
  if (red == RED_NONE && epi == XY) k_hop_lin<65, DAG, CLOV, RED_NONE, XY><<<gr, 128, 0, st>>>(a);
  else if (red == RED_NONE && epi == XZ) k_hop_lin<65, DAG, CLOV, RED_NONE, XZ><<<gr, 128, 0, st>>>(a);
  else if (red == RED_DOT_W && epi == XY) k_hop_lin<65, DAG, CLOV, RED_DOT_W, XY><<<gr, 128, 0, st>>>(a);
  else if (red == RED_TS && epi == XY) k_hop_lin<65, DAG, CLOV, RED_TS, XY><<<gr, 128, 0, st>>>(a);
  else if (red == RED_NORM && epi == XYZ) k_hop_lin<65, DAG, CLOV, RED_NORM, XYZ><<<gr, 128, 0, st>>>(a);
  else return -1;
  return 0;
}

template <bool DAG, bool CLOV>
int clinv_df(int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (epi == EPI_X) k_hop_clinv<65, DAG, CLOV, EPI_X><<<gr, 128, 0, st>>>(a);
  else if (epi == EPI_Y) k_hop_clinv<65, DAG, CLOV, EPI_Y><<<gr, 128, 0, st>>>(a);
  else if (epi == (EPI_X | EPI_Y)) k_hop_clinv<65, DAG, CLOV, EPI_X | EPI_Y><<<gr, 128, 0, st>>>(a);
  else return -1;
  return 0;
}

}  // namespace

int hop_lin_df(bool dag, bool clov, int red, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (dag) return clov ? lin_df<true, true>(red, epi, gr, a, st) : lin_df<true, false>(red, epi, gr, a, st);
  return clov ? lin_df<false, true>(red, epi, gr, a, st) : lin_df<false, false>(red, epi, gr, a, st);
}

int hop_clinv_df(bool dag, bool clov, int epi, dim3 gr, const HopArgs& a, cudaStream_t st) {
  if (dag) return clov ? clinv_df<true, true>(epi, gr, a, st) : clinv_df<true, false>(epi, gr, a, st);
  return clov ? clinv_df<false, true>(epi, gr, a, st) : clinv_df<false, false>(epi, gr, a, st);
}

}  // namespace lq
