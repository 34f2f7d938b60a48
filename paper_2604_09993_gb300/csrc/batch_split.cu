// batch_split.cu — linearized discretization and adjoint VJP of every work
// item on separate warps of one launch: the split form of the fused pass
// (batch_fused.cu) for batches too small to fill the GPU.  There a warp's
// instruction stream, not the GPU's throughput, sets the time, and the fused
// pass runs the forward and the backward sweep of an item one after the
// other in one warp; here they run side by side on two warps, each of which
// integrates the trajectory itself.  No register cap: the grid is small.
#include "batch_common.cuh"

namespace ciscvx {

namespace {

// Items [0, n) linearize, items [n, 2n) take the adjoint (c.n_items = 2n).
template <typename TP, bool CMP, bool AUX>
__global__ void __launch_bounds__(Occ<0>::T, Occ<0>::B)
    k_batch_split(BatchCommon c, int n, const double* __restrict__ X, const double* __restrict__ U,
                  const double* __restrict__ s, TP* A, TP* Bm, TP* Bp, TP* S, double* defect,
                  double* penalty, const double* __restrict__ w, const double* __restrict__ rho,
                  double* gX, double* part, double* ps, double* pL) {
  int iter = 0;
  for (;;) {
    const int item = next_item(c, iter);
    if (item >= c.n_items) break;
    if (item < n) disc_item<TP, CMP, AUX>(c, item, X, U, s, A, Bm, Bp, S, defect, penalty);
    else vjp_item<TP, AUX>(c, item - n, X, U, s, w, rho, gX, part, ps, pL);
  }
}

}  // namespace

cudaError_t launch_disc_vjp_split(const BatchCommon& c, int n, int prec, bool compact, bool aux,
                                  unsigned blocks, unsigned threads, const double* X,
                                  const double* U, const double* s, void* A, void* Bm, void* Bp,
                                  void* S, double* defect, double* penalty, const double* w,
                                  const double* rho, double* gX, double* part, double* ps,
                                  double* pL, cudaStream_t st) {
#define CISCVX_SPLIT1(TP, CMP, AUX)                                                                 \
  k_batch_split<TP, CMP, AUX><<<blocks, threads, 0, st>>>(c, n, X, U, s, (TP*)A, (TP*)Bm, (TP*)Bp,      \
                                                          (TP*)S, defect, penalty, w, rho, gX, part, ps, \
                                                          pL)
#define CISCVX_SPLIT(TP, CMP)                          \
  do {                                                 \
    if (aux) CISCVX_SPLIT1(TP, CMP, true);             \
    else CISCVX_SPLIT1(TP, CMP, false);                \
  } while (0)
  if (prec == CISCVX_FP64) {
    if (compact) CISCVX_SPLIT(double, true); else CISCVX_SPLIT(double, false);
  } else {
    if (compact) CISCVX_SPLIT(float, true); else CISCVX_SPLIT(float, false);
  }
#undef CISCVX_SPLIT1
#undef CISCVX_SPLIT
  return cudaGetLastError();
}

}  // namespace ciscvx
