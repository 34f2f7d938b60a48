// batch_common.cuh — tables and helpers shared by the batched kernels
// (batch.cu: discretize, VJP; batch_fused.cu: discretize and VJP in one pass).
#pragma once

#include "disc_link.cuh"
#include "vjp_link.cuh"

namespace ciscvx {

struct BatchCommon {
  const DevModel* const* models;
  const DevInst* inst;
  const int2* entries;   // (instance, k)
  const int4* groups;    // (model, nsub, first entry, count)
  const int2* items;     // (group, link)
  int n_items;
  int persistent;
  int* queue;
  unsigned* status;
  int layout;
  int ck_smem;  // fused pass: FP32 checkpoints in dynamic shared memory (4 n_sub floats per thread)
};

__device__ __forceinline__ int next_item(const BatchCommon& c, int& local_iter) {
  if (!c.persistent) {
    const int w = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    return local_iter++ == 0 ? w : c.n_items;
  }
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(c.queue, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// Launch bounds per occupancy variant: (threads per CTA, min CTAs per SM).
template <int OCC> struct Occ;
template <> struct Occ<0> { static constexpr int T = 256, B = 1; };  // no register cap
template <> struct Occ<1> { static constexpr int T = 128, B = 3; };  // <= 168 registers
template <> struct Occ<2> { static constexpr int T = 128, B = 4; };  // <= 128 registers

// Discretize and VJP of the items of `c` in one pass (batch_fused.cu): the
// discretization's forward sweep hands its checkpoints to the adjoint.
// prec: CISCVX_FP64 / CISCVX_FP32_PHI; occ: register-cap variant; compact outputs.
cudaError_t launch_disc_vjp_fused(const BatchCommon& c, int prec, int occ, bool compact,
                                  unsigned blocks, unsigned threads, const double* X,
                                  const double* U, const double* s, void* A, void* Bm, void* Bp,
                                  void* S, double* defect, double* penalty, const double* w,
                                  const double* rho, double* gX, double* part, double* ps,
                                  double* pL, size_t smem, cudaStream_t st);

}  // namespace ciscvx
