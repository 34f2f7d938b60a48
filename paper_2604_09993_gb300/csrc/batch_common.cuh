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
  // two_q (persistent launches, lpt_order 2): items [0, n_first) are the
  // foot-link items and [n_first, n_items) the others, each pulled from its
  // own counter (queue[0], queue[1]); the CTAs on SMs [0, split_sm) take the
  // foot-link queue, the others the second one, and each moves to the other
  // queue when its own runs dry.  An SM thus runs one link kind's code (the
  // instruction cache holds one of them), and the two kinds of an interval
  // group run at about the same time (its inputs and the output sectors its
  // links share are still in L2).
  int two_q, n_first, split_sm, sm_count;
  int* queue;
  unsigned* status;
  int layout;
  int ck_smem;  // fused pass: FP32 checkpoints in dynamic shared memory (4 n_sub floats per thread)
  // fused pass with dense outputs: the kernel writes each interval's compact
  // values (structural nonzeros, compact order) at the start of that
  // interval's dense A / B- / B+ blocks, and k_expand_dense then widens them
  // in place; entries [e0, e1) are the per-link intervals this launch covers
  int stage_dense;
  int e0, e1;
};

__device__ __forceinline__ int next_item(const BatchCommon& c, int& local_iter) {
  if (!c.persistent) {
    const int w = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    return local_iter++ == 0 ? w : c.n_items;
  }
  if (c.two_q) {
    // local_iter: 0 own queue, 1 the other one, 2 both exhausted (warp-uniform)
    int it = c.n_items;
    if ((threadIdx.x & 31) == 0) {
      // SM ids need not be contiguous: compare smid / nsmid with split_sm / sm_count
      unsigned smid, nsmid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
      const int mine =
          (unsigned long long)smid * (unsigned)c.sm_count < (unsigned long long)c.split_sm * nsmid ? 0 : 1;
      while (local_iter < 2) {
        const int q = local_iter == 0 ? mine : 1 - mine;
        const int nq = q == 0 ? c.n_first : c.n_items - c.n_first;
        const int k = atomicAdd(c.queue + q, 1);
        if (k < nq) { it = (q == 0 ? 0 : c.n_first) + k; break; }
        ++local_iter;
      }
    }
    local_iter = __shfl_sync(0xffffffffu, local_iter, 0);
    return __shfl_sync(0xffffffffu, it, 0);
  }
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(c.queue, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// Linearization of work item `item` (its warp's lanes; lanes past the group's
// width idle).  AUX: the batch holds an Eq. (12) model (its foot links take
// the CROSS path).
template <typename TP, bool CMP, bool AUX>
__device__ __forceinline__ void disc_item(const BatchCommon& c, int item, const double* __restrict__ X,
                                          const double* __restrict__ U, const double* __restrict__ s,
                                          TP* A, TP* Bm, TP* Bp, TP* S, double* defect,
                                          double* penalty) {
  const int lane = threadIdx.x & 31;
  const int2 it = c.items[item];
  const int4 g = c.groups[it.x];
  if (lane >= g.w) return;
  const DevModel& M = *c.models[g.x];
  const int b = it.y;
  const int2 e = c.entries[g.z + lane];
  const DevInst& I = c.inst[e.x];
  const long k = e.y;
  const int nxt = M.nxt, nu = M.nu, nc = M.nc;
  const double* Xi = X + I.x;
  const double* uL = (c.layout == CISCVX_FOH_NODE) ? U + I.u + k * nu : U + I.u + 2 * k * nu;
  const double* uR = uL + nu;
  const size_t sa = CMP ? (size_t)M.nnzA : (size_t)nxt * nxt;
  const size_t sb = CMP ? (size_t)M.nnzB : (size_t)nxt * nu;
  TP* Ak = A + I.a + k * sa;
  TP* Bmk = Bm ? Bm + I.b + k * sb : nullptr;
  TP* Bpk = Bp ? Bp + I.b + k * sb : nullptr;
  TP* Sk = S + I.v + (size_t)k * nxt;
  double* dk = defect + I.v + (size_t)k * nxt;
  double* pk = penalty ? penalty + I.p + (size_t)k * nc : nullptr;
  if (AUX && M.aux && M.body[b].contact >= 0)  // Eq. (12) model
    disc_link<TP, true, CMP, false, AUX>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL,
                                         uR, Ak, Bmk, Bpk, Sk, dk, pk, nullptr, c.status);
  else if (M.body[b].contact >= 0)
    disc_link<TP, true, CMP>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL, uR, Ak, Bmk,
                             Bpk, Sk, dk, pk, nullptr, c.status);
  else
    disc_link<TP, false, CMP>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL, uR, Ak,
                              Bmk, Bpk, Sk, dk, pk, nullptr, c.status);
}

// Adjoint VJP of work item `item` (its own forward sweep, then the backward
// sweep), writing the item's partial sums.  AUX: as for disc_item.
template <typename TP, bool AUX = false>
__device__ __forceinline__ void vjp_item(const BatchCommon& c, int item, const double* __restrict__ X,
                                         const double* __restrict__ U, const double* __restrict__ s,
                                         const double* __restrict__ w, const double* __restrict__ rho,
                                         double* gX, double* part, double* ps, double* pL) {
  const int lane = threadIdx.x & 31;
  const int2 it = c.items[item];
  const int4 g = c.groups[it.x];
  if (lane >= g.w) return;
  const DevModel& M = *c.models[g.x];
  const int b = it.y;
  const int2 e = c.entries[g.z + lane];
  const DevInst& I = c.inst[e.x];
  const long k = e.y;
  const int N = I.N, nxt = M.nxt, nu = M.nu, nc = M.nc, nb = M.nb;
  const double* Xi = X + I.x;
  const double* uL = (c.layout == CISCVX_FOH_NODE) ? U + I.u + k * nu : U + I.u + 2 * k * nu;
  const double* uR = uL + nu;
  const double* wi = w + I.v;
  const DevBody& B = M.body[b];
  const double rc = (B.contact >= 0) ? rho[I.p + k * nc + B.contact] : 0.0;
  const double* wkm1 = (k > 0) ? wi + (k - 1) * nxt : nullptr;
  double* gXi = gX + I.x;
  double* gXN = (k == N - 1) ? gXi + (size_t)N * nxt : nullptr;
  double* pp = part + I.part + (size_t)k * M.nslot * 2;
  double* psk = ps + I.pb + k * nb;
  double* pLk = pL + I.pb + k * nb;
  if (AUX && M.aux && B.contact >= 0)  // Eq. (12) model
    vjp_link<TP, true, false, true>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL, uR,
                                    wi + k * nxt, wkm1, rc, gXi + (size_t)k * nxt, gXN, pp, psk, pLk,
                                    c.status);
  else if (B.contact >= 0)
    vjp_link<TP, true>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL, uR, wi + k * nxt,
                       wkm1, rc, gXi + (size_t)k * nxt, gXN, pp, psk, pLk, c.status);
  else
    vjp_link<TP, false>(M, b, g.y, s[I.s + k], Xi + k * nxt, Xi + (k + 1) * nxt, uL, uR, wi + k * nxt,
                        wkm1, rc, gXi + (size_t)k * nxt, gXN, pp, psk, pLk, c.status);
}

// Launch bounds per occupancy variant: (threads per CTA, min CTAs per SM).
template <int OCC> struct Occ;
template <> struct Occ<0> { static constexpr int T = 256, B = 1; };  // no register cap
template <> struct Occ<1> { static constexpr int T = 128, B = 3; };  // <= 168 registers
template <> struct Occ<2> { static constexpr int T = 128, B = 4; };  // <= 128 registers

// Discretize and VJP of the items of `c` in one pass (batch_fused.cu): the
// discretization's forward sweep hands its checkpoints to the adjoint.
// prec: CISCVX_FP64 / CISCVX_FP32_PHI; occ: register-cap variant (ignored
// with aux: an Eq. (12) model in the batch); compact outputs.
cudaError_t launch_disc_vjp_fused(const BatchCommon& c, int prec, int occ, bool compact, bool aux,
                                  unsigned blocks, unsigned threads, const double* X,
                                  const double* U, const double* s, void* A, void* Bm, void* Bp,
                                  void* S, double* defect, double* penalty, const double* w,
                                  const double* rho, double* gX, double* part, double* ps,
                                  double* pL, size_t smem, cudaStream_t st);

// Widens the compact values that the fused pass staged at the start of each
// interval's dense blocks (BatchCommon.stage_dense) into the dense A, B-, B+
// of entries [c.e0, c.e1): one warp per interval reads its compact values
// into shared memory, then writes the whole dense blocks, structural zeros
// included.  map_a / map_b hold, per model, the compact index of every dense
// entry of A (n_x~ x n_x~) and of B-/B+ (n_x~ x n_u), -1 for a structural
// zero; smem_vals is the largest nnz_A + 2 nnz_B of the plan's models.
cudaError_t launch_expand_dense(const BatchCommon& c, int prec, const int* const* map_a,
                                const int* const* map_b, int smem_vals, void* A, void* Bm, void* Bp,
                                cudaStream_t st);

// The same outputs with the linearization and the VJP of every item on
// separate warps of one launch (items [0, n) linearize, [n, 2n) take the
// adjoint; c.n_items = 2n).  Each warp integrates the trajectory itself: more
// work than the fused pass, but a shorter path per warp, for batches too
// small to fill the GPU (batch_split.cu; no register cap).
cudaError_t launch_disc_vjp_split(const BatchCommon& c, int n, int prec, bool compact, bool aux,
                                  unsigned blocks, unsigned threads, const double* X,
                                  const double* U, const double* s, void* A, void* Bm, void* Bp,
                                  void* S, double* defect, double* penalty, const double* w,
                                  const double* rho, double* gX, double* part, double* ps,
                                  double* pL, cudaStream_t st);

}  // namespace ciscvx
