// expand.cu — dense outputs of the fused pass from staged compact values.
//
// With dense outputs the fused pass (batch_fused.cu, BatchCommon.stage_dense)
// writes each interval's structural nonzeros of A, B- and B+ in the compact
// order (common.cuh) at the start of that interval's own dense blocks: one
// store per nonzero, as for compact outputs, instead of zeroing the link's
// dense rows and scattering into them.  This kernel then widens every
// interval in place, one warp per interval: the warp copies the interval's
// compact values to shared memory, then writes its dense A, B-, B+ in full
// (coalesced, structural zeros included), taking each dense entry's value
// from the per-model map of compact indices.  Reads of an interval's compact
// values all precede the writes that overwrite them (same warp, one
// __syncwarp between).
#include <type_traits>

#include "batch_common.cuh"

namespace ciscvx {

namespace {

constexpr int EXPAND_WARPS = 4;

template <typename TP>
__global__ void __launch_bounds__(32 * EXPAND_WARPS)
    k_expand_dense(const int2* __restrict__ entries, int e0, int e1, const DevInst* __restrict__ inst,
                   const DevModel* const* __restrict__ models, const int* const* __restrict__ map_a,
                   const int* const* __restrict__ map_b, int smem_vals, TP* A, TP* Bm, TP* Bp) {
  extern __shared__ unsigned char ex_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TP* buf = reinterpret_cast<TP*>(ex_smem) + (size_t)warp * smem_vals;
  const long e = (long)e0 + (long)blockIdx.x * EXPAND_WARPS + warp;
  if (e >= e1) return;
  const int2 en = entries[e];
  const DevInst& I = inst[en.x];
  const DevModel& M = *models[I.model];
  const int nxt = M.nxt, nu = M.nu, na = M.nnzA, nbz = M.nnzB;
  const long k = en.y;
  TP* Ak = A + I.a + k * (size_t)nxt * nxt;
  for (int j = lane; j < na; j += 32) buf[j] = Ak[j];
  TP* Bmk = nullptr;
  TP* Bpk = nullptr;
  if (nu > 0) {
    Bmk = Bm + I.b + k * (size_t)nxt * nu;
    Bpk = Bp + I.b + k * (size_t)nxt * nu;
    for (int j = lane; j < nbz; j += 32) {
      buf[na + j] = Bmk[j];
      buf[na + nbz + j] = Bpk[j];
    }
  }
  __syncwarp();
  // 16-byte stores where the block and its map allow them
  constexpr int V = 16 / sizeof(TP);  // elements per 16-byte store
  using VT = typename std::conditional<sizeof(TP) == 4, float4, double2>::type;
  auto widen_block = [&](TP* dst, const int* map, int n, int off) {
    if (n % V == 0 && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(map)) & 15) == 0) {
      for (int i = lane; i < n / V; i += 32) {
        TP v[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
          const int m = map[V * i + t];
          v[t] = m >= 0 ? buf[off + m] : TP(0);
        }
        VT w;
        memcpy(&w, v, sizeof w);
        reinterpret_cast<VT*>(dst)[i] = w;
      }
    } else {
      for (int i = lane; i < n; i += 32) {
        const int m = map[i];
        dst[i] = m >= 0 ? buf[off + m] : TP(0);
      }
    }
  };
  widen_block(Ak, map_a[I.model], nxt * nxt, 0);
  if (nu > 0) {
    const int* mb = map_b[I.model];
    widen_block(Bmk, mb, nxt * nu, na);
    widen_block(Bpk, mb, nxt * nu, na + nbz);
  }
}

}  // namespace

cudaError_t launch_expand_dense(const BatchCommon& c, int prec, const int* const* map_a,
                                const int* const* map_b, int smem_vals, void* A, void* Bm, void* Bp,
                                cudaStream_t st) {
  const long n = (long)c.e1 - c.e0;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + EXPAND_WARPS - 1) / EXPAND_WARPS);
  const size_t el = prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
  const size_t smem = (size_t)EXPAND_WARPS * (size_t)smem_vals * el;
  if (smem > 48u * 1024u) {
    const cudaError_t e =
        prec == CISCVX_FP64
            ? cudaFuncSetAttribute(k_expand_dense<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(k_expand_dense<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (prec == CISCVX_FP64)
    k_expand_dense<double><<<blocks, 32 * EXPAND_WARPS, smem, st>>>(c.entries, c.e0, c.e1, c.inst, c.models, map_a,
                                                                    map_b, smem_vals, (double*)A, (double*)Bm,
                                                                    (double*)Bp);
  else
    k_expand_dense<float><<<blocks, 32 * EXPAND_WARPS, smem, st>>>(c.entries, c.e0, c.e1, c.inst, c.models, map_a,
                                                                   map_b, smem_vals, (float*)A, (float*)Bm,
                                                                   (float*)Bp);
  return cudaGetLastError();
}

}  // namespace ciscvx
