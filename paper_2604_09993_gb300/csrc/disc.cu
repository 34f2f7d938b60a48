// disc.cu — linearized discretization kernel (Sec. IV-B Eqs. (14)-(15), Eq. (17b); IND + FOH, Sec. VI).
//
// Mapping: one warp = 32 consecutive intervals x one link; lane = interval.
// Every lane of a warp runs the same link program (same code path, same
// trip counts), so each FP64 instruction does useful work in all lanes: on
// this GPU a partly masked FP64 instruction costs a full issue slot.
// Each lane integrates its link's rotation (theta, omega) and 9 tangent
// columns by RK4 in registers, uses the closed-form translation, and, for a
// foot link, the contact's penalty state and its row; it then writes the
// link's rows of A, B-, B+, S, the defect, penalty and optional z.
#include "disc_link.cuh"

namespace ciscvx {

// CMP: compact A/Bm/Bp (structural nonzeros only; strides nnzA / nnzB).
// AUX: the model uses the Eq. (12) auxiliary state (foot links take the CROSS path).
template <typename TP, bool CMP, bool AUX = false>
__global__ void __launch_bounds__(128) k_discretize(const DevModel* __restrict__ Mp, int N,
                                                    int nsub, int layout,
                                                    const double* __restrict__ X,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ s, TP* A, TP* Bm,
                                                    TP* Bp, TP* S, double* defect,
                                                    double* penalty, double* z,
                                                    unsigned* status) {
  const DevModel& M = *Mp;
  const int nb = M.nb;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long grp = warp / nb;
  const int b = (int)(warp - grp * nb);
  const long k = grp * 32 + lane;
  if (k >= N) return;
  const int nxt = M.nxt, nu = M.nu, nc = M.nc;
  const double* uL = (layout == CISCVX_FOH_NODE) ? U + k * nu : U + 2 * k * nu;
  const double* uR = uL + nu;
  const size_t sa = CMP ? (size_t)M.nnzA : (size_t)nxt * nxt;
  const size_t sb = CMP ? (size_t)M.nnzB : (size_t)nxt * nu;
  TP* Ak = A + k * sa;
  TP* Bmk = Bm ? Bm + k * sb : nullptr;
  TP* Bpk = Bp ? Bp + k * sb : nullptr;
  TP* Sk = S + (size_t)k * nxt;
  double* dk = defect + (size_t)k * nxt;
  double* pk = penalty ? penalty + (size_t)k * nc : nullptr;
  double* zk = z ? z + (size_t)k * nxt : nullptr;
  if constexpr (AUX) {
    if (M.body[b].contact >= 0) {  // Eq. (12) model (z from the dense outputs, by the caller)
      disc_link<TP, true, CMP, false, true>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL,
                                            uR, Ak, Bmk, Bpk, Sk, dk, pk, nullptr, status);
      return;
    }
  }
  if (M.body[b].contact >= 0)
    disc_link<TP, true, CMP>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL, uR, Ak, Bmk,
                             Bpk, Sk, dk, pk, zk, status);
  else
    disc_link<TP, false, CMP>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL, uR, Ak, Bmk,
                              Bpk, Sk, dk, pk, zk, status);
}

cudaError_t launch_discretize(const DevModel* dM, int nb, int N, int nsub, int prec, int layout,
                              bool compact, bool aux, const double* X, const double* U,
                              const double* s, void* A, void* Bm, void* Bp, void* S,
                              double* defect, double* penalty, double* z, unsigned* status,
                              cudaStream_t st) {
  const long warps = (long)((N + 31) / 32) * nb;
  const int threads = single_cta_threads(warps);
  const long blocks = (warps * 32 + threads - 1) / threads;
#define CISCVX_K(TP, CMP)                                                                    \
  k_discretize<TP, CMP><<<(unsigned)blocks, threads, 0, st>>>(                                \
      dM, N, nsub, layout, X, U, s, (TP*)A, (TP*)Bm, (TP*)Bp, (TP*)S, defect, penalty, z, status)
  if (aux) {  // Eq. (12) model: the kernels form no z (the caller does, from dense outputs)
#define CISCVX_KA(TP, CMP)                                                                    \
  k_discretize<TP, CMP, true><<<(unsigned)blocks, threads, 0, st>>>(                          \
      dM, N, nsub, layout, X, U, s, (TP*)A, (TP*)Bm, (TP*)Bp, (TP*)S, defect, penalty, nullptr, status)
    if (prec == CISCVX_FP64) {
      if (compact) CISCVX_KA(double, true); else CISCVX_KA(double, false);
    } else {
      if (compact) CISCVX_KA(float, true); else CISCVX_KA(float, false);
    }
#undef CISCVX_KA
  } else if (prec == CISCVX_FP64) {
    if (compact) CISCVX_K(double, true); else CISCVX_K(double, false);
  } else {
    if (compact) CISCVX_K(float, true); else CISCVX_K(float, false);
  }
#undef CISCVX_K
  return cudaGetLastError();
}

}  // namespace ciscvx
