// affine_z.cu — the affine term z_k of the linearized dynamics (Eq. (17b)),
// z_k = x~(1) - A_k x~_k - B-_k u_L - B+_k u_R - S_k s_k, formed by a post-pass
// over the stored outputs for the models whose kernels do not form it in
// registers (the Eq. (12) auxiliary state, coupled links): from the dense
// blocks, or from the compact values and the model's pattern by rows.
#include "common.cuh"

namespace ciscvx {

namespace {

// z_k = x~(1) - A_k x~_k - B-_k u_L - B+_k u_R - S_k s_k with x~(1) =
// defect_k + x~_{k+1}: thread per (interval, row), FP64 accumulation over the
// row of each block (a thread's row is contiguous, so its loads reuse L1 lines).
template <typename TP>
__global__ void __launch_bounds__(256) k_affine_z(int nxt, int nu, long N, int node_layout,
                                                  const double* __restrict__ X, const double* __restrict__ U,
                                                  const double* __restrict__ s, const TP* __restrict__ A,
                                                  const TP* __restrict__ Bm, const TP* __restrict__ Bp,
                                                  const TP* __restrict__ S, const double* __restrict__ defect,
                                                  double* __restrict__ z) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N * nxt) return;
  const long k = g / nxt;
  const double* xk = X + k * nxt;
  double acc = defect[g] + X[g + nxt];
  const TP* a = A + g * nxt;
  for (int c = 0; c < nxt; ++c) acc = fma(-(double)a[c], xk[c], acc);
  if (nu > 0) {
    const double* uL = U + (node_layout ? k : 2 * k) * nu;
    const double* uR = U + (node_layout ? k + 1 : 2 * k + 1) * nu;
    const TP* bm = Bm + g * nu;
    const TP* bp = Bp + g * nu;
    for (int q = 0; q < nu; ++q) acc = fma(-(double)bm[q], uL[q], fma(-(double)bp[q], uR[q], acc));
  }
  z[g] = fma(-(double)S[g], s[k], acc);
}

}  // namespace

cudaError_t launch_affine_z(const DevModel& M, int N, int prec, int layout, const double* X, const double* U,
                            const double* s, const void* A, const void* Bm, const void* Bp, const void* S,
                            const double* defect, double* z, cudaStream_t st) {
  const long n = (long)N * M.nxt;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  const int node = layout == CISCVX_FOH_NODE;
  if (prec == CISCVX_FP64)
    k_affine_z<double><<<grid, bs, 0, st>>>(M.nxt, M.nu, N, node, X, U, s, (const double*)A, (const double*)Bm,
                                           (const double*)Bp, (const double*)S, defect, z);
  else
    k_affine_z<float><<<grid, bs, 0, st>>>(M.nxt, M.nu, N, node, X, U, s, (const float*)A, (const float*)Bm,
                                          (const float*)Bp, (const float*)S, defect, z);
  return cudaGetLastError();
}

namespace {

// z from compact outputs: thread = (interval, row); the row's structural
// nonzeros of A and B-/B+ come from the pattern by rows (zpat: A offsets
// [nxt + 1], (entry, column) pairs, then the same for B).
template <typename TP>
__global__ void __launch_bounds__(256) k_affine_z_compact(int nxt, int nu, int nnza, int nnzb, long N,
                                                          int node_layout, const double* __restrict__ X,
                                                          const double* __restrict__ U,
                                                          const double* __restrict__ s, const TP* __restrict__ A,
                                                          const TP* __restrict__ Bm, const TP* __restrict__ Bp,
                                                          const TP* __restrict__ S,
                                                          const double* __restrict__ defect,
                                                          const int32_t* __restrict__ zpat,
                                                          double* __restrict__ z) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N * nxt) return;
  const long k = g / nxt;
  const int r = (int)(g - k * nxt);
  const double* xk = X + k * nxt;
  double acc = defect[g] + X[g + nxt];
  const int32_t* aoff = zpat;
  const int32_t* aent = zpat + nxt + 1;
  for (int j = aoff[r]; j < aoff[r + 1]; ++j)
    acc = fma(-widen(A[k * nnza + aent[2 * j]]), xk[aent[2 * j + 1]], acc);
  if (nu > 0) {
    const int32_t* boff = aent + 2 * nnza;
    const int32_t* bent = boff + nxt + 1;
    const double* uL = U + (node_layout ? k : 2 * k) * nu;
    const double* uR = U + (node_layout ? k + 1 : 2 * k + 1) * nu;
    for (int j = boff[r]; j < boff[r + 1]; ++j) {
      const long e = k * nnzb + bent[2 * j];
      const int q = bent[2 * j + 1];
      acc = fma(-widen(Bm[e]), uL[q], fma(-widen(Bp[e]), uR[q], acc));
    }
  }
  z[g] = fma(-widen(S[g]), s[k], acc);
}

}  // namespace

cudaError_t launch_affine_z_compact(const DevModel& M, int N, int prec, int layout, const double* X,
                                    const double* U, const double* s, const void* A, const void* Bm,
                                    const void* Bp, const void* S, const double* defect, const int32_t* zpat,
                                    double* z, cudaStream_t st) {
  const long n = (long)N * M.nxt;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  const int node = layout == CISCVX_FOH_NODE;
  if (prec == CISCVX_FP64)
    k_affine_z_compact<double><<<grid, bs, 0, st>>>(M.nxt, M.nu, M.nnzA, M.nnzB, N, node, X, U, s,
                                                   (const double*)A, (const double*)Bm, (const double*)Bp,
                                                   (const double*)S, defect, zpat, z);
  else
    k_affine_z_compact<float><<<grid, bs, 0, st>>>(M.nxt, M.nu, M.nnzA, M.nnzB, N, node, X, U, s,
                                                  (const float*)A, (const float*)Bm, (const float*)Bp,
                                                  (const float*)S, defect, zpat, z);
  return cudaGetLastError();
}

}  // namespace ciscvx
