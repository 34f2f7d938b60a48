// contract.cu — the VJP by linearize-and-contract, for the models without a
// reverse-mode adjoint kernel (the full Eq. (12) auxiliary state, coupled
// links).  Per chunk of intervals the dense IND blocks are formed in the
// workspace by the discretization kernels, then contracted with the cotangent
// of the scalar L = sum_k w_k . defect_k + sum_k rho_k . penalty_k:
//   lambda_k = w_k + rho_k on the path-penalty rows       (cotangent of x~(1) of interval k)
//   dL/dx~_k = A_k^T lambda_k - (rho_k on the path-penalty rows) - w_{k-1}
//   dL/du    = B-_k^T lambda_k at u_L, B+_k^T lambda_k at u_R (node layout:
//              node k collects B-_k^T lambda_k + B+_{k-1}^T lambda_{k-1})
//   dL/ds_k  = S_k . lambda_k
// (defect_k = x~(1) - x~_{k+1}, penalty_k = y(1) - y_k, Eq. (17b)).  The
// contraction runs one thread per (interval, output column), each a dot
// product down one column of a block, so a warp's loads of one row are
// contiguous; node-shared sums carry across chunk boundaries through the
// output itself (chunks run in stream order), so no atomics are needed and
// the result does not depend on the chunking.  L is reduced per chunk by one
// block in a fixed order.
#include "coupled.cuh"

namespace ciscvx {

namespace {

template <typename TP>
__global__ void k_contract(int nxt, int nu, int nc, int pen0, long i0, long n, long N, int layout,
                           const TP* __restrict__ A, const TP* __restrict__ Bm,
                           const TP* __restrict__ Bp, const TP* __restrict__ S,
                           const double* __restrict__ w, const double* __restrict__ rho,
                           double* __restrict__ gX, double* __restrict__ gU,
                           double* __restrict__ gs) {
  const int ncol = nxt + nu + 1;
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long t = g / ncol;
  if (t >= n) return;
  const int c = (int)(g - t * ncol);
  const long k = i0 + t;
  const double* wk = w + k * nxt;
  auto lam = [&](const double* wv, long kk, int r) {
    double v = wv[r];
    if (r >= pen0 && r < pen0 + nc) v += rho[kk * nc + (r - pen0)];
    return v;
  };
  // block values are widened on the integer pipe (the FP64 pipe bounds this)
  auto dot = [&](const TP* col, int stride, const double* wv, long kk) {
    double acc = 0.0;
    for (int r = 0; r < nxt; ++r) acc = fma(widen(col[(size_t)r * stride]), lam(wv, kk, r), acc);
    return acc;
  };
  if (c < nxt) {
    double acc = dot(A + (size_t)t * nxt * nxt + c, nxt, wk, k);
    if (c >= pen0 && c < pen0 + nc) acc -= rho[k * nc + (c - pen0)];
    if (k >= 1) acc -= w[(k - 1) * nxt + c];
    gX[k * nxt + c] = acc;
    if (k == N - 1) gX[N * nxt + c] = -wk[c];
  } else if (c < nxt + nu) {
    const int q = c - nxt;
    const double am = dot(Bm + (size_t)t * nxt * nu + q, nu, wk, k);
    if (layout == CISCVX_FOH_INTERVAL) {
      gU[(2 * k) * nu + q] = am;
      gU[(2 * k + 1) * nu + q] = dot(Bp + (size_t)t * nxt * nu + q, nu, wk, k);
    } else {
      // node k: B-_k^T lambda_k + B+_{k-1}^T lambda_{k-1}; the second term
      // comes from this chunk's previous interval or, at the chunk's first
      // interval, from the previous chunk (already stored in gU)
      double prev = 0.0;
      if (t > 0) prev = dot(Bp + (size_t)(t - 1) * nxt * nu + q, nu, w + (k - 1) * nxt, k - 1);
      else if (k > 0) prev = gU[k * nu + q];
      gU[k * nu + q] = am + prev;
      if (t == n - 1)  // carried into node k + 1
        gU[(k + 1) * nu + q] = dot(Bp + (size_t)t * nxt * nu + q, nu, wk, k);
    }
  } else {
    gs[k] = dot(S + (size_t)t * nxt, 1, wk, k);
  }
}

// L over a chunk, in two fixed-order passes (deterministic): block b sums a
// fixed contiguous range of w . defect + rho . penalty into part[b], then one
// block adds the partial sums in order to *L.
constexpr int LRED_BLOCKS = 512;

__global__ void __launch_bounds__(256) k_contract_L(int nxt, int nc, long i0, long n,
                                                    const double* __restrict__ defect,
                                                    const double* __restrict__ penalty,
                                                    const double* __restrict__ w,
                                                    const double* __restrict__ rho,
                                                    double* __restrict__ part) {
  __shared__ double red[256];
  const long nd = n * nxt, np = n * nc, tot = nd + np;
  const long per = (tot + gridDim.x - 1) / gridDim.x;
  const long lo = blockIdx.x * per, hi = lo + per < tot ? lo + per : tot;
  double acc = 0.0;
  for (long e = lo + threadIdx.x; e < hi; e += 256)
    acc = e < nd ? fma(w[i0 * nxt + e], defect[e], acc) : fma(rho[i0 * nc + (e - nd)], penalty[e - nd], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_contract_L_sum(const double* __restrict__ part, int nparts,
                                                        double* L) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < nparts; e += 256) acc += part[e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *L += red[0];
}

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Workspace layout of one chunk of n intervals.
struct ChunkLayout {
  size_t A, Bm, Bp, S, defect, penalty, part, stage, total;
};

ChunkLayout chunk_layout(const DevModel& M, const CplTab* T, long n, int nsub, int prec) {
  const size_t el = prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
  const size_t nxt = M.nxt, nu = M.nu, nc = M.nc;
  ChunkLayout L;
  size_t o = 0;
  L.A = o; o = align16(o + n * nxt * nxt * el);
  L.Bm = o; o = align16(o + n * nxt * nu * el);
  L.Bp = o; o = align16(o + n * nxt * nu * el);
  L.S = o; o = align16(o + n * nxt * el);
  L.defect = o; o = align16(o + n * nxt * sizeof(double));
  L.penalty = o; o = align16(o + n * nc * sizeof(double));
  L.part = o; o = align16(o + LRED_BLOCKS * sizeof(double));
  L.stage = o; o = align16(o + (T ? n * cpl_interval_bytes(*T, nsub, prec) : 0));
  L.total = o;
  return L;
}

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

namespace {

// The contraction of k_contract for entries (instance, k) of one model in a
// batch: the blocks at the instance's workspace offsets (inst_ws), the
// cotangents and gradients at its own (inst).  Chunks hold whole instances,
// so the node sum B-_k^T lambda_k + B+_{k-1}^T lambda_{k-1} is formed here.
template <typename TP>
__global__ void __launch_bounds__(128) k_contract_batch(int nxt, int nu, int nc, int pen0, long n, int layout,
                                                        const DevInst* __restrict__ inst,
                                                        const DevInst* __restrict__ inst_ws,
                                                        const int2* __restrict__ entries,
                                                        const TP* __restrict__ A, const TP* __restrict__ Bm,
                                                        const TP* __restrict__ Bp, const TP* __restrict__ S,
                                                        const double* __restrict__ w,
                                                        const double* __restrict__ rho, double* __restrict__ gX,
                                                        double* __restrict__ gU, double* __restrict__ gs) {
  const int ncol = nxt + nu + 1;
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long e = g / ncol;
  if (e >= n) return;
  const int c = (int)(g - e * ncol);
  const int2 en = entries[e];
  const DevInst I = inst[en.x];
  const DevInst W = inst_ws[en.x];
  const long k = en.y, N = I.N;
  const double* wk = w + I.v + k * nxt;
  const double* rk = rho + I.p + k * nc;
  auto lam = [&](const double* wv, const double* rv, int r) {
    double v = wv[r];
    if (r >= pen0 && r < pen0 + nc) v += rv[r - pen0];
    return v;
  };
  // block values are widened on the integer pipe (the FP64 pipe bounds this)
  auto dot = [&](const TP* col, int stride, const double* wv, const double* rv) {
    double acc = 0.0;
    for (int r = 0; r < nxt; ++r) acc = fma(widen(col[(size_t)r * stride]), lam(wv, rv, r), acc);
    return acc;
  };
  if (c < nxt) {
    double acc = dot(A + W.a + k * nxt * nxt + c, nxt, wk, rk);
    if (c >= pen0 && c < pen0 + nc) acc -= rk[c - pen0];
    if (k >= 1) acc -= wk[c - nxt];
    gX[I.x + k * nxt + c] = acc;
    if (k == N - 1) gX[I.x + N * nxt + c] = -wk[c];
  } else if (c < nxt + nu) {
    const int q = c - nxt;
    const double am = dot(Bm + W.b + k * nxt * nu + q, nu, wk, rk);
    if (layout == CISCVX_FOH_INTERVAL) {
      gU[I.u + (2 * k) * nu + q] = am;
      gU[I.u + (2 * k + 1) * nu + q] = dot(Bp + W.b + k * nxt * nu + q, nu, wk, rk);
    } else {
      // node k: B-_k^T lambda_k + B+_{k-1}^T lambda_{k-1}; node N: B+_{N-1}^T lambda_{N-1}
      const double prev = k > 0 ? dot(Bp + W.b + (k - 1) * nxt * nu + q, nu, wk - nxt, rk - nc) : 0.0;
      gU[I.u + k * nu + q] = am + prev;
      if (k == N - 1) gU[I.u + (k + 1) * nu + q] = dot(Bp + W.b + k * nxt * nu + q, nu, wk, rk);
    }
  } else {
    gs[I.s + k] = dot(S + W.v + k * nxt, 1, wk, rk);
  }
}

// L of one listed instance per block, in a fixed order.
__global__ void __launch_bounds__(256) k_contract_L_batch(const DevModel* const* models, const DevInst* inst,
                                                          const DevInst* inst_ws, const int* list,
                                                          const double* __restrict__ defect,
                                                          const double* __restrict__ penalty,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ rho, double* L) {
  __shared__ double red[256];
  const int i = list[blockIdx.x];
  const DevInst I = inst[i], W = inst_ws[i];
  const DevModel& M = *models[I.model];
  const long nd = (long)I.N * M.nxt, np = (long)I.N * M.nc;
  double acc = 0.0;
  for (long e = threadIdx.x; e < nd + np; e += 256)
    acc = e < nd ? fma(w[I.v + e], defect[W.v + e], acc) : fma(rho[I.p + e - nd], penalty[W.p + e - nd], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) L[i] = red[0];
}

}  // namespace

cudaError_t launch_contract_batch(const DevModel& Mh, const DevInst* inst, const DevInst* inst_ws,
                                  const int2* entries, long n_entries, int prec, int layout, const void* A,
                                  const void* Bm, const void* Bp, const void* S, const double* w,
                                  const double* rho, double* gX, double* gU, double* gs, cudaStream_t st) {
  if (n_entries == 0) return cudaSuccess;
  const int nxt = Mh.nxt, nu = Mh.nu, nc = Mh.nc;
  const int pen0 = 6 * Mh.nb + (Mh.aux ? 4 * nc : 0);
  const long threads = n_entries * (nxt + nu + 1);
  const int bs = 128;
  const unsigned grid = (unsigned)((threads + bs - 1) / bs);
  if (prec == CISCVX_FP64)
    k_contract_batch<double><<<grid, bs, 0, st>>>(nxt, nu, nc, pen0, n_entries, layout, inst, inst_ws, entries,
                                                  (const double*)A, (const double*)Bm, (const double*)Bp,
                                                  (const double*)S, w, rho, gX, gU, gs);
  else
    k_contract_batch<float><<<grid, bs, 0, st>>>(nxt, nu, nc, pen0, n_entries, layout, inst, inst_ws, entries,
                                                 (const float*)A, (const float*)Bm, (const float*)Bp,
                                                 (const float*)S, w, rho, gX, gU, gs);
  return cudaGetLastError();
}

cudaError_t launch_contract_L_batch(const DevModel* const* models, const DevInst* inst, const DevInst* inst_ws,
                                    const int* list, int n_list, const double* defect, const double* penalty,
                                    const double* w, const double* rho, double* L, cudaStream_t st) {
  if (n_list == 0) return cudaSuccess;
  k_contract_L_batch<<<n_list, 256, 0, st>>>(models, inst, inst_ws, list, defect, penalty, w, rho, L);
  return cudaGetLastError();
}

size_t contract_bytes(const DevModel& M, const CplTab* T, long n, int nsub, int prec) {
  return chunk_layout(M, T, n, nsub, prec).total;
}

cudaError_t launch_contract_vjp(const DevModel& Mh, const DevModel* dM, const CplTab* T, int N,
                                int nsub, int prec, int layout, const double* X, const double* U,
                                const double* s, const double* w, const double* rho, double* gX,
                                double* gU, double* gs, double* L, void* ws, size_t ws_bytes,
                                unsigned* status, cudaStream_t st) {
  const int nxt = Mh.nxt, nu = Mh.nu, nc = Mh.nc;
  const int pen0 = 6 * Mh.nb + (Mh.aux ? 4 * nc : 0);
  // largest chunk that fits (the caller checked that min(N, 32) intervals do)
  long lo = 1, hi = N;
  while (lo < hi) {
    const long mid = (lo + hi + 1) / 2;
    if (contract_bytes(Mh, T, mid, nsub, prec) <= ws_bytes) lo = mid; else hi = mid - 1;
  }
  const long chunk = lo;
  cudaError_t e = cudaSuccess;
  if (L) e = cudaMemsetAsync(L, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  char* base = (char*)ws;
  for (long i0 = 0; i0 < N; i0 += chunk) {
    const long n = std::min<long>(chunk, N - i0);
    const ChunkLayout Ly = chunk_layout(Mh, T, n, nsub, prec);
    void *A = base + Ly.A, *Bm = base + Ly.Bm, *Bp = base + Ly.Bp, *S = base + Ly.S;
    double* defect = (double*)(base + Ly.defect);
    double* penalty = (double*)(base + Ly.penalty);
    const double* Xc = X + i0 * nxt;
    const double* Uc = U ? (layout == CISCVX_FOH_NODE ? U + i0 * nu : U + 2 * i0 * nu) : nullptr;
    if (T)
      e = launch_coupled(*T, (int)n, nsub, prec, layout, Xc, Uc, s + i0, A, Bm, Bp, S, defect, penalty,
                         base + Ly.stage, n, status, st);
    else
      e = launch_discretize(dM, Mh.nb, (int)n, nsub, prec, layout, false, Mh.aux != 0, Xc, Uc, s + i0,
                            A, Bm, Bp, S, defect, penalty, nullptr, status, st);
    if (e != cudaSuccess) return e;
    const long threads = n * (nxt + nu + 1);
    const int bs = 128;
    if (prec == CISCVX_FP64)
      k_contract<double><<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(
          nxt, nu, nc, pen0, i0, n, N, layout, (const double*)A, (const double*)Bm,
          (const double*)Bp, (const double*)S, w, rho, gX, gU, gs);
    else
      k_contract<float><<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(
          nxt, nu, nc, pen0, i0, n, N, layout, (const float*)A, (const float*)Bm,
          (const float*)Bp, (const float*)S, w, rho, gX, gU, gs);
    if (L) {
      double* part = (double*)(base + Ly.part);
      const long tot = n * (nxt + nc);
      const int nblk = (int)std::min<long>(LRED_BLOCKS, (tot + 2047) / 2048);
      k_contract_L<<<nblk, 256, 0, st>>>(nxt, nc, i0, n, defect, penalty, w, rho, part);
      k_contract_L_sum<<<1, 256, 0, st>>>(part, nblk, L);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ciscvx
