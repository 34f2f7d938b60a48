// vjp.cu — vector-Jacobian product of L = sum_k w_k . defect_k + sum_k rho_k . penalty_k.
//
// defect_k = F~(x~_k, U_k, s_k) - x~_{k+1} (Eq. (17b)), penalty_k = y(1) - y_k.
// The gradient is the discrete adjoint of the RK4 substeps (the exact
// derivative of the same discrete map the forward kernel linearizes): a
// forward sweep checkpoints (theta, omega) — and for a foot link (p_y, v_y) —
// at every substep start; the backward sweep recomputes the four stages of a
// substep from its checkpoint and applies the transposed stage Jacobians.
// Translation uses the transposed closed forms.
//
// Mapping as in the forward kernel: one warp = 32 intervals x one link.  Each
// lane writes its link's rows of gX directly and its per-input partials (the
// link's share of dL/du_L, dL/du_R), its share of dL/ds and of L to the
// workspace; k_vjp_gu / k_vjp_gs / k_vjp_L sum the partials in a fixed order (no atomics),
// including the node-layout sum dL/dU_k = (u_L part of interval k) + (u_R part
// of interval k-1).
#include "vjp_link.cuh"

namespace ciscvx {

// Workspace layout (doubles): part [N][nslot][2], ps [N][nb], pL [N][nb], Lblk [nblk].
struct VjpWs {
  double* part;
  double* ps;
  double* pL;
  double* Lblk;
};

constexpr int FIN_THREADS = 256;

__host__ __device__ inline VjpWs vjp_ws_split(void* ws, int nb, int nslot, long N) {
  double* base = (double*)ws;
  VjpWs w;
  w.part = base;
  w.ps = w.part + (size_t)N * nslot * 2;
  w.pL = w.ps + (size_t)N * nb;
  w.Lblk = w.pL + (size_t)N * nb;
  return w;
}

size_t vjp_workspace_bytes(int nb, int nu, int nslot, int N, int layout) {
  (void)nu; (void)layout;
  const size_t nblk = ((size_t)N + FIN_THREADS - 1) / FIN_THREADS;
  return sizeof(double) * ((size_t)N * nslot * 2 + 2 * (size_t)N * nb + nblk);
}

// AUX: the model uses the Eq. (12) auxiliary state (its foot links take the
// CROSS adjoint; a separate instantiation keeps those registers out of the
// common kernel).
template <typename TP, bool AUX>
__global__ void __launch_bounds__(128) k_vjp(const DevModel* __restrict__ Mp, int N, int nsub,
                                             int layout, const double* __restrict__ X,
                                             const double* __restrict__ U,
                                             const double* __restrict__ s,
                                             const double* __restrict__ w,
                                             const double* __restrict__ rho, double* gX,
                                             VjpWs ws, unsigned* status) {
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
  const DevBody& B = M.body[b];
  const double rc = (B.contact >= 0) ? rho[k * nc + B.contact] : 0.0;
  const double* wkm1 = (k > 0) ? w + (k - 1) * nxt : nullptr;
  double* gXN = (k == N - 1) ? gX + (size_t)N * nxt : nullptr;
  double* part = ws.part + (size_t)k * M.nslot * 2;
  if (AUX && B.contact >= 0)
    vjp_link<TP, true, false, true>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL, uR,
                                    w + k * nxt, wkm1, rc, gX + (size_t)k * nxt, gXN, part,
                                    ws.ps + k * nb, ws.pL + k * nb, status);
  else if (B.contact >= 0)
    vjp_link<TP, true>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL, uR, w + k * nxt,
                       wkm1, rc, gX + (size_t)k * nxt, gXN, part, ws.ps + k * nb, ws.pL + k * nb,
                       status);
  else
    vjp_link<TP, false>(M, b, nsub, s[k], X + k * nxt, X + (k + 1) * nxt, uL, uR, w + k * nxt,
                        wkm1, rc, gX + (size_t)k * nxt, gXN, part, ws.ps + k * nb,
                        ws.pL + k * nb, status);
}

// dL/dU from the per-link partials (fixed summation order).  One thread per (node or interval, input).
__global__ void k_vjp_gu(const DevModel* __restrict__ Mp, int N, int layout, VjpWs ws,
                         double* __restrict__ gU) {
  const DevModel& M = *Mp;
  const int nu = M.nu, nslot = M.nslot;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nrow = (layout == CISCVX_FOH_NODE) ? (long)N + 1 : 2L * N;
  if (idx >= nrow * nu) return;
  const long r = idx / nu;
  const int q = (int)(idx - r * nu);
  const int n = M.in_n[q];
  auto sum_side = [&](long k, int side) {
    const double* p = ws.part + (size_t)k * nslot * 2;
    double v = 0.0;
    for (int t = 0; t < n; ++t) v += p[2 * M.in_slot[q][t] + side];
    return v;
  };
  double v;
  if (layout == CISCVX_FOH_NODE) {
    v = 0.0;
    if (r < N) v += sum_side(r, 0);        // u_L of interval r
    if (r > 0) v += sum_side(r - 1, 1);    // u_R of interval r-1
  } else {
    v = sum_side(r >> 1, (int)(r & 1));
  }
  gU[idx] = v;
}

// dL/ds_k and block sums of L.
__global__ void __launch_bounds__(FIN_THREADS) k_vjp_gs(int nb, int N, VjpWs ws,
                                                        double* __restrict__ gs) {
  __shared__ double red[FIN_THREADS];
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double Lk = 0.0;
  if (k < N) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) { v += ws.ps[k * nb + b]; Lk += ws.pL[k * nb + b]; }
    gs[k] = v;
  }
  red[threadIdx.x] = Lk;
  __syncthreads();
  for (int o = FIN_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ws.Lblk[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(FIN_THREADS) k_vjp_L(int nblk, const double* __restrict__ Lblk,
                                                       double* __restrict__ L) {
  __shared__ double red[FIN_THREADS];
  double v = 0.0;
  for (int i = threadIdx.x; i < nblk; i += FIN_THREADS) v += Lblk[i];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = FIN_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *L = red[0];
}

cudaError_t launch_vjp(const DevModel* dM, int nb, int nxt, int nu, int nslot, int N, int nsub,
                       int prec, int layout, const double* X, const double* U, const double* s,
                       const double* w, const double* rho, double* gX, double* gU, double* gs,
                       double* L, void* ws_ptr, unsigned* status, bool aux, cudaStream_t st) {
  (void)nxt;
  VjpWs ws = vjp_ws_split(ws_ptr, nb, nslot, N);
  const long warps = (long)((N + 31) / 32) * nb;
  const int threads = single_cta_threads(warps);
  const long blocks = (warps * 32 + threads - 1) / threads;
#define CISCVX_KVJP(TP, AUX)                                                                     \
  k_vjp<TP, AUX><<<(unsigned)blocks, threads, 0, st>>>(dM, N, nsub, layout, X, U, s, w, rho, gX, ws, \
                                                       status)
  if (prec == CISCVX_FP64) {
    if (aux) CISCVX_KVJP(double, true); else CISCVX_KVJP(double, false);
  } else {
    if (aux) CISCVX_KVJP(float, true); else CISCVX_KVJP(float, false);
  }
#undef CISCVX_KVJP
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nu > 0) {
    const long nrow = (layout == CISCVX_FOH_NODE) ? (long)N + 1 : 2L * N;
    const long tot = nrow * nu;
    k_vjp_gu<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dM, N, layout, ws, gU);
  }
  const int nblk = (N + FIN_THREADS - 1) / FIN_THREADS;
  k_vjp_gs<<<nblk, FIN_THREADS, 0, st>>>(nb, N, ws, gs);
  if (L) k_vjp_L<<<1, FIN_THREADS, 0, st>>>(nblk, ws.Lblk, L);
  return cudaGetLastError();
}

}  // namespace ciscvx
