// psi.cu — Psi^{delta,eps}(y-_{k+1}, y+_k) <= 0 of Eq. (17c) on every grid
// interval, with its Jacobian.  Psi depends on the auxiliary-state increment
// d = y-_{k+1} - y+_k alone:
//   Eq. (12) auxiliary state (per contact i the integrals of phi_n, lambda^c,
//   gamma, rho^c at y index 4i..4i+3, the path penalty at 4 n_c + i):
//     row 2i     FB(d[4i], d[4i+1])       (phi_n, lambda^c), Eq. (11) relaxed by Eq. (16)
//     row 2i+1   FB(d[4i+2], d[4i+3])     (gamma, rho^c)
//     row 2n_c+i d[4 n_c + i] - eps        relaxed path constraint, Eq. (13)
//   one path-penalty state per contact: row i = d[i] - eps.
// FB(a, b) = a + b - sqrt(a^2 + b^2 + delta); dFB/da = 1 - a / sqrt(.).
//
// One thread per row (interval k, row r) evaluates FB once and writes its
// value and its dense Jacobian row into shared memory; the block then copies
// its intervals' rows, which are contiguous in psi and dpsi, to global memory
// with consecutive threads on consecutive doubles.  8 (2 n_y + n_psi (1 + n_y))
// bytes per interval against about 20 FP64 operations per FB row: on this
// part's FP64 rate the two bounds are of the same order.
#include "common.cuh"

namespace ciscvx {

namespace {

constexpr int PSI_THREADS = 256;
constexpr int PSI_SMEM = 48 * 1024;  // staging per block (no opt-in needed)

// Intervals one block stages: as many as fit, at most one per thread row.
__host__ __device__ inline int psi_block_intervals(int npsi, int ny) {
  const int per = npsi * (ny + 1) * (int)sizeof(double);
  int ib = PSI_SMEM / per;
  if (ib * npsi > PSI_THREADS) ib = PSI_THREADS / npsi;
  return ib < 1 ? 1 : ib;
}

__global__ void __launch_bounds__(PSI_THREADS) k_psi(int nx, int nxt, int nc, int aux, long N,
                                                     const double* __restrict__ Xp,
                                                     const double* __restrict__ Xm, double delta,
                                                     double eps, double* __restrict__ psi,
                                                     double* __restrict__ dpsi, unsigned* status) {
  extern __shared__ double sh[];
  const int ny = nxt - nx, npsi = aux ? 3 * nc : nc;
  const int ib = psi_block_intervals(npsi, ny);
  const long k0 = (long)blockIdx.x * ib;
  const int nk = (int)(N - k0 < ib ? N - k0 : ib);
  double* sv = sh;                      // [nk][npsi] values
  double* sd = sh + (size_t)ib * npsi;  // [nk][npsi][ny] Jacobian rows
  const int t = threadIdx.x;
  if (t < nk * npsi) {
    const int kk = t / npsi, r = t - kk * npsi;
    const long k = k0 + kk;
    const double* yp = Xp + k * nxt + nx;
    const double* ym = Xm + (k + 1) * nxt + nx;
    int ja, jb = -1;
    if (aux && r < 2 * nc) {
      ja = 4 * (r >> 1) + 2 * (r & 1);
      jb = ja + 1;
    } else {
      ja = aux ? 4 * nc + (r - 2 * nc) : r;
    }
    const double a = ym[ja] - yp[ja];
    double val, da = 1.0, db = 0.0;
    if (jb >= 0) {
      const double b = ym[jb] - yp[jb];
      // one reciprocal square root gives both q and 1/q (the FP64 pipe, two
      // lanes per SM per clock on this part, bounds the kernel with HBM)
      const double x = fma(a, a, fma(b, b, delta));
      const double iq = rsqrt(x);
      val = (a + b) - x * iq;
      da = fma(-a, iq, 1.0);
      db = fma(-b, iq, 1.0);
    } else {
      val = a - eps;
    }
    if (!isfinite(val)) atomicOr(status, ST_NONFINITE);
    sv[t] = val;
    double* row = sd + (size_t)t * ny;
    for (int c = 0; c < ny; ++c) row[c] = c == ja ? da : (c == jb ? db : 0.0);
  }
  __syncthreads();
  const long nv = (long)nk * npsi;
  double* gv = psi + k0 * npsi;
  for (long e = t; e < nv; e += PSI_THREADS) gv[e] = sv[e];
  if (dpsi) {
    double* gd = dpsi + k0 * npsi * ny;
    for (long e = t; e < nv * ny; e += PSI_THREADS) gd[e] = sd[e];
  }
}

}  // namespace

int psi_rows(const DevModel& M) { return M.aux ? 3 * M.nc : M.nc; }

cudaError_t launch_psi(const DevModel& M, int N, const double* Xp, const double* Xm, double delta,
                       double eps, double* psi, double* dpsi, unsigned* status, cudaStream_t st) {
  const int nx = 6 * M.nb, ny = M.nxt - nx, npsi = psi_rows(M);
  if (npsi == 0 || N == 0) return cudaSuccess;
  const int ib = psi_block_intervals(npsi, ny);
  const size_t smem = (size_t)ib * npsi * (ny + 1) * sizeof(double);
  const long blocks = (N + ib - 1) / ib;
  k_psi<<<(unsigned)blocks, PSI_THREADS, smem, st>>>(nx, M.nxt, M.nc, M.aux ? 1 : 0, N, Xp, Xm, delta,
                                                     eps, psi, dpsi, status);
  return cudaGetLastError();
}

}  // namespace ciscvx
