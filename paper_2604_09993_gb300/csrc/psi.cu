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
// The FP64 pipe (two lanes per SM per clock on this part) and HBM bound the
// kernel with times of the same order, so the FP64 work is laid out without
// divergence and the writes are coalesced:
//  * one thread per (interval, contact) evaluates that contact's rows (two FB
//    rows and one path row, or one path row), so every lane of a warp runs
//    the same FP64 instructions;
//  * the block keeps only the values and the two slopes of each FB row in
//    shared memory (a few dozen bytes per contact), and then writes its
//    intervals' slice of psi and of the dense Jacobian, which are contiguous,
//    with consecutive threads on consecutive 16-byte pairs; each Jacobian
//    entry is formed from its (interval, row, column) index and that table.
#include <cstdint>

#include "common.cuh"

namespace ciscvx {

namespace {

constexpr int PSI_THREADS = 256;

// Intervals per block: one thread per (interval, contact), rounded down to an
// even count so that every block's slice of psi and dpsi starts on a 16-byte
// boundary when the arrays do.
__host__ __device__ inline int psi_block_intervals(int nc) {
  int ib = PSI_THREADS / nc;
  if (ib > 1) ib &= ~1;
  return ib < 1 ? 1 : ib;
}

// floor(e / d) for 0 <= e < 2^22 and d >= 1 from the FP32 reciprocal rd = 1/d
// (rounded): (e + 1/2)/d lies at least 1/(2d) from every integer, and the two
// FP32 roundings move it by at most 2^-23 (e + 1/2)/d < 1/(2d).
__device__ __forceinline__ int div_small(int e, float rd) {
  return __float2int_rz(__fmul_rn(__int2float_rn(e) + 0.5f, rd));
}

// non-finite test on the exponent bits (integer pipe)
__device__ __forceinline__ bool nonfinite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}

struct PsiShape {
  int nx, nxt, nc, ny, npsi, aux;
  float r_rowlen, r_ny;  // 1/(n_psi n_y), 1/n_y in FP32 (see div_small)
};

// Entry e of a block's Jacobian slice [nk][n_psi][n_y]; sj holds the slopes
// (da, db) of the two FB rows of each (interval, contact) of the block.
__device__ __forceinline__ double dpsi_entry(const PsiShape& p, const double* sj, int e) {
  const int kk = div_small(e, p.r_rowlen);
  const int rem = e - kk * p.npsi * p.ny;
  const int r = div_small(rem, p.r_ny);
  const int c = rem - r * p.ny;
  if (!p.aux) return c == r ? 1.0 : 0.0;
  if (r >= 2 * p.nc) return c == 4 * p.nc + (r - 2 * p.nc) ? 1.0 : 0.0;
  const int ja = 2 * r;  // 4 (r >> 1) + 2 (r & 1)
  if (c != ja && c != ja + 1) return 0.0;
  return sj[(kk * p.nc + (r >> 1)) * 4 + 2 * (r & 1) + (c - ja)];
}

__global__ void __launch_bounds__(PSI_THREADS) k_psi(PsiShape p, long N, const double* __restrict__ Xp,
                                                     const double* __restrict__ Xm, double delta,
                                                     double eps, double* __restrict__ psi,
                                                     double* __restrict__ dpsi, int vec,
                                                     unsigned* status) {
  extern __shared__ double sh[];
  const int nc = p.nc, npsi = p.npsi;
  const int ib = psi_block_intervals(nc);
  const long k0 = (long)blockIdx.x * ib;
  const int nk = (int)(N - k0 < ib ? N - k0 : ib);
  double* sv = sh;                      // [nk][n_psi] values
  double* sj = sh + (size_t)ib * npsi;  // [nk][n_c][4] slopes (da, db) of the two FB rows
  const int t = threadIdx.x;
  bool bad = false;
  for (int u = t; u < nk * nc; u += PSI_THREADS) {
    const int kk = u / nc, i = u - kk * nc;
    const long k = k0 + kk;
    const double* yp = Xp + k * p.nxt + p.nx;
    const double* ym = Xm + (k + 1) * p.nxt + p.nx;
    double* v = sv + (size_t)kk * npsi;
    if (p.aux) {
      double* s4 = sj + (size_t)u * 4;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ja = 4 * i + 2 * q;
        const double a = ym[ja] - yp[ja], b = ym[ja + 1] - yp[ja + 1];
        // one reciprocal square root gives both sqrt(x) = x / sqrt(x) and 1/sqrt(x)
        const double x = fma(a, a, fma(b, b, delta));
        const double iq = rsqrt(x);
        const double val = (a + b) - x * iq;
        s4[2 * q] = fma(-a, iq, 1.0);
        s4[2 * q + 1] = fma(-b, iq, 1.0);
        v[2 * i + q] = val;
        bad |= nonfinite_bits(val);
      }
      const int jp = 4 * nc + i;
      const double val = (ym[jp] - yp[jp]) - eps;
      v[2 * nc + i] = val;
      bad |= nonfinite_bits(val);
    } else {
      const double val = (ym[i] - yp[i]) - eps;
      v[i] = val;
      bad |= nonfinite_bits(val);
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  __syncthreads();
  const int nv = nk * npsi;
  double* gv = psi + k0 * npsi;
  for (int e = t; e < nv; e += PSI_THREADS) gv[e] = sv[e];
  if (!dpsi) return;
  double* gd = dpsi + k0 * npsi * p.ny;
  const int nd = nv * p.ny;
  int e0 = 0;
  if (vec) {  // the slice starts on a 16-byte boundary: pairs of entries
    double2* gd2 = reinterpret_cast<double2*>(gd);
    for (int q = t; q < nd / 2; q += PSI_THREADS)
      gd2[q] = make_double2(dpsi_entry(p, sj, 2 * q), dpsi_entry(p, sj, 2 * q + 1));
    e0 = nd & ~1;
  }
  for (int e = e0 + t; e < nd; e += PSI_THREADS) gd[e] = dpsi_entry(p, sj, e);
}

}  // namespace

int psi_rows(const DevModel& M) { return M.aux ? 3 * M.nc : M.nc; }

cudaError_t launch_psi(const DevModel& M, int N, const double* Xp, const double* Xm, double delta,
                       double eps, double* psi, double* dpsi, unsigned* status, cudaStream_t st) {
  PsiShape p;
  p.nx = 6 * M.nb;
  p.nxt = M.nxt;
  p.nc = M.nc;
  p.ny = M.nxt - p.nx;
  p.npsi = psi_rows(M);
  p.aux = M.aux ? 1 : 0;
  if (p.npsi == 0 || N == 0) return cudaSuccess;
  const int ib = psi_block_intervals(p.nc);
  // div_small's range: a block's Jacobian slice has ib n_psi n_y < 2^22
  // entries (at most 8 * 96 * 160 for 32 contacts)
  p.r_rowlen = 1.0f / (float)(p.npsi * p.ny);
  p.r_ny = 1.0f / (float)p.ny;
  const size_t smem = (size_t)ib * (p.npsi + 4 * p.nc) * sizeof(double);
  const long blocks = (N + ib - 1) / ib;
  // every block slice starts at an even entry (ib even, or ib == 1 with an
  // even row length); pairs are stored when dpsi itself is 16-byte aligned
  const int vec = dpsi && ((reinterpret_cast<uintptr_t>(dpsi) & 15) == 0) &&
                  (ib % 2 == 0 || (p.npsi * p.ny) % 2 == 0);
  k_psi<<<(unsigned)blocks, PSI_THREADS, smem, st>>>(p, N, Xp, Xm, delta, eps, psi, dpsi, vec,
                                                     status);
  return cudaGetLastError();
}

}  // namespace ciscvx
