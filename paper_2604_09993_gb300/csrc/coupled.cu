// coupled.cu — linearized discretization (Eqs. (14)-(15), (17b); IND with a
// first-order hold, Sec. VI) for models whose links are coupled within an
// interval: joint reaction forces eliminated by Eq. (3), the sinusoidal
// contact surface of Sec. VI-B, the Runge-Kutta-Fehlberg tableau (see
// coupled.cuh for the row classes).
//
// Two kernels per chunk of intervals, joined by a stage-data buffer:
//  * k_cpl_nominal — lane = interval, FP64.  Integrates the state with the
//    scheme's stages.  At every stage it evaluates the right-hand side: lever
//    arms, contact frames and forces, the generalized forces, and with
//    elimination the L D L^T factor of K = grad C M^-1 grad C^T and the
//    reaction forces lambda = K^-1 (kappa - grad C M^-1 F), kappa_j =
//    omega_c^2 r_c - omega_p^2 r_p.  It records, per stage, what the
//    tangents need (the right-hand side, lever arms, the factor, contact
//    frames and penalty slopes) and writes defects and penalty increments.
//  * k_cpl_tangent — thread = (interval, tangent column).  Integrates one
//    column of [A | B- | B+ | S] with the same stages from the recorded data.
//    Per stage, the derivative of the right-hand side along the column's
//    stage tangent: with e = dF + dgrad C^T lambda (the generalized-force
//    tangent), the reaction-force tangent solves
//      K dlambda = sum over joint ends s (2 omega r domega + (omega^2 r_perp +
//                  omega' r) dtheta - e_lin / m - r_perp e_ang / I)
//    with the recorded factor, and dv' = M^-1 (e + grad C^T dlambda).
// The FP64 state work runs one interval per lane, so every FP64 instruction
// has 32 useful lanes; the tangent work (n_x~ + 2 n_u + 1 columns per
// interval) runs one column per thread in the tangent precision.  Per-lane /
// per-thread arrays live in shared memory, element major, so a warp's access
// to one element is one contiguous row.
#include <algorithm>
#include <type_traits>
#include <cstring>

#include "coupled.cuh"

namespace ciscvx {

namespace {

template <int SCH>
struct Scheme {
  static constexpr int S = SCH ? 6 : 4;    // stages
  static constexpr int NKS = SCH ? 5 : 1;  // stored slopes per row (RK4 only reads the previous one)
  __device__ static constexpr int slot(int l) { return NKS == 1 ? 0 : l; }
  // nonzero weights (Fehlberg's fifth-order weights skip the second stage)
  __device__ static constexpr bool bnz(int m) { return SCH ? m != 1 : true; }
};

// pseudo-Huber absolute value sqrt(1 + x^2) - 1 and its slope
__device__ __forceinline__ double sabs_d(double x, double& d) {
  const double r = sqrt(fma(x, x, 1.0));
  d = x / r;
  return r - 1.0;
}

// pseudo-Huber ramp h(z) and slope h'(z)
__device__ __forceinline__ double ramp_d(double z, double& d) {
  double H;
  huber(z, H, d);
  return H;
}

// Tableau constants and link inverses in the precision of the arithmetic
// that uses them (FP32 copies keep conversions out of the FP32 loops).
template <typename TP>
struct Cst {
  __device__ static double a(const CplTab& M, int j, int l) { return M.a[j][l]; }
  __device__ static double b(const CplTab& M, int j) { return M.b[j]; }
  __device__ static double c(const CplTab& M, int j) { return M.c[j]; }
  __device__ static double beta(const CplTab& M, int j) { return M.beta[j]; }
  __device__ static double minv(const CplTab& M, int b) { return M.minv[b]; }
  __device__ static double iinv(const CplTab& M, int b) { return M.iinv[b]; }
};
template <>
struct Cst<float> {
  __device__ static float a(const CplTab& M, int j, int l) { return M.af[j][l]; }
  __device__ static float b(const CplTab& M, int j) { return M.bf[j]; }
  __device__ static float c(const CplTab& M, int j) { return M.cf[j]; }
  __device__ static float beta(const CplTab& M, int j) { return M.betaf[j]; }
  __device__ static float minv(const CplTab& M, int b) { return M.minvf[b]; }
  __device__ static float iinv(const CplTab& M, int b) { return M.iinvf[b]; }
};

// Where interval e's data live: for a single instance (entries null) interval
// e itself; in a batch, entry e = (instance, k) of the batch's instance table.
// a_stride: elements of A per interval (n_x~^2 dense, colptr[n_x~] compact).
struct IvAddr {
  const double *x0, *x1, *uL, *uR;
  long long s, a, b, v, p;  // element offsets: s, A, Bm/Bp, S/defect, penalty
};

__device__ __forceinline__ IvAddr iv_addr(long e, int nxt, int nu, int nc, int layout,
                                          const double* X, const double* U, const int2* entries,
                                          const DevInst* inst, long long a_stride) {
  long long k = e, xo, uo;
  IvAddr r;
  if (entries) {
    const int2 en = entries[e];
    const DevInst& I = inst[en.x];
    k = en.y;
    xo = I.x + k * nxt;
    uo = I.u + (layout == 0 ? k : 2 * k) * nu;
    r.s = I.s + k;
    r.a = I.a + k * a_stride;
    r.b = I.b + k * nxt * nu;
    r.v = I.v + k * nxt;
    r.p = I.p + k * nc;
  } else {
    xo = k * nxt;
    uo = (layout == 0 ? k : 2 * k) * nu;
    r.s = k;
    r.a = k * a_stride;
    r.b = k * nxt * nu;
    r.v = k * nxt;
    r.p = k * nc;
  }
  r.x0 = X + xo;
  r.x1 = r.x0 + nxt;
  r.uL = U ? U + uo : nullptr;
  r.uR = U ? U + uo + nu : nullptr;
  return r;
}

#define EL(o) sm[(o) * 32]
#define LK(i, kk) EL(M.n_K + M.noff[i] + (kk) - M.nf[i])

template <typename TP, int SCH>
__global__ void __launch_bounds__(32) k_cpl_nominal(const __grid_constant__ CplTab M, long i0,
                                                    long n, int nsub, int layout,
                                                    const double* __restrict__ X,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ s,
                                                    TP* __restrict__ sd, TP* __restrict__ A,
                                                    double* __restrict__ defect,
                                                    double* __restrict__ penalty, unsigned* status,
                                                    const int2* __restrict__ entries,
                                                    const DevInst* __restrict__ inst, int cmp) {
  using Sc = Scheme<SCH>;
  constexpr int NS = Sc::S;
  extern __shared__ double smem1[];
  const long t = (long)blockIdx.x * 32 + threadIdx.x;
  if (t >= n) return;
  double* sm = smem1 + threadIdx.x;
  const int nb = M.nb, nj = M.nj, nc = M.nc, nxt = M.nxt, nu = M.nu, nq = 3 * nb, nk = M.nk;
  const int nl = M.nlive;
  const IvAddr ad = iv_addr(i0 + t, nxt, nu, nc, layout, X, U, entries, inst,
                            cmp ? (long long)M.colptr[nxt] : (long long)nxt * nxt);
  const double* uL = ad.uL;
  const double* uR = ad.uR;
  const double sk = s[ad.s];
  const double h = 1.0 / nsub;
  for (int r = 0; r < nxt; ++r) {
    const double v = ad.x0[r];
    if (M.lrow[r] >= 0) EL(M.n_xl + M.lrow[r]) = v;
    else EL(M.n_xq + M.qrow[r]) = v;
  }
  TP* sdk = sd + (size_t)t * nsub * NS * M.sd_size;
  // stage value of state row r (live rows only)
#define XS(r) EL(M.n_xs + M.lrow[r])

  for (int i = 0; i < nsub; ++i) {
    // quadrature rows: p += h s v at the substep start (the rest below)
    for (int b = 0; b < nb; ++b) {
      if (M.contact[b] >= 0) continue;
      for (int c2 = 0; c2 < 2; ++c2)
        EL(M.n_xq + M.qrow[3 * b + c2]) = fma(h * sk, EL(M.n_xq + M.qrow[nq + 3 * b + c2]),
                                              EL(M.n_xq + M.qrow[3 * b + c2]));
    }
    for (int j = 0; j < NS; ++j) {
      const double tau = (i + M.c[j]) * h;
      const double bj = M.b[j];
      const double h2b = h * h * sk * M.beta[j];
      TP* D = sdk + (size_t)(i * NS + j) * M.sd_size;
      for (int l = 0; l < nl; ++l) EL(M.n_xs + l) = EL(M.n_xl + l);
      for (int m = 0; m < j; ++m) {
        const double ah = M.a[j][m] * h;
        if (ah == 0.0) continue;
        for (int l = 0; l < nl; ++l)
          EL(M.n_xs + l) = fma(ah, EL(M.n_k + Sc::slot(m) * nl + l), EL(M.n_xs + l));
      }
      auto u_at = [&](int q) { return (1.0 - tau) * uL[q] + tau * uR[q]; };
      // records F_r and integrates row r with the slope s F_r
      auto emit = [&](int r, double F) {
        const int l = M.lrow[r];
        D[M.sd_F + r] = TP(F);
        const double kv = sk * F;
        if (l >= 0) {
          if (Sc::NKS == 1) {
            if (j < NS - 1) EL(M.n_k + l) = kv;
            EL(M.n_acc + l) = (j == 0) ? bj * kv : fma(bj, kv, EL(M.n_acc + l));
            if (j == NS - 1) EL(M.n_xl + l) = fma(h, EL(M.n_acc + l), EL(M.n_xl + l));
          } else if (j < NS - 1) {
            EL(M.n_k + Sc::slot(j) * nl + l) = kv;
          } else {  // last stage: x += h sum_m b_m k_m from the stored slopes
            double acc = bj * kv;
            for (int m = NS - 2; m >= 0; --m)
              if (Sc::bnz(m)) acc = fma(M.b[m], EL(M.n_k + Sc::slot(m) * nl + l), acc);
            EL(M.n_xl + l) = fma(h, acc, EL(M.n_xl + l));
          }
        } else {
          const int q = M.qrow[r];
          EL(M.n_xq + q) = fma(h * bj, kv, EL(M.n_xq + q));
          // a velocity row of a link without a contact also moves its position:
          // p += h^2 s beta_j k_v (p += h s v was added at the substep start)
          if (r >= nq && r < 2 * nq && (r - nq) % 3 != 2) {
            const int qp = M.qrow[r - nq];
            EL(M.n_xq + qp) = fma(h2b, kv, EL(M.n_xq + qp));
          }
        }
      };
      // lever arms r = R(theta) rho of every joint end and contact point
      for (int b = 0; b < nb; ++b) {
        double sn, cs;
        sincos(XS(3 * b + 2), &sn, &cs);
        for (int tt = 0; tt < M.nadj[b]; ++tt) {
          const int code = M.adj[b][tt], jj = code >> 1, role = code & 1;
          const double* rho = role ? M.jrp[jj] : M.jrc[jj];
          const double rx = fma(cs, rho[0], -sn * rho[1]), ry = fma(sn, rho[0], cs * rho[1]);
          EL(M.n_arm + 4 * jj + 2 * role) = rx;
          EL(M.n_arm + 4 * jj + 2 * role + 1) = ry;
          D[M.sd_arm + 4 * jj + 2 * role] = TP(rx);
          D[M.sd_arm + 4 * jj + 2 * role + 1] = TP(ry);
        }
        const int ic = M.contact[b];
        if (ic >= 0) {
          EL(M.n_carm + 2 * ic) = fma(cs, M.crho[ic][0], -sn * M.crho[ic][1]);
          EL(M.n_carm + 2 * ic + 1) = fma(sn, M.crho[ic][0], cs * M.crho[ic][1]);
        }
      }
      // generalized forces (F_x, F_y, torque) per link; QW_b = sum r . F over
      // the forces applied at points of the link (the -dtheta coefficient of
      // the torque's derivative)
      for (int b = 0; b < nb; ++b) {
        EL(M.n_f + 3 * b) = 0.0;
        EL(M.n_f + 3 * b + 1) = -M.mass[b] * M.g;
        EL(M.n_f + 3 * b + 2) = 0.0;
        EL(M.n_qw + b) = 0.0;
      }
      for (int jj = 0; jj < nj; ++jj) {
        const int c = M.jchi[jj], p = M.jpar[jj];
        const double tq = u_at(jj);
        EL(M.n_f + 3 * c + 2) += tq;
        EL(M.n_f + 3 * p + 2) -= tq;
        if (!M.jelim) {  // reaction force as an input: +lambda on the child, -lambda on the parent
          const double lx = u_at(nj + 2 * jj), ly = u_at(nj + 2 * jj + 1);
          const double rcx = EL(M.n_arm + 4 * jj), rcy = EL(M.n_arm + 4 * jj + 1);
          const double rpx = EL(M.n_arm + 4 * jj + 2), rpy = EL(M.n_arm + 4 * jj + 3);
          EL(M.n_f + 3 * c) += lx;
          EL(M.n_f + 3 * c + 1) += ly;
          EL(M.n_f + 3 * c + 2) += fma(rcx, ly, -rcy * lx);
          EL(M.n_f + 3 * p) -= lx;
          EL(M.n_f + 3 * p + 1) -= ly;
          EL(M.n_f + 3 * p + 2) -= fma(rpx, ly, -rpy * lx);
          EL(M.n_qw + c) += fma(rcx, lx, rcy * ly);
          EL(M.n_qw + p) -= fma(rpx, lx, rpy * ly);
        }
      }
      // contacts: frame, force, auxiliary right-hand sides and their slopes
      for (int ic = 0; ic < nc; ++ic) {
        const int b = M.cbody[ic];
        const double rx = EL(M.n_carm + 2 * ic), ry = EL(M.n_carm + 2 * ic + 1);
        const SurfFrame f = contact_surface(M.ta, M.tk, XS(3 * b) + rx, XS(3 * b + 1) + ry);
        const double u0 = u_at(M.ci0 + 3 * ic), u1 = u_at(M.ci0 + 3 * ic + 1),
                     u2 = u_at(M.ci0 + 3 * ic + 2);
        // contact-frame components (tangential, normal)
        const double ft = M.aux ? u0 : u1 - u2, fn = M.aux ? u1 : u0;
        const double fx = fma(f.tx, ft, f.nx * fn), fy = fma(f.ty, ft, f.ny * fn);
        EL(M.n_f + 3 * b) += fx;
        EL(M.n_f + 3 * b + 1) += fy;
        EL(M.n_f + 3 * b + 2) += fma(rx, fy, -ry * fx);
        EL(M.n_qw + b) += fma(rx, fx, ry * fy);
        TP* Dc = D + M.sd_con + M.ncf * ic;
        Dc[0] = TP(rx); Dc[1] = TP(ry);
        Dc[2] = TP(f.tx); Dc[3] = TP(f.ty); Dc[4] = TP(f.nx); Dc[5] = TP(f.ny);
        Dc[6] = TP(fma(f.dtx, ft, f.dnx * fn));  // dF/dx_c at fixed inputs
        Dc[7] = TP(fma(f.dty, ft, f.dny * fn));
        Dc[8] = TP(f.phix); Dc[9] = TP(f.phiy);
        const double mu = M.mu[ic];
        if (!M.aux) {
          // Omega = h(-lambda_n) + h(-lambda_t+) + h(-lambda_t-) + h(-phi) + h(lambda_t+ + lambda_t- - mu lambda_n)
          double d1, d2, d3, dp, d5;
          const double H = ramp_d(-u0, d1) + ramp_d(-u1, d2) + ramp_d(-u2, d3) + ramp_d(-f.phi, dp) +
                           ramp_d(u1 + u2 - mu * u0, d5);
          Dc[10] = TP(-dp);
          Dc[11] = TP(-d1 - mu * d5);
          Dc[12] = TP(-d2 + d5);
          Dc[13] = TP(-d3 + d5);
          emit(6 * nb + ic, H);
        } else {
          // Eq. (12): phi_n, lambda^c, gamma, rho^c, then the path penalty
          const double gam = u2;
          const double om = XS(nq + 3 * b + 2);
          const double vcx = fma(-om, ry, XS(nq + 3 * b));
          const double vcy = fma(om, rx, XS(nq + 3 * b + 1));
          const double rt = 1.0 / sqrt(fma(ft, ft, 1.0));
          double dmn, dft;
          const double rho_c = sabs_d(mu * fn, dmn) - sabs_d(ft, dft);
          const double lam = fma(f.tx, vcx, f.ty * vcy) + gam * (ft * rt);
          double dfn_, dph, dga, drh;
          const double H = ramp_d(-fn, dfn_) + ramp_d(-f.phi, dph) + ramp_d(-gam, dga) +
                           ramp_d(-rho_c, drh);
          const double rho_ft = -dft, rho_fn = mu * dmn;
          Dc[10] = TP(-dph);
          Dc[11] = TP(drh * dft);             // dH/dphi_t = -h'(-rho) drho/dphi_t
          Dc[12] = TP(-dfn_ - drh * rho_fn);  // dH/dphi_n
          Dc[13] = TP(-dga);                  // dH/dgamma
          Dc[14] = TP(vcx); Dc[15] = TP(vcy);
          Dc[16] = TP(fma(f.dtx, vcx, f.dty * vcy));  // (dt/dx_c) . v_c
          Dc[17] = TP(gam * rt * rt * rt);            // dlambda^c/dphi_t
          Dc[18] = TP(ft * rt);                       // dlambda^c/dgamma
          Dc[19] = TP(rho_ft);
          Dc[20] = TP(rho_fn);
          emit(6 * nb + 4 * ic, fn);
          emit(6 * nb + 4 * ic + 1, lam);
          emit(6 * nb + 4 * ic + 2, gam);
          emit(6 * nb + 4 * ic + 3, rho_c);
          emit(6 * nb + 4 * nc + ic, H);
        }
      }
      // Eq. (3): K lambda = kappa - grad C M^-1 F, then F += grad C^T lambda
      if (M.jelim && nk > 0) {
        for (int r1 = 0; r1 < nk; ++r1) {
          const int j1 = M.nord[r1 >> 1], a1 = r1 & 1;
          for (int r2 = M.nf[r1]; r2 <= r1; ++r2) {
            const int j2 = M.nord[r2 >> 1], a2 = r2 & 1;
            double acc = 0.0;
            for (int u = 0; u < 2; ++u) {
              const int b1 = u ? M.jpar[j1] : M.jchi[j1];
              // perp(r) = (-r_y, r_x), component a1
              const double p1 = a1 ? EL(M.n_arm + 4 * j1 + 2 * u) : -EL(M.n_arm + 4 * j1 + 2 * u + 1);
              for (int v = 0; v < 2; ++v) {
                const int b2 = v ? M.jpar[j2] : M.jchi[j2];
                if (b1 != b2) continue;
                const double p2 =
                    a2 ? EL(M.n_arm + 4 * j2 + 2 * v) : -EL(M.n_arm + 4 * j2 + 2 * v + 1);
                const double e = fma(p1 * p2, M.iinv[b1], (a1 == a2) ? M.minv[b1] : 0.0);
                acc = (u == v) ? acc + e : acc - e;
              }
            }
            LK(r1, r2) = acc;
          }
        }
        // Cholesky within the envelopes (diagonal slot: 1 / L_ii), then unit
        // L = L_c diag(1 / L_c,kk) and 1/D = (1 / L_c,ii)^2
        for (int ii = 0; ii < nk; ++ii) {
          const int fi = M.nf[ii];
          for (int kk = fi; kk < ii; ++kk) {
            double acc = LK(ii, kk);
            const int m0 = fi > M.nf[kk] ? fi : M.nf[kk];
            for (int m = m0; m < kk; ++m) acc = fma(-LK(ii, m), LK(kk, m), acc);
            LK(ii, kk) = acc * LK(kk, kk);
          }
          double d = LK(ii, ii);
          for (int m = fi; m < ii; ++m) d = fma(-LK(ii, m), LK(ii, m), d);
          LK(ii, ii) = 1.0 / sqrt(d);
        }
        for (int ii = 0; ii < nk; ++ii)
          for (int kk = M.nf[ii]; kk < ii; ++kk) LK(ii, kk) *= LK(kk, kk);
        for (int ii = 0; ii < nk; ++ii) LK(ii, ii) = LK(ii, ii) * LK(ii, ii);
        for (int e = 0; e < M.nsky; ++e) D[M.sd_K + e] = TP(EL(M.n_K + e));
        // right-hand side, joints in factor order
        for (int jj = 0; jj < nj; ++jj) {
          double a0 = 0.0, a1 = 0.0;
          for (int role = 0; role < 2; ++role) {
            const int b = role ? M.jpar[jj] : M.jchi[jj];
            const double rx = EL(M.n_arm + 4 * jj + 2 * role), ry = EL(M.n_arm + 4 * jj + 2 * role + 1);
            const double om = XS(nq + 3 * b + 2);
            const double aa = EL(M.n_f + 3 * b + 2) * M.iinv[b];
            const double c0 = fma(om * om, rx, fma(ry, aa, -EL(M.n_f + 3 * b) * M.minv[b]));
            const double c1 = fma(om * om, ry, fma(-rx, aa, -EL(M.n_f + 3 * b + 1) * M.minv[b]));
            if (role) { a0 -= c0; a1 -= c1; } else { a0 += c0; a1 += c1; }
          }
          EL(M.n_lam + 2 * M.npos[jj]) = a0;
          EL(M.n_lam + 2 * M.npos[jj] + 1) = a1;
        }
        for (int ii = 1; ii < nk; ++ii) {
          double acc = EL(M.n_lam + ii);
          for (int kk = M.nf[ii]; kk < ii; ++kk) acc = fma(-LK(ii, kk), EL(M.n_lam + kk), acc);
          EL(M.n_lam + ii) = acc;
        }
        for (int ii = nk - 1; ii >= 0; --ii) {
          double acc = EL(M.n_lam + ii) * LK(ii, ii);
          for (int kk = ii + 1; kk < nk; ++kk)
            if (M.nf[kk] <= ii) acc = fma(-LK(kk, ii), EL(M.n_lam + kk), acc);
          EL(M.n_lam + ii) = acc;
        }
        for (int jj = 0; jj < nj; ++jj) {
          const double lx = EL(M.n_lam + 2 * M.npos[jj]), ly = EL(M.n_lam + 2 * M.npos[jj] + 1);
          const int c = M.jchi[jj], p = M.jpar[jj];
          const double rcx = EL(M.n_arm + 4 * jj), rcy = EL(M.n_arm + 4 * jj + 1);
          const double rpx = EL(M.n_arm + 4 * jj + 2), rpy = EL(M.n_arm + 4 * jj + 3);
          EL(M.n_f + 3 * c) += lx;
          EL(M.n_f + 3 * c + 1) += ly;
          EL(M.n_f + 3 * c + 2) += fma(rcx, ly, -rcy * lx);
          EL(M.n_f + 3 * p) -= lx;
          EL(M.n_f + 3 * p + 1) -= ly;
          EL(M.n_f + 3 * p + 2) -= fma(rpx, ly, -rpy * lx);
          EL(M.n_qw + c) += fma(rcx, lx, rcy * ly);
          EL(M.n_qw + p) -= fma(rpx, lx, rpy * ly);
        }
      }
      for (int b = 0; b < nb; ++b) D[M.sd_qw + b] = TP(EL(M.n_qw + b));
      // q' = v: live position rows take the stage velocity; a link without a
      // contact records its velocity at the substep start only (the tangent
      // kernel needs no more of it)
      for (int b = 0; b < nb; ++b) {
        emit(3 * b + 2, XS(nq + 3 * b + 2));
        if (M.contact[b] >= 0) {
          emit(3 * b, XS(nq + 3 * b));
          emit(3 * b + 1, XS(nq + 3 * b + 1));
        } else if (j == 0) {
          D[M.sd_F + 3 * b] = TP(EL(M.n_xq + M.qrow[nq + 3 * b]));
          D[M.sd_F + 3 * b + 1] = TP(EL(M.n_xq + M.qrow[nq + 3 * b + 1]));
        }
      }
      // v' = M^-1 F
      for (int b = 0; b < nb; ++b) {
        emit(nq + 3 * b, EL(M.n_f + 3 * b) * M.minv[b]);
        emit(nq + 3 * b + 1, EL(M.n_f + 3 * b + 1) * M.minv[b]);
        emit(nq + 3 * b + 2, EL(M.n_f + 3 * b + 2) * M.iinv[b]);
      }
    }
  }
#undef XS
  double chk = 0.0;
  for (int r = 0; r < nxt; ++r) {
    const double x = M.lrow[r] >= 0 ? EL(M.n_xl + M.lrow[r]) : EL(M.n_xq + M.qrow[r]);
    const double d = x - ad.x1[r];
    defect[ad.v + r] = d;
    chk += d;
  }
  for (int ic = 0; ic < nc; ++ic) {
    const int r = M.pen0 + ic;
    const double x = M.lrow[r] >= 0 ? EL(M.n_xl + M.lrow[r]) : EL(M.n_xq + M.qrow[r]);
    penalty[ad.p + ic] = x - ad.x0[r];
  }
  if (!isfinite(chk)) atomicOr(status, ST_NONFINITE);
  // closed-form columns of A: e_p, e_v + s e_p (links without a contact), e_y
  // (not written by the adjoint's forward pass, which has no A)
  if (!A) return;
  TP* Ak = A + ad.a;
  // compact: the column's one or two entries (row r2 < c first)
  auto unit_col = [&](int c, int r2, TP v2) {
    if (cmp) {
      TP* o = Ak + M.colptr[c];
      if (r2 >= 0) *o++ = v2;
      *o = TP(1);
      return;
    }
    for (int r = 0; r < nxt; ++r) Ak[(size_t)r * nxt + c] = (r == c) ? TP(1) : (r == r2 ? v2 : TP(0));
  };
  for (int b = 0; b < nb; ++b) {
    if (M.contact[b] >= 0) continue;
    for (int c2 = 0; c2 < 2; ++c2) {
      unit_col(3 * b + c2, -1, TP(0));
      unit_col(nq + 3 * b + c2, 3 * b + c2, TP(sk));
    }
  }
  for (int r = 6 * nb; r < nxt; ++r) unit_col(r, -1, TP(0));
}

#undef LK

#define ET(o) tm[(o) * bs]

template <typename TP, int SCH>
__global__ void k_cpl_tangent(const __grid_constant__ CplTab M, long i0, long n, int nsub,
                              const double* __restrict__ s, const TP* __restrict__ sd,
                              TP* __restrict__ A, TP* __restrict__ Bm, TP* __restrict__ Bp,
                              TP* __restrict__ S, unsigned* status, int layout,
                              const int2* __restrict__ entries, const DevInst* __restrict__ inst,
                              int cmp) {
  using Sc = Scheme<SCH>;
  using K = Cst<TP>;
  constexpr int NS = Sc::S;
  extern __shared__ __align__(16) unsigned char smem2[];
  const int bs = blockDim.x;
  TP* tm = reinterpret_cast<TP*>(smem2) + threadIdx.x;
  const int C = M.cnt;
  const long g = (long)blockIdx.x * bs + threadIdx.x;
  const long t = g / C;
  if (t >= n) return;
  const int col = M.cperm[g - t * C];
  const int nb = M.nb, nj = M.nj, nc = M.nc, nxt = M.nxt, nu = M.nu, nq = 3 * nb, nk = M.nk;
  const IvAddr ad = iv_addr(i0 + t, nxt, nu, nc, layout, nullptr, nullptr, entries, inst,
                            cmp ? (long long)M.colptr[nxt] : (long long)nxt * nxt);
  const int nl = M.nlive, nqd = M.nquad;
  int qin = -1;
  bool right = false, scol = false;
  if (col >= nxt) {
    if (col < nxt + nu) qin = col - nxt;
    else if (col < nxt + 2 * nu) { qin = col - nxt - nu; right = true; }
    else scol = true;
  }
  for (int l = 0; l < nl; ++l) ET(M.t_pl + l) = TP(0);
  for (int q = 0; q < nqd; ++q) ET(M.t_pq + q) = TP(0);
  if (col < nxt) {
    if (M.lrow[col] >= 0) ET(M.t_pl + M.lrow[col]) = TP(1);
    else ET(M.t_pq + M.qrow[col]) = TP(1);
  }
  const TP sk = TP(s[ad.s]);
  const TP h = TP(1) / TP(nsub);
  const TP hsk = h * sk;
  const TP* sdk = sd + (size_t)t * nsub * NS * M.sd_size;
  // the column's input: a torque, a reaction force (inputs only without
  // elimination) or a contact input
  const int ci0 = M.ci0;
  const bool q_torque = qin >= 0 && qin < nj;
  const bool q_force = qin >= nj && qin < ci0;
  const int q_con = qin >= ci0 ? (qin - ci0) / 3 : -1;
  const int q_comp = qin >= ci0 ? (qin - ci0) % 3 : 0;
#define TXS(r) ET(M.t_xs + M.lrow[r])

  for (int i = 0; i < nsub; ++i) {
    // quadrature rows: p += h s v at the substep start
    for (int b = 0; b < nb; ++b) {
      if (M.contact[b] >= 0) continue;
      for (int c2 = 0; c2 < 2; ++c2)
        ET(M.t_pq + M.qrow[3 * b + c2]) += hsk * ET(M.t_pq + M.qrow[nq + 3 * b + c2]);
    }
    for (int j = 0; j < NS; ++j) {
      const TP* D = sdk + (size_t)(i * NS + j) * M.sd_size;
      const TP* F = D + M.sd_F;
      const TP bj = K::b(M, j), hbj = h * bj, h2b = h * h * sk * K::beta(M, j);
      // stage tangent of the live rows
      for (int l = 0; l < nl; ++l) ET(M.t_xs + l) = ET(M.t_pl + l);
      for (int m = 0; m < j; ++m) {
        const TP ah = K::a(M, j, m) * h;
        if (ah == TP(0)) continue;
        for (int l = 0; l < nl; ++l) ET(M.t_xs + l) += ah * ET(M.t_k + Sc::slot(m) * nl + l);
      }
      const TP tau = (TP(i) + K::c(M, j)) * h;
      const TP w = qin < 0 ? TP(0) : (right ? tau : TP(1) - tau);
      // generalized-force tangent e: -dtheta QW (moving application points) + direct inputs
      for (int b = 0; b < nb; ++b) {
        ET(M.t_e + 3 * b) = TP(0);
        ET(M.t_e + 3 * b + 1) = TP(0);
        ET(M.t_e + 3 * b + 2) = -TXS(3 * b + 2) * D[M.sd_qw + b];
      }
      if (q_torque) {
        ET(M.t_e + 3 * M.jchi[qin] + 2) += w;
        ET(M.t_e + 3 * M.jpar[qin] + 2) -= w;
      } else if (q_force) {
        const int jj = (qin - nj) >> 1, cp = (qin - nj) & 1;
        for (int role = 0; role < 2; ++role) {
          const int b = role ? M.jpar[jj] : M.jchi[jj];
          const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
          const TP sw = role ? -w : w;
          ET(M.t_e + 3 * b + cp) += sw;
          ET(M.t_e + 3 * b + 2) += sw * (cp ? rx : -ry);
        }
      }
      // contacts: force tangent and the auxiliary rows
      for (int ic = 0; ic < nc; ++ic) {
        const int b = M.cbody[ic];
        const TP* Dc = D + M.sd_con + M.ncf * ic;
        const TP rx = Dc[0], ry = Dc[1];
        const TP dth = TXS(3 * b + 2);
        const TP dxc = TXS(3 * b) - ry * dth;
        const TP dyc = TXS(3 * b + 1) + rx * dth;
        TP dft = TP(0), dfn = TP(0), dga = TP(0);
        if (q_con == ic) {
          if (M.aux) {
            if (q_comp == 0) dft = w; else if (q_comp == 1) dfn = w; else dga = w;
          } else {
            if (q_comp == 0) dfn = w; else if (q_comp == 1) dft = w; else dft = -w;
          }
        }
        const TP dfx = Dc[2] * dft + Dc[4] * dfn + Dc[6] * dxc;
        const TP dfy = Dc[3] * dft + Dc[5] * dfn + Dc[7] * dxc;
        ET(M.t_e + 3 * b) += dfx;
        ET(M.t_e + 3 * b + 1) += dfy;
        ET(M.t_e + 3 * b + 2) += rx * dfy - ry * dfx;
        const TP dphi = Dc[8] * dxc + Dc[9] * dyc;
        auto quad = [&](int row, TP dy) {
          TP kv = sk * dy;
          if (scol) kv += F[row];
          ET(M.t_pq + M.qrow[row]) += hbj * kv;
        };
        if (!M.aux) {
          TP dy = Dc[10] * dphi;
          if (q_con == ic) dy += Dc[11 + q_comp] * w;
          quad(6 * nb + ic, dy);
        } else {
          // lambda^c = t . v_c + gamma phi_t / sqrt(1 + phi_t^2), v_c = (v_x - omega r_y, v_y + omega r_x)
          const TP om = F[3 * b + 2];
          const TP dom = TXS(nq + 3 * b + 2);
          const TP dvcx = TXS(nq + 3 * b) - dom * ry - om * rx * dth;
          const TP dvcy = TXS(nq + 3 * b + 1) + dom * rx - om * ry * dth;
          const TP dlam = Dc[16] * dxc + Dc[2] * dvcx + Dc[3] * dvcy + Dc[17] * dft + Dc[18] * dga;
          quad(6 * nb + 4 * ic, dfn);
          quad(6 * nb + 4 * ic + 1, dlam);
          quad(6 * nb + 4 * ic + 2, dga);
          quad(6 * nb + 4 * ic + 3, Dc[19] * dft + Dc[20] * dfn);
          quad(6 * nb + 4 * nc + ic, Dc[10] * dphi + Dc[11] * dft + Dc[12] * dfn + Dc[13] * dga);
        }
      }
      // Eq. (3): K dlambda = sum over joint ends s (alpha domega + beta dtheta - e_lin / m - perp(r) e_ang / I)
      if (M.jelim && nk > 0) {
        for (int jj = 0; jj < nj; ++jj) {
          TP a0 = TP(0), a1 = TP(0);
          for (int role = 0; role < 2; ++role) {
            const int b = role ? M.jpar[jj] : M.jchi[jj];
            const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
            const TP om = F[3 * b + 2], omd = F[nq + 3 * b + 2];
            const TP dth = TXS(3 * b + 2), dom = TXS(nq + 3 * b + 2);
            const TP mi = K::minv(M, b), ii = K::iinv(M, b);
            const TP ea = ET(M.t_e + 3 * b + 2) * ii;
            // alpha = 2 omega r, beta = omega^2 perp(r) + omega' r, perp(r) = (-r_y, r_x)
            const TP c0 = TP(2) * om * rx * dom + (-om * om * ry + omd * rx) * dth -
                          ET(M.t_e + 3 * b) * mi + ry * ea;
            const TP c1 = TP(2) * om * ry * dom + (om * om * rx + omd * ry) * dth -
                          ET(M.t_e + 3 * b + 1) * mi - rx * ea;
            if (role) { a0 -= c0; a1 -= c1; } else { a0 += c0; a1 += c1; }
          }
          ET(M.t_x + 2 * M.npos[jj]) = a0;
          ET(M.t_x + 2 * M.npos[jj] + 1) = a1;
        }
        const TP* Kf = D + M.sd_K;
        for (int ii = 1; ii < nk; ++ii) {
          TP acc = ET(M.t_x + ii);
          const TP* row = Kf + M.noff[ii] - M.nf[ii];
          for (int kk = M.nf[ii]; kk < ii; ++kk) acc -= row[kk] * ET(M.t_x + kk);
          ET(M.t_x + ii) = acc;
        }
        for (int ii = nk - 1; ii >= 0; --ii) {
          TP acc = ET(M.t_x + ii) * Kf[M.noff[ii] + ii - M.nf[ii]];
          for (int kk = ii + 1; kk < nk; ++kk)
            if (M.nf[kk] <= ii) acc -= Kf[M.noff[kk] + ii - M.nf[kk]] * ET(M.t_x + kk);
          ET(M.t_x + ii) = acc;
        }
        for (int jj = 0; jj < nj; ++jj) {
          const TP lx = ET(M.t_x + 2 * M.npos[jj]), ly = ET(M.t_x + 2 * M.npos[jj] + 1);
          for (int role = 0; role < 2; ++role) {
            const int b = role ? M.jpar[jj] : M.jchi[jj];
            const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
            const TP sx = role ? -lx : lx, sy = role ? -ly : ly;
            ET(M.t_e + 3 * b) += sx;
            ET(M.t_e + 3 * b + 1) += sy;
            ET(M.t_e + 3 * b + 2) += rx * sy - ry * sx;
          }
        }
      }
      // slopes: live rows (RK stages) and quadrature rows
      auto live = [&](int row, TP dy) {
        TP kv = sk * dy;
        if (scol) kv += F[row];
        const int l = M.lrow[row];
        if (Sc::NKS == 1) {
          if (j < NS - 1) ET(M.t_k + l) = kv;
          ET(M.t_acc + l) = (j == 0) ? bj * kv : ET(M.t_acc + l) + bj * kv;
          if (j == NS - 1) ET(M.t_pl + l) += h * ET(M.t_acc + l);
        } else if (j < NS - 1) {
          ET(M.t_k + Sc::slot(j) * nl + l) = kv;
        } else {  // last stage: x += h sum_m b_m k_m from the stored slopes
          TP acc = bj * kv;
          for (int m = NS - 2; m >= 0; --m)
            if (Sc::bnz(m)) acc += K::b(M, m) * ET(M.t_k + Sc::slot(m) * nl + l);
          ET(M.t_pl + l) += h * acc;
        }
      };
      for (int b = 0; b < nb; ++b) {
        const TP mi = K::minv(M, b);
        const TP dv0 = ET(M.t_e + 3 * b) * mi, dv1 = ET(M.t_e + 3 * b + 1) * mi;
        const TP dw = ET(M.t_e + 3 * b + 2) * K::iinv(M, b);
        live(3 * b + 2, TXS(nq + 3 * b + 2));
        live(nq + 3 * b + 2, dw);
        if (M.contact[b] >= 0) {
          live(3 * b, TXS(nq + 3 * b));
          live(3 * b + 1, TXS(nq + 3 * b + 1));
          live(nq + 3 * b, dv0);
          live(nq + 3 * b + 1, dv1);
        } else {
          // p' = s v with v a quadrature row: p gains h^2 s beta_j k_v here
          // (h s v at the substep start); for the s column also the nominal
          // velocity's own contribution h sum_j b_j v_j = h (v_0 + h s sum_j beta_j F_v,j)
          const TP dv[2] = {dv0, dv1};
          for (int c2 = 0; c2 < 2; ++c2) {
            TP kv = sk * dv[c2];
            TP pinc = TP(0);
            if (scol) {
              kv += F[nq + 3 * b + c2];
              pinc = h2b * F[nq + 3 * b + c2];
              if (j == 0) pinc += h * F[3 * b + c2];
            }
            ET(M.t_pq + M.qrow[3 * b + c2]) += h2b * kv + pinc;
            ET(M.t_pq + M.qrow[nq + 3 * b + c2]) += hbj * kv;
          }
        }
      }
    }
  }
#undef TXS
  // column `col` of [A | B- | B+ | S]
  TP* out;
  size_t stride;
  if (cmp) {  // compact: column-major, the column's rows contiguous
    if (col < nxt) out = A + ad.a + M.colptr[col];
    else if (!scol) out = (right ? Bp : Bm) + ad.b + (size_t)qin * nxt;
    else out = S + ad.v;
    stride = 1;
  } else if (col < nxt) { out = A + ad.a + col; stride = nxt; }
  else if (!scol) { out = (right ? Bp : Bm) + ad.b + qin; stride = nu; }
  else { out = S + ad.v; stride = 1; }
  float chk = 0.0f;
  for (int r = 0; r < nxt; ++r) {
    const TP v = M.lrow[r] >= 0 ? ET(M.t_pl + M.lrow[r]) : ET(M.t_pq + M.qrow[r]);
    out[(size_t)r * stride] = v;
    chk += float(v);
  }
  if (!isfinite(chk)) atomicOr(status, ST_NONFINITE);
}

#undef ET
#undef EL

// Tangent-kernel block size: the largest of 128 / 64 / 32 threads whose
// scratch fits in 76 KB (two or more blocks per SM).
template <typename TP>
int tangent_block(const CplTab& T) {
  for (int bs = 128; bs > 32; bs /= 2)
    if ((size_t)bs * T.t_size * sizeof(TP) <= 76u * 1024u) return bs;
  return 32;
}

template <typename TP, int SCH>
cudaError_t prepare(const CplTab& T) {
  static bool done = false;  // generic kernels' shared-memory limit (raised once, before any capture)
  if (done) return cudaSuccess;
  const int bs = tangent_block<TP>(T);
  cudaError_t e = cudaFuncSetAttribute(k_cpl_nominal<TP, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cpl_tangent<TP, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  (void)bs;
  done = e == cudaSuccess;
  return e;
}

// The chunk rounded down to whole waves of the nominal kernel (SMs x its
// resident one-warp blocks x 32 intervals) when it holds more than one: that
// kernel is latency-bound at a few warps per SM, so a chunk of 1.1 waves takes
// as long as two.  Chunks stay multiples of 32 intervals past the first wave.
template <typename TP, int SCH>
long wave_chunk(const CplJit* jnom, size_t sm1, long chunk) {
  int bps = jnom ? jnom->blocks_per_sm : 0;
  if (!jnom && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cpl_nominal<TP, SCH>, 32, sm1) != cudaSuccess) {
    (void)cudaGetLastError();
    bps = 0;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return chunk;
  }
  const long wave = (long)bps * sms * 32;
  return (wave > 0 && chunk > wave) ? chunk / wave * wave : chunk;
}

template <typename TP, int SCH>
cudaError_t run(const CplTab& T, long N, int nsub, int layout, const double* X, const double* U,
                const double* s, void* A, void* Bm, void* Bp, void* S, double* defect,
                double* penalty, void* ws, long chunk, unsigned* status, cudaStream_t st,
                const int2* entries, const DevInst* inst, int cmp) {
  const size_t sm1 = (size_t)T.n_size * sizeof(double) * 32;
  const int prec = std::is_same<TP, double>::value ? CISCVX_FP64 : CISCVX_FP32_PHI;
  const CplJit* jit = cpl_jit_tangent(T, prec);
  const CplJit* jnom = cpl_jit_nominal(T, prec);
  const int bs = tangent_block<TP>(T);
  const size_t sm2 = (size_t)bs * T.t_size * sizeof(TP);
  cudaError_t e = prepare<TP, SCH>(T);
  if (e != cudaSuccess) return e;
  chunk = wave_chunk<TP, SCH>(jnom, sm1, chunk);
  for (long i0 = 0; i0 < N; i0 += chunk) {
    const long n = std::min<long>(chunk, N - i0);
    if (jnom)
      e = cpl_jit_launch_nominal(*jnom, T, i0, n, nsub, layout, X, U, s, ws, A, defect, penalty, status, st,
                                 entries, inst, cmp);
    else
      k_cpl_nominal<TP, SCH><<<(unsigned)((n + 31) / 32), 32, sm1, st>>>(
          T, i0, n, nsub, layout, X, U, s, (TP*)ws, (TP*)A, defect, penalty, status, entries, inst, cmp);
    if (e != cudaSuccess) return e;
    const long threads = n * T.cnt;
    if (jit) {
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cpl_jit_launch(*jit, T, prec, i0, n, nsub, s, ws, A, Bm, Bp, S, status, st, layout, entries,
                           inst, cmp);
    } else {
      k_cpl_tangent<TP, SCH><<<(unsigned)((threads + bs - 1) / bs), bs, sm2, st>>>(
          T, i0, n, nsub, s, (const TP*)ws, (TP*)A, (TP*)Bm, (TP*)Bp, (TP*)S, status, layout, entries,
          inst, cmp);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Reverse-mode adjoint (VJP) of the coupled path: thread = interval.  The
// forward pass is k_cpl_nominal (stage data, defects, penalty increments; no
// A).  This kernel runs the transpose of k_cpl_tangent's stage map backward
// over the substeps and stages, from the cotangent of x~(1),
//   lambda = w_k + rho_k on the path-penalty rows,
// to lambda^T [A | B- | B+ | S] = (dL/dx~_k, dL/du_L, dL/du_R, dL/ds_k) of the
// interval — the gradient of L = sum_k w_k . defect_k + rho_k . penalty_k
// without forming a single block.  Per stage, in reverse:
//  * slopes: k_bar of each live row (h b_j of the substep-end cotangent plus
//    h a_mj of every later stage's stage-tangent cotangent) and of the
//    quadrature rows (h b_j, and h^2 s beta_j for the positions of links
//    without a contact) give the generalized-force cotangent e_bar = M^-1 s
//    k_bar and the velocity rows' stage cotangents;
//  * Eq. (3): x_bar = grad C e_bar, a_bar = K^-1 x_bar (K symmetric: the same
//    recorded factor as the forward solve), then the transposed right-hand
//    side a(theta, omega, e) adds to the angle / rate cotangents and e_bar;
//  * contacts: the force, its direction and the signed distance (the
//    sinusoid's frame derivatives recorded by the nominal kernel), the
//    penalty and Eq. (12) rows; inputs collect (1 - tau) / tau of their stage
//    cotangent into dL/du_L / dL/du_R; s collects k_bar . F.
// Cotangent arrays live in shared memory, element major (per thread).

#define AT(o) am[(o) * bs]

template <typename TP, int SCH>
__global__ void k_cpl_adjoint(const __grid_constant__ CplTab M, long i0, long n, long N, int nsub,
                              const double* __restrict__ s, const TP* __restrict__ sd,
                              const double* __restrict__ w, const double* __restrict__ rho,
                              double* __restrict__ gX, double* __restrict__ gs,
                              double* __restrict__ ubar, unsigned* status) {
  using Sc = Scheme<SCH>;
  using K = Cst<TP>;
  constexpr int NS = Sc::S;
  extern __shared__ __align__(16) unsigned char smem3[];
  const int bs = blockDim.x;
  TP* am = reinterpret_cast<TP*>(smem3) + threadIdx.x;
  const long t = (long)blockIdx.x * bs + threadIdx.x;
  if (t >= n) return;
  const long k = i0 + t;
  const int nb = M.nb, nj = M.nj, nc = M.nc, nxt = M.nxt, nu = M.nu, nq = 3 * nb, nk = M.nk;
  const int nl = M.nlive, nqd = M.nquad;
  const int o_pl = 0, o_pq = nl, o_kb = o_pq + nqd, o_xs = o_kb + NS * nl, o_e = o_xs + nl;
  const int o_x = o_e + 3 * nb, o_ub = o_x + nk;
  const double* wk = w + k * nxt;
  const int pen0 = M.pen0;
  auto lam = [&](int r) {
    double v = wk[r];
    if (r >= pen0 && r < pen0 + nc) v += rho[k * nc + (r - pen0)];
    return v;
  };
  for (int r = 0; r < nxt; ++r) {
    if (M.lrow[r] >= 0) AT(o_pl + M.lrow[r]) = TP(lam(r));
    else AT(o_pq + M.qrow[r]) = TP(lam(r));
  }
  for (int q = 0; q < 2 * nu; ++q) AT(o_ub + q) = TP(0);
  const TP sk = TP(s[k]);
  const TP h = TP(1) / TP(nsub);
  const TP hsk = h * sk;
  TP sbar = TP(0);
  const TP* sdk = sd + (size_t)t * nsub * NS * M.sd_size;
  const int ci0 = M.ci0;
#define XB(r) AT(o_xs + M.lrow[r])
#define EB(c) AT(o_e + (c))
#define KB(r) AT(o_kb + j * nl + M.lrow[r])
#define PQ(r) AT(o_pq + M.qrow[r])

  for (int i = nsub - 1; i >= 0; --i) {
    // slope cotangents of every stage start at h b_j (cotangent at the substep end)
    for (int j = 0; j < NS; ++j) {
      const TP hb = h * K::b(M, j);
      for (int l = 0; l < nl; ++l) AT(o_kb + j * nl + l) = hb * AT(o_pl + l);
    }
    for (int j = NS - 1; j >= 0; --j) {
      const TP* D = sdk + (size_t)(i * NS + j) * M.sd_size;
      const TP* F = D + M.sd_F;
      const TP bj = K::b(M, j), hbj = h * bj, h2b = h * h * sk * K::beta(M, j);
      const TP tau = (TP(i) + K::c(M, j)) * h;
      const TP wl = TP(1) - tau, wr = tau;
      for (int l = 0; l < nl; ++l) AT(o_xs + l) = TP(0);
      for (int c = 0; c < 3 * nb; ++c) EB(c) = TP(0);
      // input cotangent of this stage -> dL/du_L, dL/du_R
      auto uput = [&](int q, TP v) {
        AT(o_ub + q) += wl * v;
        AT(o_ub + nu + q) += wr * v;
      };
      // ---- slopes (transposed) ----
      for (int b = 0; b < nb; ++b) {
        const TP mi = K::minv(M, b), ii = K::iinv(M, b);
        {
          const TP kb = KB(3 * b + 2);  // theta' = s omega
          XB(nq + 3 * b + 2) += sk * kb;
          sbar += kb * F[3 * b + 2];
        }
        {
          const TP kb = KB(nq + 3 * b + 2);  // omega' = s e_ang / I
          EB(3 * b + 2) += sk * kb * ii;
          sbar += kb * F[nq + 3 * b + 2];
        }
        if (M.contact[b] >= 0) {
          for (int c2 = 0; c2 < 2; ++c2) {
            const TP kp = KB(3 * b + c2);  // p' = s v
            XB(nq + 3 * b + c2) += sk * kp;
            sbar += kp * F[3 * b + c2];
            const TP kv = KB(nq + 3 * b + c2);  // v' = s e_lin / m
            EB(3 * b + c2) += sk * kv * mi;
            sbar += kv * F[nq + 3 * b + c2];
          }
        } else {
          // quadrature rows: v += h b_j k_v, p += h^2 s beta_j k_v
          for (int c2 = 0; c2 < 2; ++c2) {
            const TP Pp = PQ(3 * b + c2), Pv = PQ(nq + 3 * b + c2);
            const TP kvb = h2b * Pp + hbj * Pv;
            EB(3 * b + c2) += sk * kvb * mi;
            sbar += kvb * F[nq + 3 * b + c2] + Pp * h2b * F[nq + 3 * b + c2];
            if (j == 0) sbar += Pp * h * F[3 * b + c2];  // d(h s v_start)/ds
          }
        }
      }
      // ---- Eq. (3) (transposed): e += grad C^T x, x = K^-1 a(theta, omega, e) ----
      if (M.jelim && nk > 0) {
        for (int jj = 0; jj < nj; ++jj) {
          TP lx = TP(0), ly = TP(0);
          for (int role = 0; role < 2; ++role) {
            const int b = role ? M.jpar[jj] : M.jchi[jj];
            const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
            const TP vx = EB(3 * b) - ry * EB(3 * b + 2), vy = EB(3 * b + 1) + rx * EB(3 * b + 2);
            if (role) { lx -= vx; ly -= vy; } else { lx += vx; ly += vy; }
          }
          AT(o_x + 2 * M.npos[jj]) = lx;
          AT(o_x + 2 * M.npos[jj] + 1) = ly;
        }
        const TP* Kf = D + M.sd_K;
        for (int ii = 1; ii < nk; ++ii) {
          TP acc = AT(o_x + ii);
          const TP* row = Kf + M.noff[ii] - M.nf[ii];
          for (int kk = M.nf[ii]; kk < ii; ++kk) acc -= row[kk] * AT(o_x + kk);
          AT(o_x + ii) = acc;
        }
        for (int ii = nk - 1; ii >= 0; --ii) {
          TP acc = AT(o_x + ii) * Kf[M.noff[ii] + ii - M.nf[ii]];
          for (int kk = ii + 1; kk < nk; ++kk)
            if (M.nf[kk] <= ii) acc -= Kf[M.noff[kk] + ii - M.nf[kk]] * AT(o_x + kk);
          AT(o_x + ii) = acc;
        }
        for (int jj = 0; jj < nj; ++jj) {
          const TP a0b = AT(o_x + 2 * M.npos[jj]), a1b = AT(o_x + 2 * M.npos[jj] + 1);
          for (int role = 0; role < 2; ++role) {
            const int b = role ? M.jpar[jj] : M.jchi[jj];
            const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
            const TP om = F[3 * b + 2], omd = F[nq + 3 * b + 2];
            const TP c0 = role ? -a0b : a0b, c1 = role ? -a1b : a1b;
            XB(nq + 3 * b + 2) += TP(2) * om * (rx * c0 + ry * c1);
            XB(3 * b + 2) += (-om * om * ry + omd * rx) * c0 + (om * om * rx + omd * ry) * c1;
            EB(3 * b) -= K::minv(M, b) * c0;
            EB(3 * b + 1) -= K::minv(M, b) * c1;
            EB(3 * b + 2) += K::iinv(M, b) * (ry * c0 - rx * c1);
          }
        }
      }
      // ---- contacts (transposed): force, frame, signed distance, auxiliary rows ----
      for (int ic = 0; ic < nc; ++ic) {
        const int b = M.cbody[ic];
        const TP* Dc = D + M.sd_con + M.ncf * ic;
        const TP rx = Dc[0], ry = Dc[1];
        const TP fxb = EB(3 * b) - ry * EB(3 * b + 2), fyb = EB(3 * b + 1) + rx * EB(3 * b + 2);
        TP ftb = Dc[2] * fxb + Dc[3] * fyb, fnb = Dc[4] * fxb + Dc[5] * fyb, gab = TP(0);
        TP xcb = Dc[6] * fxb + Dc[7] * fyb, phib = TP(0);
        // cotangent of a quadrature row's slope argument dy (kv = s dy + F)
        auto qrow_bar = [&](int row) {
          const TP kvb = hbj * PQ(row);
          sbar += kvb * F[row];
          return sk * kvb;
        };
        const int u0 = ci0 + 3 * ic;
        if (!M.aux) {
          const TP yb = qrow_bar(6 * nb + ic);
          phib = Dc[10] * yb;
          // inputs (lambda_n, lambda_t+, lambda_t-): force components and penalty slopes
          uput(u0, fnb + Dc[11] * yb);
          uput(u0 + 1, ftb + Dc[12] * yb);
          uput(u0 + 2, -ftb + Dc[13] * yb);
        } else {
          const TP y0 = qrow_bar(6 * nb + 4 * ic), y1 = qrow_bar(6 * nb + 4 * ic + 1);
          const TP y2 = qrow_bar(6 * nb + 4 * ic + 2), y3 = qrow_bar(6 * nb + 4 * ic + 3);
          const TP y4 = qrow_bar(6 * nb + 4 * nc + ic);
          fnb += y0 + Dc[20] * y3 + Dc[12] * y4;
          gab += y2 + Dc[18] * y1 + Dc[13] * y4;
          ftb += Dc[17] * y1 + Dc[19] * y3 + Dc[11] * y4;
          xcb += Dc[16] * y1;
          phib = Dc[10] * y4;
          // lambda^c's contact-point velocity (v_x - omega r_y, v_y + omega r_x)
          const TP om = F[3 * b + 2];
          const TP vxb = Dc[2] * y1, vyb = Dc[3] * y1;
          XB(nq + 3 * b) += vxb;
          XB(nq + 3 * b + 1) += vyb;
          XB(nq + 3 * b + 2) += -ry * vxb + rx * vyb;
          XB(3 * b + 2) += -om * (rx * vxb + ry * vyb);
          // inputs (phi_t, phi_n, gamma)
          uput(u0, ftb);
          uput(u0 + 1, fnb);
          uput(u0 + 2, gab);
        }
        xcb += Dc[8] * phib;
        const TP ycb = Dc[9] * phib;
        XB(3 * b) += xcb;
        XB(3 * b + 1) += ycb;
        XB(3 * b + 2) += -ry * xcb + rx * ycb;
      }
      // ---- direct inputs: torques, and reaction forces when they are inputs ----
      for (int jj = 0; jj < nj; ++jj) {
        uput(jj, EB(3 * M.jchi[jj] + 2) - EB(3 * M.jpar[jj] + 2));
        if (!M.jelim) {
          for (int cp = 0; cp < 2; ++cp) {
            TP v = TP(0);
            for (int role = 0; role < 2; ++role) {
              const int b = role ? M.jpar[jj] : M.jchi[jj];
              const TP rx = D[M.sd_arm + 4 * jj + 2 * role], ry = D[M.sd_arm + 4 * jj + 2 * role + 1];
              const TP c = EB(3 * b + cp) + (cp ? rx : -ry) * EB(3 * b + 2);
              v = role ? v - c : v + c;
            }
            uput(nj + 2 * jj + cp, v);
          }
        }
      }
      // ---- moving application points: e_ang = -dtheta QW ----
      for (int b = 0; b < nb; ++b) XB(3 * b + 2) -= D[M.sd_qw + b] * EB(3 * b + 2);
      // stage-tangent cotangent -> the substep start and the earlier stages' slopes
      for (int l = 0; l < nl; ++l) {
        const TP xb = AT(o_xs + l);
        AT(o_pl + l) += xb;
        for (int m = 0; m < j; ++m) {
          const TP ah = K::a(M, j, m) * h;
          if (ah != TP(0)) AT(o_kb + m * nl + l) += ah * xb;
        }
      }
    }
    // p += h s v at the substep start (links without a contact)
    for (int b = 0; b < nb; ++b) {
      if (M.contact[b] >= 0) continue;
      for (int c2 = 0; c2 < 2; ++c2) PQ(nq + 3 * b + c2) += hsk * PQ(3 * b + c2);
    }
  }
#undef XB
#undef EB
#undef KB
#undef PQ
  // dL/dx~_k = A^T lambda - rho (own penalty rows) - w_{k-1}
  double chk = 0.0;
  for (int r = 0; r < nxt; ++r) {
    double v = widen(M.lrow[r] >= 0 ? AT(o_pl + M.lrow[r]) : AT(o_pq + M.qrow[r]));
    if (r >= pen0 && r < pen0 + nc) v -= rho[k * nc + (r - pen0)];
    if (k >= 1) v -= w[(k - 1) * nxt + r];
    gX[k * nxt + r] = v;
    if (k == N - 1) gX[N * nxt + r] = -wk[r];
    chk += v;
  }
  gs[k] = widen(sbar);
  double* ub = ubar + (size_t)t * 2 * nu;
  for (int q = 0; q < 2 * nu; ++q) ub[q] = widen(AT(o_ub + q));
  if (!isfinite(chk + widen(sbar))) atomicOr(status, ST_NONFINITE);
}

#undef AT

// dL/du from the per-interval input cotangents of a chunk [i0, i0 + n):
// interval layout gU[k] = (u_L bar, u_R bar); node layout gU[k] = u_L bar(k) +
// u_R bar(k - 1), the term of the chunk's previous interval carried through
// gU itself across chunk boundaries (chunks run in stream order).
__global__ void k_cpl_adjoint_u(int nu, long i0, long n, int layout, const double* __restrict__ ubar,
                                double* __restrict__ gU) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long t = g / nu;
  if (t >= n) return;
  const int q = (int)(g - t * nu);
  const long k = i0 + t;
  const double* ub = ubar + (size_t)t * 2 * nu;
  if (layout == CISCVX_FOH_INTERVAL) {
    gU[(2 * k) * nu + q] = ub[q];
    gU[(2 * k + 1) * nu + q] = ub[nu + q];
  } else {
    double prev = 0.0;
    if (t > 0) prev = ubar[(size_t)(t - 1) * 2 * nu + nu + q];
    else if (k > 0) prev = gU[k * nu + q];
    gU[k * nu + q] = ub[q] + prev;
    if (t == n - 1) gU[(k + 1) * nu + q] = ub[nu + q];
  }
}

// L over a chunk in two fixed-order passes (deterministic): block b sums a
// contiguous range of w . defect + rho . penalty into part[b], then one block
// adds the partial sums in order to *L.
constexpr int ADJ_LRED_BLOCKS = 512;

__global__ void k_cpl_adjoint_L(int nxt, int nc, long i0, long n, const double* __restrict__ defect,
                                const double* __restrict__ penalty, const double* __restrict__ w,
                                const double* __restrict__ rho, double* __restrict__ part) {
  __shared__ double red[256];
  const long tot = n * (nxt + nc);
  const long per = (tot + gridDim.x - 1) / gridDim.x;
  const long lo = (long)blockIdx.x * per, hi = lo + per < tot ? lo + per : tot;
  double acc = 0.0;
  for (long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    if (e < n * nxt) acc = fma(w[i0 * nxt + e], defect[e], acc);
    else {
      const long f = e - n * nxt;
      acc = fma(rho[i0 * nc + f], penalty[f], acc);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_cpl_adjoint_L_sum(const double* __restrict__ part, int nblk, double* L) {
  if (threadIdx.x != 0) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[b];
  *L += acc;
}

// Adjoint block size: the largest of 128 / 64 / 32 threads whose cotangent
// scratch fits in 96 KB.
template <typename TP>
int adjoint_block(const CplTab& T) {
  const size_t per = (size_t)(2 * T.nlive + T.nquad + T.stages * T.nlive + 3 * T.nb + T.nk + 2 * T.nu) *
                     sizeof(TP);
  for (int bs = 128; bs > 32; bs /= 2)
    if (bs * per <= 96u * 1024u) return bs;
  return 32;
}

template <typename TP, int SCH>
cudaError_t run_vjp(const CplTab& T, long N, int nsub, int layout, const double* X, const double* U,
                    const double* s, const double* w, const double* rho, double* gX, double* gU,
                    double* gs, double* L, void* ws, size_t ws_bytes, unsigned* status, cudaStream_t st) {
  const int prec = std::is_same<TP, double>::value ? CISCVX_FP64 : CISCVX_FP32_PHI;
  const CplJit* jnom = cpl_jit_nominal(T, prec);
  const CplJit* jadj = cpl_jit_adjoint(T, prec);
  cudaError_t e = prepare<TP, SCH>(T);
  if (e != cudaSuccess) return e;
  static bool adj_ready = false;  // raise the adjoint's shared-memory limit once
  if (!adj_ready) {
    e = cudaFuncSetAttribute(k_cpl_adjoint<TP, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    adj_ready = true;
  }
  const size_t sm1 = (size_t)T.n_size * sizeof(double) * 32;
  const int bs = adjoint_block<TP>(T);
  const size_t sm3 = (size_t)bs * (2 * T.nlive + T.nquad + T.stages * T.nlive + 3 * T.nb + T.nk + 2 * T.nu) *
                     sizeof(TP);
  long lo = 1, hi = N;  // largest chunk whose workspace fits (the caller checked that min(N, 32) does)
  while (lo < hi) {
    const long mid = (lo + hi + 1) / 2;
    if (cpl_adjoint_bytes(T, mid, nsub, prec) <= ws_bytes) lo = mid; else hi = mid - 1;
  }
  const long chunk = wave_chunk<TP, SCH>(jnom, sm1, lo);
  const CplAdjLayout Ly = cpl_adjoint_layout(T, chunk, nsub, prec);
  char* base = (char*)ws;
  TP* sd = (TP*)(base + Ly.stage);
  double* defect = (double*)(base + Ly.defect);
  double* penalty = (double*)(base + Ly.penalty);
  double* ubar = (double*)(base + Ly.ubar);
  if (L) e = cudaMemsetAsync(L, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int nxt = T.nxt, nu = T.nu;
  for (long i0 = 0; i0 < N; i0 += chunk) {
    const long n = std::min<long>(chunk, N - i0);
    const double* Xc = X + i0 * nxt;
    const double* Uc = U ? (layout == CISCVX_FOH_NODE ? U + i0 * nu : U + 2 * i0 * nu) : nullptr;
    if (jnom)
      e = cpl_jit_launch_nominal(*jnom, T, 0, n, nsub, layout, Xc, Uc, s + i0, sd, nullptr, defect, penalty,
                                 status, st, nullptr, nullptr, 0);
    else
      k_cpl_nominal<TP, SCH><<<(unsigned)((n + 31) / 32), 32, sm1, st>>>(
          T, 0, n, nsub, layout, Xc, Uc, s + i0, sd, (TP*)nullptr, defect, penalty, status, nullptr, nullptr,
          0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (jadj) {
      e = cpl_jit_launch_adjoint(*jadj, T, prec, i0, n, N, nsub, s, sd, w, rho, gX, gs, ubar, status, st);
      if (e != cudaSuccess) return e;
    } else {
      k_cpl_adjoint<TP, SCH><<<(unsigned)((n + bs - 1) / bs), bs, sm3, st>>>(T, i0, n, N, nsub, s, sd, w, rho,
                                                                           gX, gs, ubar, status);
    }
    if (nu > 0)
      k_cpl_adjoint_u<<<(unsigned)((n * nu + 127) / 128), 128, 0, st>>>(nu, i0, n, layout, ubar, gU);
    if (L) {
      const long tot = n * (nxt + T.nc);
      const int nblk = (int)std::min<long>(ADJ_LRED_BLOCKS, (tot + 2047) / 2048);
      double* part = (double*)(base + Ly.lpart);
      k_cpl_adjoint_L<<<nblk, 256, 0, st>>>(nxt, T.nc, i0, n, defect, penalty, w, rho, part);
      k_cpl_adjoint_L_sum<<<1, 32, 0, st>>>(part, nblk, L);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The linearization and the reverse-mode VJP of intervals [0, N) of one
// instance from one nominal pass per chunk: the nominal kernel writes the
// stage data (and the defects, penalty increments and closed-form columns of
// A into the outputs), then the tangent kernel forms the integrated columns
// and the adjoint kernel the gradient from the same stage data.  Workspace as
// for the VJP (cpl_adjoint_bytes of a chunk; its defect / penalty regions are
// unused).  Outputs equal those of the two calls.
template <typename TP, int SCH>
cudaError_t run_both(const CplTab& T, long N, int nsub, int layout, const double* X, const double* U,
                     const double* s, void* A, void* Bm, void* Bp, void* S, double* defect, double* penalty,
                     const double* w, const double* rho, double* gX, double* gU, double* gs, double* L, void* ws,
                     size_t ws_bytes, unsigned* status, cudaStream_t st, int cmp) {
  const int prec = std::is_same<TP, double>::value ? CISCVX_FP64 : CISCVX_FP32_PHI;
  const CplJit* jnom = cpl_jit_nominal(T, prec);
  const CplJit* jtan = cpl_jit_tangent(T, prec);
  const CplJit* jadj = cpl_jit_adjoint(T, prec);
  cudaError_t e = prepare<TP, SCH>(T);
  if (e != cudaSuccess) return e;
  static bool adj_ready = false;
  if (!adj_ready) {
    e = cudaFuncSetAttribute(k_cpl_adjoint<TP, SCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    adj_ready = true;
  }
  const size_t sm1 = (size_t)T.n_size * sizeof(double) * 32;
  const int tbs = tangent_block<TP>(T);
  const size_t sm2 = (size_t)tbs * T.t_size * sizeof(TP);
  const int bs = adjoint_block<TP>(T);
  const size_t sm3 = (size_t)bs * (2 * T.nlive + T.nquad + T.stages * T.nlive + 3 * T.nb + T.nk + 2 * T.nu) *
                     sizeof(TP);
  long lo = 1, hi = N;
  while (lo < hi) {
    const long mid = (lo + hi + 1) / 2;
    if (cpl_adjoint_bytes(T, mid, nsub, prec) <= ws_bytes) lo = mid; else hi = mid - 1;
  }
  const long chunk = wave_chunk<TP, SCH>(jnom, sm1, lo);
  const CplAdjLayout Ly = cpl_adjoint_layout(T, chunk, nsub, prec);
  char* base = (char*)ws;
  TP* sd = (TP*)(base + Ly.stage);
  double* ubar = (double*)(base + Ly.ubar);
  if (L) e = cudaMemsetAsync(L, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int nxt = T.nxt, nu = T.nu, nc = T.nc;
  for (long i0 = 0; i0 < N; i0 += chunk) {
    const long n = std::min<long>(chunk, N - i0);
    if (jnom)
      e = cpl_jit_launch_nominal(*jnom, T, i0, n, nsub, layout, X, U, s, sd, A, defect, penalty, status, st,
                                 nullptr, nullptr, cmp);
    else
      k_cpl_nominal<TP, SCH><<<(unsigned)((n + 31) / 32), 32, sm1, st>>>(
          T, i0, n, nsub, layout, X, U, s, sd, (TP*)A, defect, penalty, status, nullptr, nullptr, cmp);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long threads = n * T.cnt;
    if (jtan)
      e = cpl_jit_launch(*jtan, T, prec, i0, n, nsub, s, sd, A, Bm, Bp, S, status, st, layout, nullptr, nullptr,
                         cmp);
    else
      k_cpl_tangent<TP, SCH><<<(unsigned)((threads + tbs - 1) / tbs), tbs, sm2, st>>>(
          T, i0, n, nsub, s, (const TP*)sd, (TP*)A, (TP*)Bm, (TP*)Bp, (TP*)S, status, layout, nullptr, nullptr,
          cmp);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (jadj)
      e = cpl_jit_launch_adjoint(*jadj, T, prec, i0, n, N, nsub, s, sd, w, rho, gX, gs, ubar, status, st);
    else
      k_cpl_adjoint<TP, SCH><<<(unsigned)((n + bs - 1) / bs), bs, sm3, st>>>(T, i0, n, N, nsub, s, sd, w, rho,
                                                                           gX, gs, ubar, status);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nu > 0)
      k_cpl_adjoint_u<<<(unsigned)((n * nu + 127) / 128), 128, 0, st>>>(nu, i0, n, layout, ubar, gU);
    if (L) {
      const long tot = n * (nxt + nc);
      const int nblk = (int)std::min<long>(ADJ_LRED_BLOCKS, (tot + 2047) / 2048);
      double* part = (double*)(base + Ly.lpart);
      k_cpl_adjoint_L<<<nblk, 256, 0, st>>>(nxt, nc, i0, n, defect + i0 * nxt,
                                            nc > 0 ? penalty + i0 * nc : nullptr, w, rho, part);
      k_cpl_adjoint_L_sum<<<1, 32, 0, st>>>(part, nblk, L);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Butcher tableaux: classical RK4 and Fehlberg's 4(5) pair advanced with its
// fifth-order weights (the published coefficients).
void set_tableau(int scheme, CplTab& T) {
  std::memset(T.c, 0, sizeof T.c);
  std::memset(T.a, 0, sizeof T.a);
  std::memset(T.b, 0, sizeof T.b);
  if (scheme == 0) {
    T.stages = 4;
    T.nks = 1;
    const double c[4] = {0.0, 0.5, 0.5, 1.0}, b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int i = 0; i < 4; ++i) { T.c[i] = c[i]; T.b[i] = b[i]; }
    T.a[1][0] = 0.5; T.a[2][1] = 0.5; T.a[3][2] = 1.0;
  } else {
    T.stages = 6;
    T.nks = 5;
    const double c[6] = {0.0, 0.25, 0.375, 12.0 / 13.0, 1.0, 0.5};
    const double b[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
    for (int i = 0; i < 6; ++i) { T.c[i] = c[i]; T.b[i] = b[i]; }
    T.a[1][0] = 0.25;
    T.a[2][0] = 3.0 / 32.0; T.a[2][1] = 9.0 / 32.0;
    T.a[3][0] = 1932.0 / 2197.0; T.a[3][1] = -7200.0 / 2197.0; T.a[3][2] = 7296.0 / 2197.0;
    T.a[4][0] = 439.0 / 216.0; T.a[4][1] = -8.0; T.a[4][2] = 3680.0 / 513.0; T.a[4][3] = -845.0 / 4104.0;
    T.a[5][0] = -8.0 / 27.0; T.a[5][1] = 2.0; T.a[5][2] = -3544.0 / 2565.0; T.a[5][3] = 1859.0 / 4104.0;
    T.a[5][4] = -11.0 / 40.0;
  }
  for (int l = 0; l < CPL_MAXSTAGE; ++l) {
    double bl = 0.0;
    for (int j = 0; j < CPL_MAXSTAGE; ++j) bl += T.b[j] * T.a[j][l];
    T.beta[l] = bl;
  }
}

}  // namespace

const char* cpl_build(const DevModel& M, CplTab& T) {
  std::memset(&T, 0, sizeof T);
  const int nb = M.nb, nj = M.nj, nc = M.nc;
  T.nb = nb; T.nj = nj; T.nc = nc; T.nxt = M.nxt; T.nu = M.nu; T.ny = M.ny;
  T.aux = M.aux; T.jelim = M.jelim; T.scheme = M.scheme;
  T.C = M.nxt + 2 * M.nu + 1;
  T.ci0 = (M.jelim ? 1 : 3) * nj;
  T.pen0 = 6 * nb + (M.aux ? 4 * nc : 0);
  T.g = M.g; T.ta = M.ta; T.tk = M.tk;
  if (M.jelim && nj > 0) {
    if (!M.tree) return "eliminated joint forces need every link to be the child of at most one joint";
    if (nj > CPL_MAXJ) return "eliminated joint forces support at most 12 joints";
    for (int b = 0; b < nb; ++b)
      if (M.nadj[b] > NODE_MAXADJ) return "eliminated joint forces support at most 8 joints on one link";
    T.nk = 2 * nj;
    T.nsky = M.noff[2 * nj];
    for (int j = 0; j < nj; ++j) { T.npos[j] = M.npos[j]; T.nord[j] = M.nord[j]; }
    for (int i = 0; i < 2 * nj; ++i) T.nf[i] = M.nf[i];
    for (int i = 0; i <= 2 * nj; ++i) T.noff[i] = M.noff[i];
  }
  set_tableau(M.scheme, T);
  for (int b = 0; b < nb; ++b) {
    T.mass[b] = M.mass[b]; T.inertia[b] = M.inertia[b];
    T.minv[b] = M.minv[b]; T.iinv[b] = M.iinv[b];
    T.contact[b] = M.body[b].contact;
    T.nadj[b] = std::min(M.nadj[b], NODE_MAXADJ);
    for (int t = 0; t < T.nadj[b]; ++t) T.adj[b][t] = (unsigned char)M.adj[b][t];
    if (M.body[b].contact >= 0) {
      const int i = M.body[b].contact;
      T.cbody[i] = b;
      T.crho[i][0] = M.body[b].crho[0];
      T.crho[i][1] = M.body[b].crho[1];
      T.mu[i] = M.body[b].mu;
    }
  }
  for (int j = 0; j < nj; ++j) {
    T.jpar[j] = M.jpar[j]; T.jchi[j] = M.jchi[j];
    T.jrp[j][0] = M.jrp[j][0]; T.jrp[j][1] = M.jrp[j][1];
    T.jrc[j][0] = M.jrc[j][0]; T.jrc[j][1] = M.jrc[j][1];
  }
  // row classes
  const int nq = 3 * nb;
  for (int r = 0; r < M.nxt; ++r) { T.lrow[r] = -1; T.qrow[r] = -1; }
  int nl = 0, nqd = 0;
  for (int b = 0; b < nb; ++b) {
    T.lrow[3 * b + 2] = (short)nl++;
    T.lrow[nq + 3 * b + 2] = (short)nl++;
    const bool foot = M.body[b].contact >= 0;
    for (int c2 = 0; c2 < 2; ++c2) {
      if (foot) {
        T.lrow[3 * b + c2] = (short)nl++;
        T.lrow[nq + 3 * b + c2] = (short)nl++;
      } else {
        T.qrow[3 * b + c2] = (short)nqd++;
        T.qrow[nq + 3 * b + c2] = (short)nqd++;
      }
    }
  }
  for (int r = 6 * nb; r < M.nxt; ++r) T.qrow[r] = (short)nqd++;
  T.nlive = nl;
  T.nquad = nqd;
  // integrated columns: every column but the closed-form ones
  int cnt = 0;
  for (int c = 0; c < T.C; ++c) {
    const bool trivial = c < M.nxt && cpl_col_kind(M, c) != 0;
    if (!trivial) T.cperm[cnt++] = (short)c;
  }
  T.cnt = cnt;
  T.colptr[0] = 0;
  for (int c = 0; c < M.nxt; ++c) T.colptr[c + 1] = T.colptr[c] + cpl_col_nnz(M, c);
  // stage data
  T.ncf = M.aux ? CPL_CF1 : CPL_CF0;
  T.sd_arm = 0;
  T.sd_qw = T.sd_arm + 4 * nj;
  T.sd_F = T.sd_qw + nb;
  T.sd_K = T.sd_F + M.nxt;
  T.sd_con = T.sd_K + T.nsky;
  T.sd_size = T.sd_con + T.ncf * nc;
  // nominal kernel scratch (doubles per lane)
  const bool acc = T.nks == 1;  // RK4 keeps an accumulator; RKF45 sums its stored slopes
  T.n_xl = 0;
  T.n_xs = T.n_xl + nl;
  T.n_acc = T.n_xs + nl;
  T.n_k = T.n_acc + (acc ? nl : 0);
  T.n_xq = T.n_k + T.nks * nl;
  T.n_f = T.n_xq + nqd;
  T.n_arm = T.n_f + 3 * nb;
  T.n_carm = T.n_arm + 4 * nj;
  T.n_K = T.n_carm + 2 * nc;
  T.n_lam = T.n_K + T.nsky;
  T.n_qw = T.n_lam + T.nk;
  T.n_size = T.n_qw + nb;
  // tangent kernel scratch (elements per thread)
  T.t_pl = 0;
  T.t_acc = T.t_pl + nl;
  T.t_k = T.t_acc + (acc ? nl : 0);
  T.t_xs = T.t_k + T.nks * nl;
  T.t_pq = T.t_xs + nl;
  T.t_e = T.t_pq + nqd;
  T.t_x = T.t_e + 3 * nb;
  T.t_size = T.t_x + T.nk;
  for (int i = 0; i < CPL_MAXSTAGE; ++i) {
    T.cf[i] = (float)T.c[i];
    T.bf[i] = (float)T.b[i];
    T.betaf[i] = (float)T.beta[i];
    for (int j = 0; j < CPL_MAXSTAGE; ++j) T.af[i][j] = (float)T.a[i][j];
  }
  for (int b = 0; b < nb; ++b) {
    T.minvf[b] = (float)T.minv[b];
    T.iinvf[b] = (float)T.iinv[b];
  }
  if ((size_t)T.n_size * sizeof(double) * 32 > 220u * 1024u)
    return "model too large for the coupled path's shared memory";
  return nullptr;
}

size_t cpl_interval_bytes(const CplTab& T, int nsub, int prec) {
  const size_t el = prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
  return (size_t)nsub * T.stages * T.sd_size * el;
}

cudaError_t launch_coupled(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                           const double* U, const double* s, void* A, void* Bm, void* Bp, void* S,
                           double* defect, double* penalty, void* ws, long chunk,
                           unsigned* status, cudaStream_t st, const int2* entries,
                           const DevInst* inst, bool compact) {
  const int c = compact ? 1 : 0;
  if (prec == CISCVX_FP64)
    return T.scheme ? run<double, 1>(T, N, nsub, layout, X, U, s, A, Bm, Bp, S, defect, penalty, ws, chunk, status, st, entries, inst, c)
                    : run<double, 0>(T, N, nsub, layout, X, U, s, A, Bm, Bp, S, defect, penalty, ws, chunk, status, st, entries, inst, c);
  return T.scheme ? run<float, 1>(T, N, nsub, layout, X, U, s, A, Bm, Bp, S, defect, penalty, ws, chunk, status, st, entries, inst, c)
                  : run<float, 0>(T, N, nsub, layout, X, U, s, A, Bm, Bp, S, defect, penalty, ws, chunk, status, st, entries, inst, c);
}

CplAdjLayout cpl_adjoint_layout(const CplTab& T, long n, int nsub, int prec) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  CplAdjLayout Ly;
  Ly.stage = 0;
  Ly.defect = al(Ly.stage + (size_t)n * cpl_interval_bytes(T, nsub, prec));
  Ly.penalty = al(Ly.defect + (size_t)n * T.nxt * sizeof(double));
  Ly.ubar = al(Ly.penalty + (size_t)n * (T.nc > 0 ? T.nc : 1) * sizeof(double));
  Ly.lpart = al(Ly.ubar + (size_t)n * 2 * (T.nu > 0 ? T.nu : 1) * sizeof(double));
  Ly.total = al(Ly.lpart + ADJ_LRED_BLOCKS * sizeof(double));
  return Ly;
}

size_t cpl_adjoint_bytes(const CplTab& T, long n, int nsub, int prec) {
  return cpl_adjoint_layout(T, n, nsub, prec).total;
}

cudaError_t launch_coupled_vjp(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                               const double* U, const double* s, const double* w, const double* rho,
                               double* gX, double* gU, double* gs, double* L, void* ws, size_t ws_bytes,
                               unsigned* status, cudaStream_t st) {
  if (prec == CISCVX_FP64)
    return T.scheme ? run_vjp<double, 1>(T, N, nsub, layout, X, U, s, w, rho, gX, gU, gs, L, ws, ws_bytes, status, st)
                    : run_vjp<double, 0>(T, N, nsub, layout, X, U, s, w, rho, gX, gU, gs, L, ws, ws_bytes, status, st);
  return T.scheme ? run_vjp<float, 1>(T, N, nsub, layout, X, U, s, w, rho, gX, gU, gs, L, ws, ws_bytes, status, st)
                  : run_vjp<float, 0>(T, N, nsub, layout, X, U, s, w, rho, gX, gU, gs, L, ws, ws_bytes, status, st);
}

cudaError_t launch_coupled_and_vjp(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                                   const double* U, const double* s, void* A, void* Bm, void* Bp, void* S,
                                   double* defect, double* penalty, const double* w, const double* rho,
                                   double* gX, double* gU, double* gs, double* L, void* ws, size_t ws_bytes,
                                   unsigned* status, cudaStream_t st, bool compact) {
  const int c = compact ? 1 : 0;
#define CISCVX_BOTH(TP, SCH)                                                                               \
  run_both<TP, SCH>(T, N, nsub, layout, X, U, s, A, Bm, Bp, S, defect, penalty, w, rho, gX, gU, gs, L, ws, \
                    ws_bytes, status, st, c)
  if (prec == CISCVX_FP64) return T.scheme ? CISCVX_BOTH(double, 1) : CISCVX_BOTH(double, 0);
  return T.scheme ? CISCVX_BOTH(float, 1) : CISCVX_BOTH(float, 0);
#undef CISCVX_BOTH
}

cudaError_t cpl_prepare(const CplTab& T, int prec) {
  cpl_jit_tangent(T, prec);
  cpl_jit_nominal(T, prec);
  cpl_jit_adjoint(T, prec);
  if (prec == CISCVX_FP64) return T.scheme ? prepare<double, 1>(T) : prepare<double, 0>(T);
  return T.scheme ? prepare<float, 1>(T) : prepare<float, 0>(T);
}

}  // namespace ciscvx
