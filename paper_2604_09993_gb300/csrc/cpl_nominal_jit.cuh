// cpl_nominal_jit.cuh — device source of the coupled path's nominal kernel,
// compiled at run time (NVRTC) once per model shape, like the tangent kernel
// (cpl_tangent_jit.cuh; the same generated prelude precedes it, plus CPL_NW,
// the warps per block).  It computes what k_cpl_nominal in coupled.cu
// computes — the FP64 state over the scheme's stages, the stage data the
// tangents read (same layout), defects, penalty increments and the
// closed-form columns of A — with the model's shape fixed at compile time,
// and with fewer FP64 instructions:
//  * the stage sin/cos of every link angle come from those at the substep
//    start by angle addition with a Taylor series of the increment
//    (sincos_step), and those at the substep start from the previous ones;
//  * K = L D L^T is factored with one reciprocal per row (no square root),
//    an FP32 estimate refined by Newton-Raphson steps in FP64;
//  * the penalty values use the a rsqrt(a) - 1 form, and the slopes the
//    tangents need are taken in the tangent precision;
//  * on the sinusoidal surface, sin/cos of tk x at each contact point come
//    from those at the substep's first stage the same way, and the frame's
//    normalization is one rsqrt;
//  * FP32 stage data are narrowed on the integer pipe (to_f32_rz): a
//    conversion instruction would take an FP64-pipe slot.
// The stored stage slopes, K, the quadrature rows and the lever arms sit in
// shared memory (element major); the live rows, stage values, generalized
// forces and sin/cos stay in registers.  Under RKF45 only the slopes of the
// live rows that are not kinematic are stored: theta and the contact links'
// p have the slope s v, so their stage values are
// x0 + h s c_j v0 + h^2 s sum_m (A^2)_jm k_m(v) and their substep update is
// h s v0 + h^2 s sum_m beta_m k_m(v), beta = b^T A.
constexpr int SCH = CPL_SCH;
constexpr int NW = CPL_NW;
constexpr int BLK = 32 * NW;
constexpr int NSTG = SCH ? 6 : 4;
constexpr int NKS = SCH ? 5 : 1;
constexpr int NQ = 3 * NB;
// shared-memory elements per lane
constexpr int NKR = SCH ? NLD : NL;  // rows whose slopes are stored
constexpr int E_K = 0, E_KST = E_K + NSKY, E_ACC = E_KST + NKS * NKR,
              E_XQ = E_ACC + (NKS == 1 ? NL : 0), E_ARM = E_XQ + NQD, E_SIZE = E_ARM + 4 * NJ;

struct NumN {
  double mass[NB], minv[NB], iinv[NB];
  double jrp[NJ > 0 ? NJ : 1][2], jrc[NJ > 0 ? NJ : 1][2];
  double crho[NC > 0 ? NC : 1][2], mu[NC > 0 ? NC : 1];
  double g, ta, tk;
};

using namespace ciscvx;

// FP64 value -> stage-data precision (FP32: toward zero, on the integer pipe)
__device__ __forceinline__ void narrow_to(float& d, double x) { d = to_f32_rz(x); }
__device__ __forceinline__ void narrow_to(double& d, double x) { d = x; }
__device__ __forceinline__ TP nar(double x) {
  TP r;
  narrow_to(r, x);
  return r;
}

__device__ __forceinline__ TP ramp_slope(double z) { return huber_slope(nar(z)); }

// 1 / d for a pivot of K's L D L^T factor: an FP32 estimate (rcp.approx,
// error about one FP32 ulp, with d narrowed and the estimate widened on the
// integer pipe) refined by two Newton-Raphson steps r <- r + r (1 - d r) in
// FP64.  Each step squares the relative error (2^-22 -> 2^-44 -> below FP64
// rounding), so the result is within a few FP64 ulp of 1 / d; four FP64
// instructions on the critical path of the factorization instead of a
// correctly rounded division.  Pivots of magnitude outside 2^-100 .. 2^100
// (and zeros and non-finite values, whose results are non-finite either way)
// take the division.
__device__ __forceinline__ double pivot_inv(double d) {
  const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7FFu;  // biased exponent
  if (ex < 1023u - 100u || ex > 1023u + 100u) return 1.0 / d;
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(to_f32_rz(d)));
  double r = widen(rf);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}
// pseudo-Huber absolute value sqrt(1 + x^2) - 1 (FP64) as a rsqrt(a) - 1
__device__ __forceinline__ double sabs_v(double x) {
  const double a = fma(x, x, 1.0);
  return fma(a, rsqrt(a), -1.0);
}

extern "C" __global__ void __launch_bounds__(BLK) cpl_nominal(const __grid_constant__ NumN P, long i0,
                                                             long n, int nsub, int layout,
                                                             const double* __restrict__ X,
                                                             const double* __restrict__ U,
                                                             const double* __restrict__ s,
                                                             TP* __restrict__ sd, TP* __restrict__ A,
                                                             double* __restrict__ defect,
                                                             double* __restrict__ penalty,
                                                             unsigned* status,
                                                             const int2* __restrict__ entries,
                                                             const InstRec* __restrict__ inst, int cmp) {
  extern __shared__ double jit_sm1[];
  double* sm = jit_sm1 + threadIdx.x;
#define SE(o) sm[(o) * BLK]
  const long t = (long)blockIdx.x * BLK + threadIdx.x;
  if (t >= n) return;
  const unsigned active = __activemask();
  const double *uL, *uR, *x0;
  double sk;
  {
    const IvRef ad = iv_ref(i0 + t, NXT, NU, NC, layout, entries, inst, 0);
    uL = U + ad.u;
    uR = U + ad.u + NU;
    x0 = X + ad.x;
    sk = s[ad.s];
  }
  const double h = 1.0 / nsub;
  double xl[NL], f[3 * NB], qw[NB], sn0[NB], cs0[NB];
#pragma unroll
  for (int r = 0; r < NXT; ++r) {
    const double v = x0[r];
    if (LROW[r] >= 0) xl[LROW[r]] = v;
    else SE(E_XQ + QROW[r]) = v;
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) sincos(xl[LROW[3 * b + 2]], &sn0[b], &cs0[b]);
  TP* sdk = sd + (size_t)t * nsub * NSTG * SD_SIZE;
  // sinusoidal surface: tk xc and its sin/cos at each contact, first stage of the substep
  double targ0[NC > 0 ? NC : 1], tsn0[NC > 0 ? NC : 1], tcs0[NC > 0 ? NC : 1];

  for (int i = 0; i < nsub; ++i) {
    // quadrature rows: p += h s v at the substep start
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (CONTACT[b] >= 0) continue;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
        SE(E_XQ + QROW[3 * b + c2]) = fma(h * sk, SE(E_XQ + QROW[NQ + 3 * b + c2]), SE(E_XQ + QROW[3 * b + c2]));
    }
    double th_start[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) th_start[b] = xl[LROW[3 * b + 2]];
    for (int j = 0; j < NSTG; ++j) {
      const double tau = (i + TABD_C[j]) * h;
      const double bj = TABD_B[j];
      const double h2b = h * h * sk * TABD_BETA[j];
      TP* D = sdk + (size_t)(i * NSTG + j) * SD_SIZE;
      // stage values of the live rows: xs = xl + d, d = h sum_m a_jm k_m
      // (the increments first: the angle increments give the stage sin/cos)
      double xs[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) xs[l] = 0.0;
      if (SCH) {
        for (int m = 0; m < j; ++m) {
          const double ah = TABD_A(j, m) * h, a2h = TABD_A2(j, m) * (h * h * sk);
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            if (LVEL[l] < 0) {
              if (ah != 0.0) xs[l] = fma(ah, SE(E_KST + m * NKR + LDYN[l]), xs[l]);
            } else if (a2h != 0.0) {
              xs[l] = fma(a2h, SE(E_KST + m * NKR + LDYN[LVEL[l]]), xs[l]);
            }
          }
        }
#pragma unroll
        for (int l = 0; l < NL; ++l)
          if (LVEL[l] >= 0) xs[l] = fma(h * sk * TABD_C[j], xl[LVEL[l]], xs[l]);
      } else if (j > 0) {
        const double ah = TABD_A(j, j - 1) * h;
#pragma unroll
        for (int l = 0; l < NL; ++l) xs[l] = ah * SE(E_KST + l);
      }
      // stage sin/cos
      double sn[NB], cs[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (j == 0) { sn[b] = sn0[b]; cs[b] = cs0[b]; }
        else sincos_step(th_start[b], sn0[b], cs0[b], xs[LROW[3 * b + 2]], active, sn[b], cs[b]);
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) xs[l] += xl[l];
      auto u_at = [&](int q) { return (1.0 - tau) * uL[q] + tau * uR[q]; };
      // records F_r and integrates row r with the slope s F_r
      auto emit = [&](int r, double Fv) {
        D[SD_F + r] = nar(Fv);
        const double kv = sk * Fv;
        const int l = LROW[r];
        if (l >= 0) {
          if (NKS == 1) {
            if (j < NSTG - 1) SE(E_KST + l) = kv;
            const double acc = (j == 0) ? bj * kv : fma(bj, kv, SE(E_ACC + l));
            if (j < NSTG - 1) SE(E_ACC + l) = acc;
            else xl[l] = fma(h, acc, xl[l]);
          } else if (LVEL[l] >= 0) {
            // kinematic: from the velocity's stored slopes; the velocity's own
            // update comes later in this stage (its rows are emitted after)
            if (j == NSTG - 1) {
              double acc = 0.0;
#pragma unroll
              for (int m = NSTG - 2; m >= 0; --m)
                if (TABD_BETA[m] != 0.0) acc = fma(TABD_BETA[m], SE(E_KST + m * NKR + LDYN[LVEL[l]]), acc);
              xl[l] = fma(h * sk, fma(h, acc, xl[LVEL[l]]), xl[l]);
            }
          } else if (j < NSTG - 1) {
            SE(E_KST + j * NKR + LDYN[l]) = kv;
          } else {
            double acc = bj * kv;
#pragma unroll
            for (int m = NSTG - 2; m >= 0; --m)
              if (m != 1) acc = fma(TABD_B[m], SE(E_KST + m * NKR + LDYN[l]), acc);
            xl[l] = fma(h, acc, xl[l]);
          }
        } else {
          const int q = QROW[r];
          SE(E_XQ + q) = fma(h * bj, kv, SE(E_XQ + q));
          if (r >= NQ && r < 2 * NQ && (r - NQ) % 3 != 2)
            SE(E_XQ + QROW[r - NQ]) = fma(h2b, kv, SE(E_XQ + QROW[r - NQ]));
        }
      };
      // lever arms
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
#pragma unroll
        for (int role = 0; role < 2; ++role) {
          const int b = role ? JPAR[jj] : JCHI[jj];
          const double* rho = role ? P.jrp[jj] : P.jrc[jj];
          const double rx = fma(cs[b], rho[0], -sn[b] * rho[1]), ry = fma(sn[b], rho[0], cs[b] * rho[1]);
          SE(E_ARM + 4 * jj + 2 * role) = rx;
          SE(E_ARM + 4 * jj + 2 * role + 1) = ry;
          D[SD_ARM + 4 * jj + 2 * role] = nar(rx);
          D[SD_ARM + 4 * jj + 2 * role + 1] = nar(ry);
        }
      }
      // generalized forces and QW (the -dtheta coefficient of the torque's derivative)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        f[3 * b] = 0.0;
        f[3 * b + 1] = -P.mass[b] * P.g;
        f[3 * b + 2] = 0.0;
        qw[b] = 0.0;
      }
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int c = JCHI[jj], p = JPAR[jj];
        const double tq = u_at(jj);
        f[3 * c + 2] += tq;
        f[3 * p + 2] -= tq;
        if (!JELIM) {
          const double lx = u_at(NJ + 2 * jj), ly = u_at(NJ + 2 * jj + 1);
          const double rcx = SE(E_ARM + 4 * jj), rcy = SE(E_ARM + 4 * jj + 1);
          const double rpx = SE(E_ARM + 4 * jj + 2), rpy = SE(E_ARM + 4 * jj + 3);
          f[3 * c] += lx;
          f[3 * c + 1] += ly;
          f[3 * c + 2] += fma(rcx, ly, -rcy * lx);
          f[3 * p] -= lx;
          f[3 * p + 1] -= ly;
          f[3 * p + 2] -= fma(rpx, ly, -rpy * lx);
          qw[c] += fma(rcx, lx, rcy * ly);
          qw[p] -= fma(rpx, lx, rpy * ly);
        }
      }
      // contacts
#pragma unroll
      for (int ic = 0; ic < NC; ++ic) {
        const int b = CBODY[ic];
        const double rx = fma(cs[b], P.crho[ic][0], -sn[b] * P.crho[ic][1]);
        const double ry = fma(sn[b], P.crho[ic][0], cs[b] * P.crho[ic][1]);
        const double xc = xs[LROW[3 * b]] + rx, yc = xs[LROW[3 * b + 1]] + ry;
        SurfFrame fr;
        if (TERRAIN) {
          // sin/cos of tk xc: evaluated at the substep's first stage, chained
          // from there at the later stages (tk (xc - xc_0) stays small)
          double ssn, scs;
          if (j == 0) {
            targ0[ic] = P.tk * xc;
            sincos(targ0[ic], &tsn0[ic], &tcs0[ic]);
            ssn = tsn0[ic];
            scs = tcs0[ic];
          } else {
            sincos_step(targ0[ic], tsn0[ic], tcs0[ic], fma(P.tk, xc, -targ0[ic]), active, ssn, scs);
          }
          fr = contact_surface_sc(P.ta, P.tk, yc, ssn, scs);
        } else {
          fr = contact_surface(0.0, P.tk, xc, yc);
        }
        const double u0 = u_at(CI0 + 3 * ic), u1 = u_at(CI0 + 3 * ic + 1), u2 = u_at(CI0 + 3 * ic + 2);
        const double ft = AUX ? u0 : u1 - u2, fn = AUX ? u1 : u0;
        const double fx = fma(fr.tx, ft, fr.nx * fn), fy = fma(fr.ty, ft, fr.ny * fn);
        f[3 * b] += fx;
        f[3 * b + 1] += fy;
        f[3 * b + 2] += fma(rx, fy, -ry * fx);
        qw[b] += fma(rx, fx, ry * fy);
        TP* Dc = D + SD_CON + NCF * ic;
        Dc[0] = nar(rx); Dc[1] = nar(ry);
        Dc[2] = nar(fr.tx); Dc[3] = nar(fr.ty); Dc[4] = nar(fr.nx); Dc[5] = nar(fr.ny);
        Dc[6] = nar(fma(fr.dtx, ft, fr.dnx * fn));
        Dc[7] = nar(fma(fr.dty, ft, fr.dny * fn));
        Dc[8] = nar(fr.phix); Dc[9] = nar(fr.phiy);
        const double mu = P.mu[ic];
        if (!AUX) {
          const double zc = u1 + u2 - mu * u0;
          const double H = huber_value(-u0) + huber_value(-u1) + huber_value(-u2) + huber_value(-fr.phi) +
                           huber_value(zc);
          const TP d1 = ramp_slope(-u0), d2 = ramp_slope(-u1), d3 = ramp_slope(-u2), dp = ramp_slope(-fr.phi),
                   d5 = ramp_slope(zc);
          Dc[10] = -dp;
          Dc[11] = -d1 - nar(mu) * d5;
          Dc[12] = -d2 + d5;
          Dc[13] = -d3 + d5;
          emit(6 * NB + ic, H);
        } else {
          const double gam = u2;
          const double om = xs[LROW[NQ + 3 * b + 2]];
          const double vcx = fma(-om, ry, xs[LROW[NQ + 3 * b]]);
          const double vcy = fma(om, rx, xs[LROW[NQ + 3 * b + 1]]);
          const double at = fma(ft, ft, 1.0), rt = rsqrt(at);
          const double rho_c = sabs_v(mu * fn) - fma(at, rt, -1.0);
          const double lam = fma(fr.tx, vcx, fr.ty * vcy) + gam * (ft * rt);
          const double H = huber_value(-fn) + huber_value(-fr.phi) + huber_value(-gam) + huber_value(-rho_c);
          const TP ftP = nar(ft), mfn = nar(mu * fn);
          const TP rtP = TP(1) / sqrt(TP(1) + ftP * ftP);
          const TP dft = ftP * rtP, dmn = mfn / sqrt(TP(1) + mfn * mfn);
          const TP drh = ramp_slope(-rho_c);
          const TP rho_ft = -dft, rho_fn = nar(mu) * dmn;
          Dc[10] = -ramp_slope(-fr.phi);
          Dc[11] = drh * dft;
          Dc[12] = -ramp_slope(-fn) - drh * rho_fn;
          Dc[13] = -ramp_slope(-gam);
          Dc[14] = nar(vcx); Dc[15] = nar(vcy);
          Dc[16] = nar(fma(fr.dtx, vcx, fr.dty * vcy));
          Dc[17] = nar(gam) * rtP * rtP * rtP;
          Dc[18] = dft;
          Dc[19] = rho_ft;
          Dc[20] = rho_fn;
          emit(6 * NB + 4 * ic, fn);
          emit(6 * NB + 4 * ic + 1, lam);
          emit(6 * NB + 4 * ic + 2, gam);
          emit(6 * NB + 4 * ic + 3, rho_c);
          emit(6 * NB + 4 * NC + ic, H);
        }
      }
      // Eq. (3): K lambda = kappa - grad C M^-1 F, then F += grad C^T lambda
      if (JELIM && NK > 0) {
#define KS(i, kk) SE(E_K + NOFF[i] + (kk) - NF[i])
#pragma unroll
        for (int r1 = 0; r1 < NK; ++r1) {
          const int j1 = NORD[r1 >> 1], a1 = r1 & 1;
#pragma unroll
          for (int r2 = 0; r2 <= r1; ++r2) {
            if (r2 < NF[r1]) continue;
            const int j2 = NORD[r2 >> 1], a2 = r2 & 1;
            double acc = 0.0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int b1 = u ? JPAR[j1] : JCHI[j1];
              const double p1 = a1 ? SE(E_ARM + 4 * j1 + 2 * u) : -SE(E_ARM + 4 * j1 + 2 * u + 1);
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                const int b2 = v ? JPAR[j2] : JCHI[j2];
                if (b1 != b2) continue;
                const double p2 = a2 ? SE(E_ARM + 4 * j2 + 2 * v) : -SE(E_ARM + 4 * j2 + 2 * v + 1);
                const double e = fma(p1 * p2, P.iinv[b1], (a1 == a2) ? P.minv[b1] : 0.0);
                acc = (u == v) ? acc + e : acc - e;
              }
            }
            KS(r1, r2) = acc;
          }
        }
        // K = L D L^T within the envelopes: row i holds t_k = L_ik D_k while it
        // is formed, then L_ik = t_k / D_k; the diagonal slot holds 1 / D_i
#pragma unroll
        for (int ii = 0; ii < NK; ++ii) {
#pragma unroll
          for (int kk = 0; kk < ii; ++kk) {
            if (kk < NF[ii]) continue;
            double acc = KS(ii, kk);
#pragma unroll
            for (int m = 0; m < kk; ++m)
              if (m >= NF[ii] && m >= NF[kk]) acc = fma(-KS(ii, m), KS(kk, m), acc);
            KS(ii, kk) = acc;
          }
          double dd = KS(ii, ii);
#pragma unroll
          for (int kk = 0; kk < ii; ++kk) {
            if (kk < NF[ii]) continue;
            const double tk = KS(ii, kk);
            const double l = tk * KS(kk, kk);
            dd = fma(-tk, l, dd);
            KS(ii, kk) = l;
          }
          KS(ii, ii) = pivot_inv(dd);
        }
#pragma unroll
        for (int e = 0; e < NSKY; ++e) D[SD_K + e] = nar(SE(E_K + e));
        double lam[NK > 0 ? NK : 1];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          double a0 = 0.0, a1 = 0.0;
#pragma unroll
          for (int role = 0; role < 2; ++role) {
            const int b = role ? JPAR[jj] : JCHI[jj];
            const double rx = SE(E_ARM + 4 * jj + 2 * role), ry = SE(E_ARM + 4 * jj + 2 * role + 1);
            const double om = xs[LROW[NQ + 3 * b + 2]];
            const double aa = f[3 * b + 2] * P.iinv[b];
            const double c0 = fma(om * om, rx, fma(ry, aa, -f[3 * b] * P.minv[b]));
            const double c1 = fma(om * om, ry, fma(-rx, aa, -f[3 * b + 1] * P.minv[b]));
            if (role) { a0 -= c0; a1 -= c1; } else { a0 += c0; a1 += c1; }
          }
          lam[2 * NPOS[jj]] = a0;
          lam[2 * NPOS[jj] + 1] = a1;
        }
#pragma unroll
        for (int ii = 1; ii < NK; ++ii) {
          double acc = lam[ii];
#pragma unroll
          for (int kk = 0; kk < ii; ++kk)
            if (kk >= NF[ii]) acc = fma(-KS(ii, kk), lam[kk], acc);
          lam[ii] = acc;
        }
#pragma unroll
        for (int ii = NK - 1; ii >= 0; --ii) {
          double acc = lam[ii] * KS(ii, ii);
#pragma unroll
          for (int kk = ii + 1; kk < NK; ++kk)
            if (NF[kk] <= ii) acc = fma(-KS(kk, ii), lam[kk], acc);
          lam[ii] = acc;
        }
#undef KS
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const double lx = lam[2 * NPOS[jj]], ly = lam[2 * NPOS[jj] + 1];
          const int c = JCHI[jj], p = JPAR[jj];
          const double rcx = SE(E_ARM + 4 * jj), rcy = SE(E_ARM + 4 * jj + 1);
          const double rpx = SE(E_ARM + 4 * jj + 2), rpy = SE(E_ARM + 4 * jj + 3);
          f[3 * c] += lx;
          f[3 * c + 1] += ly;
          f[3 * c + 2] += fma(rcx, ly, -rcy * lx);
          f[3 * p] -= lx;
          f[3 * p + 1] -= ly;
          f[3 * p + 2] -= fma(rpx, ly, -rpy * lx);
          qw[c] += fma(rcx, lx, rcy * ly);
          qw[p] -= fma(rpx, lx, rpy * ly);
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) D[SD_QW + b] = nar(qw[b]);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        emit(3 * b + 2, xs[LROW[NQ + 3 * b + 2]]);
        if (CONTACT[b] >= 0) {
          emit(3 * b, xs[LROW[NQ + 3 * b]]);
          emit(3 * b + 1, xs[LROW[NQ + 3 * b + 1]]);
        } else if (j == 0) {
          D[SD_F + 3 * b] = nar(SE(E_XQ + QROW[NQ + 3 * b]));
          D[SD_F + 3 * b + 1] = nar(SE(E_XQ + QROW[NQ + 3 * b + 1]));
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        emit(NQ + 3 * b, f[3 * b] * P.minv[b]);
        emit(NQ + 3 * b + 1, f[3 * b + 1] * P.minv[b]);
        emit(NQ + 3 * b + 2, f[3 * b + 2] * P.iinv[b]);
      }
    }
    // sin/cos at the next substep start
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double sn, cs;
      sincos_step(th_start[b], sn0[b], cs0[b], xl[LROW[3 * b + 2]] - th_start[b], active, sn, cs);
      sn0[b] = sn;
      cs0[b] = cs;
    }
  }
  double chk = 0.0;
  const IvRef ad = iv_ref(i0 + t, NXT, NU, NC, layout, entries, inst,
                          cmp ? (long long)COLPTR[NXT] : (long long)NXT * NXT);
  const double* x1 = x0 + NXT;
#pragma unroll
  for (int r = 0; r < NXT; ++r) {
    const double x = LROW[r] >= 0 ? xl[LROW[r]] : SE(E_XQ + QROW[r]);
    const double dv = x - x1[r];
    defect[ad.v + r] = dv;
    chk += dv;
  }
#pragma unroll
  for (int ic = 0; ic < NC; ++ic) {
    const int r = PEN0 + ic;
    const double x = LROW[r] >= 0 ? xl[LROW[r]] : SE(E_XQ + QROW[r]);
    penalty[ad.p + ic] = x - x0[r];
  }
  if (!isfinite(chk)) atomicOr(status, 1u);
  // closed-form columns of A: e_p, e_v + s e_p (links without a contact), e_y
  // (not written by the adjoint's forward pass, which has no A)
  if (!A) return;
  TP* Ak = A + ad.a;
  if (cmp) {  // compact (column-major): e_p -> 1; e_v + s e_p -> (s, 1); e_y -> 1
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (CONTACT[b] >= 0) continue;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        const int cp = 3 * b + c2, cv = NQ + 3 * b + c2;
        Ak[COLPTR[cp]] = TP(1);
        Ak[COLPTR[cv]] = TP(sk);
        Ak[COLPTR[cv] + 1] = TP(1);
      }
    }
#pragma unroll
    for (int c = 6 * NB; c < NXT; ++c) Ak[COLPTR[c]] = TP(1);
    return;
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (CONTACT[b] >= 0) continue;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      const int cp = 3 * b + c2, cv = NQ + 3 * b + c2;
      for (int r = 0; r < NXT; ++r) {
        Ak[(size_t)r * NXT + cp] = (r == cp) ? TP(1) : TP(0);
        Ak[(size_t)r * NXT + cv] = (r == cv) ? TP(1) : (r == cp ? TP(sk) : TP(0));
      }
    }
  }
  for (int c = 6 * NB; c < NXT; ++c)
    for (int r = 0; r < NXT; ++r) Ak[(size_t)r * NXT + c] = (r == c) ? TP(1) : TP(0);
#undef SE
}
