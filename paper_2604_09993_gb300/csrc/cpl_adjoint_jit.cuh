// cpl_adjoint_jit.cuh — device source of the coupled path's reverse-mode
// adjoint kernel, compiled at run time (NVRTC) once per model shape, with the
// prelude the tangent kernel gets (sizes, topology, row maps, skyline
// structure, stage-data layout and tableau as compile-time constants).  The
// arithmetic is that of k_cpl_adjoint in coupled.cu (see its comments): per
// substep and stage, in reverse, the transpose of the tangent kernel's stage
// map — slopes, the Eq. (3) solve by the recorded L D L^T factor of K (K is
// symmetric), contacts and direct inputs — from the cotangent of x~(1).  With
// static indices the cotangents (live and quadrature rows, generalized force,
// KKT vector, input cotangents) live in registers; under RKF45 the slope
// cotangents of the six stages stay in shared memory (every stage feeds all
// earlier ones), under RK4 only the next stage's term is carried.
constexpr int SCH = CPL_SCH;
constexpr int BS = CPL_BS;
constexpr int NSTG = SCH ? 6 : 4;

struct NumA {
  TP minv[NB], iinv[NB];
};

extern "C" __global__ void __launch_bounds__(BS) cpl_adjoint(const __grid_constant__ NumA P, long i0, long n,
                                                            long N, int nsub, const double* __restrict__ s,
                                                            const TP* __restrict__ sd,
                                                            const double* __restrict__ w,
                                                            const double* __restrict__ rho,
                                                            double* __restrict__ gX,
                                                            double* __restrict__ gs,
                                                            double* __restrict__ ubar, unsigned* status) {
  extern __shared__ __align__(16) unsigned char jit_smem[];
  TP* ksh = reinterpret_cast<TP*>(jit_smem) + threadIdx.x;  // RKF45: slope cotangents, element major
  const long t = (long)blockIdx.x * BS + threadIdx.x;
  if (t >= n) return;
  const long k = i0 + t;
  constexpr int NQ = 3 * NB;
  constexpr int NU2 = NU > 0 ? 2 * NU : 1;
  TP PL[NL], PQ[NQD > 0 ? NQD : 1], UB[NU2], PLE[NL], KN[NL];
  const double* wk = w + k * NXT;
#pragma unroll
  for (int r = 0; r < NXT; ++r) {
    double v = wk[r];
    if (r >= PEN0 && r < PEN0 + NC) v += rho[k * NC + (r - PEN0)];
    if (LROW[r] >= 0) PL[LROW[r]] = TP(v);
    else PQ[QROW[r]] = TP(v);
  }
#pragma unroll
  for (int q = 0; q < NU2; ++q) UB[q] = TP(0);
  const TP sk = TP(s[k]);
  const TP h = TP(1) / TP(nsub);
  const TP hsk = h * sk;
  TP sbar = TP(0);
  const TP* sdk = sd + (size_t)t * nsub * NSTG * SD_SIZE;

  for (int i = nsub - 1; i >= 0; --i) {
    if (SCH) {
      for (int j = 0; j < NSTG; ++j) {
        const TP hb = h * TAB_B[j];
#pragma unroll
        for (int l = 0; l < NL; ++l) ksh[(j * NL + l) * BS] = hb * PL[l];
      }
    } else {
#pragma unroll
      for (int l = 0; l < NL; ++l) { PLE[l] = PL[l]; KN[l] = TP(0); }
    }
    for (int j = NSTG - 1; j >= 0; --j) {
      const TP* D = sdk + (size_t)(i * NSTG + j) * SD_SIZE;
      const TP* F = D + SD_F;
      const TP bj = TAB_B[j], hbj = h * bj, h2b = h * h * sk * TAB_BETA[j];
      const TP tau = (TP(i) + TAB_C[j]) * h;
      const TP wl = TP(1) - tau, wr = tau;
      TP KB[NL];
#pragma unroll
      for (int l = 0; l < NL; ++l) KB[l] = SCH ? ksh[(j * NL + l) * BS] : hbj * PLE[l] + KN[l];
      TP XS[NL], e[3 * NB];
#pragma unroll
      for (int l = 0; l < NL; ++l) XS[l] = TP(0);
#pragma unroll
      for (int c = 0; c < 3 * NB; ++c) e[c] = TP(0);
      // ---- slopes (transposed) ----
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const TP mi = P.minv[b], ii = P.iinv[b];
        {
          const TP kb = KB[LROW[3 * b + 2]];
          XS[LROW[NQ + 3 * b + 2]] += sk * kb;
          sbar += kb * F[3 * b + 2];
        }
        {
          const TP kb = KB[LROW[NQ + 3 * b + 2]];
          e[3 * b + 2] += sk * kb * ii;
          sbar += kb * F[NQ + 3 * b + 2];
        }
        if (CONTACT[b] >= 0) {
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            const TP kp = KB[LROW[3 * b + c2]];
            XS[LROW[NQ + 3 * b + c2]] += sk * kp;
            sbar += kp * F[3 * b + c2];
            const TP kv = KB[LROW[NQ + 3 * b + c2]];
            e[3 * b + c2] += sk * kv * mi;
            sbar += kv * F[NQ + 3 * b + c2];
          }
        } else {
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            const TP Pp = PQ[QROW[3 * b + c2]], Pv = PQ[QROW[NQ + 3 * b + c2]];
            const TP kvb = h2b * Pp + hbj * Pv;
            e[3 * b + c2] += sk * kvb * mi;
            sbar += kvb * F[NQ + 3 * b + c2] + Pp * h2b * F[NQ + 3 * b + c2];
            if (j == 0) sbar += Pp * h * F[3 * b + c2];
          }
        }
      }
      // ---- Eq. (3) (transposed) ----
      if (JELIM && NK > 0) {
        TP x[NK > 0 ? NK : 1];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          TP lx = TP(0), ly = TP(0);
#pragma unroll
          for (int role = 0; role < 2; ++role) {
            const int b = role ? JPAR[jj] : JCHI[jj];
            const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
            const TP vx = e[3 * b] - ry * e[3 * b + 2], vy = e[3 * b + 1] + rx * e[3 * b + 2];
            if (role) { lx -= vx; ly -= vy; } else { lx += vx; ly += vy; }
          }
          x[2 * NPOS[jj]] = lx;
          x[2 * NPOS[jj] + 1] = ly;
        }
        const TP* Kf = D + SD_K;
#pragma unroll
        for (int ii = 1; ii < NK; ++ii) {
          TP acc = x[ii];
#pragma unroll
          for (int kk = 0; kk < ii; ++kk)
            if (kk >= NF[ii]) acc -= Kf[NOFF[ii] + kk - NF[ii]] * x[kk];
          x[ii] = acc;
        }
#pragma unroll
        for (int ii = NK - 1; ii >= 0; --ii) {
          TP acc = x[ii] * Kf[NOFF[ii] + ii - NF[ii]];
#pragma unroll
          for (int kk = ii + 1; kk < NK; ++kk)
            if (NF[kk] <= ii) acc -= Kf[NOFF[kk] + ii - NF[kk]] * x[kk];
          x[ii] = acc;
        }
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const TP a0b = x[2 * NPOS[jj]], a1b = x[2 * NPOS[jj] + 1];
#pragma unroll
          for (int role = 0; role < 2; ++role) {
            const int b = role ? JPAR[jj] : JCHI[jj];
            const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
            const TP om = F[3 * b + 2], omd = F[NQ + 3 * b + 2];
            const TP c0 = role ? -a0b : a0b, c1 = role ? -a1b : a1b;
            XS[LROW[NQ + 3 * b + 2]] += TP(2) * om * (rx * c0 + ry * c1);
            XS[LROW[3 * b + 2]] += (-om * om * ry + omd * rx) * c0 + (om * om * rx + omd * ry) * c1;
            e[3 * b] -= P.minv[b] * c0;
            e[3 * b + 1] -= P.minv[b] * c1;
            e[3 * b + 2] += P.iinv[b] * (ry * c0 - rx * c1);
          }
        }
      }
      // ---- contacts (transposed) ----
#pragma unroll
      for (int ic = 0; ic < NC; ++ic) {
        const int b = CBODY[ic];
        const TP* Dc = D + SD_CON + NCF * ic;
        const TP rx = Dc[0], ry = Dc[1];
        const TP fxb = e[3 * b] - ry * e[3 * b + 2], fyb = e[3 * b + 1] + rx * e[3 * b + 2];
        TP ftb = Dc[2] * fxb + Dc[3] * fyb, fnb = Dc[4] * fxb + Dc[5] * fyb, gab = TP(0);
        TP xcb = Dc[6] * fxb + Dc[7] * fyb, phib = TP(0);
        const int u0 = CI0 + 3 * ic;
        if (!AUX) {
          const int row = 6 * NB + ic;
          const TP kvb = hbj * PQ[QROW[row]];
          sbar += kvb * F[row];
          const TP yb = sk * kvb;
          phib = Dc[10] * yb;
          const TP g0 = fnb + Dc[11] * yb, g1 = ftb + Dc[12] * yb, g2 = -ftb + Dc[13] * yb;
          UB[u0] += wl * g0; UB[NU + u0] += wr * g0;
          UB[u0 + 1] += wl * g1; UB[NU + u0 + 1] += wr * g1;
          UB[u0 + 2] += wl * g2; UB[NU + u0 + 2] += wr * g2;
        } else {
          const int rows[5] = {6 * NB + 4 * ic, 6 * NB + 4 * ic + 1, 6 * NB + 4 * ic + 2,
                               6 * NB + 4 * ic + 3, 6 * NB + 4 * NC + ic};
          TP y[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const TP kvb = hbj * PQ[QROW[rows[q]]];
            sbar += kvb * F[rows[q]];
            y[q] = sk * kvb;
          }
          fnb += y[0] + Dc[20] * y[3] + Dc[12] * y[4];
          gab += y[2] + Dc[18] * y[1] + Dc[13] * y[4];
          ftb += Dc[17] * y[1] + Dc[19] * y[3] + Dc[11] * y[4];
          xcb += Dc[16] * y[1];
          phib = Dc[10] * y[4];
          const TP om = F[3 * b + 2];
          const TP vxb = Dc[2] * y[1], vyb = Dc[3] * y[1];
          XS[LROW[NQ + 3 * b]] += vxb;
          XS[LROW[NQ + 3 * b + 1]] += vyb;
          XS[LROW[NQ + 3 * b + 2]] += -ry * vxb + rx * vyb;
          XS[LROW[3 * b + 2]] += -om * (rx * vxb + ry * vyb);
          UB[u0] += wl * ftb; UB[NU + u0] += wr * ftb;
          UB[u0 + 1] += wl * fnb; UB[NU + u0 + 1] += wr * fnb;
          UB[u0 + 2] += wl * gab; UB[NU + u0 + 2] += wr * gab;
        }
        xcb += Dc[8] * phib;
        const TP ycb = Dc[9] * phib;
        XS[LROW[3 * b]] += xcb;
        XS[LROW[3 * b + 1]] += ycb;
        XS[LROW[3 * b + 2]] += -ry * xcb + rx * ycb;
      }
      // ---- direct inputs: torques, and reaction forces when they are inputs ----
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const TP g = e[3 * JCHI[jj] + 2] - e[3 * JPAR[jj] + 2];
        UB[jj] += wl * g;
        UB[NU + jj] += wr * g;
        if (!JELIM) {
#pragma unroll
          for (int cp = 0; cp < 2; ++cp) {
            TP v = TP(0);
#pragma unroll
            for (int role = 0; role < 2; ++role) {
              const int b = role ? JPAR[jj] : JCHI[jj];
              const TP rx = D[SD_ARM + 4 * jj + 2 * role], ry = D[SD_ARM + 4 * jj + 2 * role + 1];
              const TP c = e[3 * b + cp] + (cp ? rx : -ry) * e[3 * b + 2];
              v = role ? v - c : v + c;
            }
            UB[NJ + 2 * jj + cp] += wl * v;
            UB[NU + NJ + 2 * jj + cp] += wr * v;
          }
        }
      }
      // ---- moving application points ----
#pragma unroll
      for (int b = 0; b < NB; ++b) XS[LROW[3 * b + 2]] -= D[SD_QW + b] * e[3 * b + 2];
      // stage-tangent cotangent -> the substep start and the earlier stages' slopes
#pragma unroll
      for (int l = 0; l < NL; ++l) PL[l] += XS[l];
      if (SCH) {
        for (int m = 0; m < j; ++m) {
          const TP ah = TAB_A(j, m) * h;
          if (ah == TP(0)) continue;
#pragma unroll
          for (int l = 0; l < NL; ++l) ksh[(m * NL + l) * BS] += ah * XS[l];
        }
      } else if (j > 0) {
        const TP ah = TAB_A(j, j - 1) * h;
#pragma unroll
        for (int l = 0; l < NL; ++l) KN[l] = ah * XS[l];
      }
    }
    // p += h s v at the substep start (links without a contact)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (CONTACT[b] >= 0) continue;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) PQ[QROW[NQ + 3 * b + c2]] += hsk * PQ[QROW[3 * b + c2]];
    }
  }
  double chk = 0.0;
#pragma unroll
  for (int r = 0; r < NXT; ++r) {
    double v = (double)(LROW[r] >= 0 ? PL[LROW[r]] : PQ[QROW[r]]);
    if (r >= PEN0 && r < PEN0 + NC) v -= rho[k * NC + (r - PEN0)];
    if (k >= 1) v -= w[(k - 1) * NXT + r];
    gX[k * NXT + r] = v;
    if (k == N - 1) gX[N * NXT + r] = -wk[r];
    chk += v;
  }
  gs[k] = (double)sbar;
  double* ub = ubar + (size_t)t * 2 * NU;
#pragma unroll
  for (int q = 0; q < 2 * NU; ++q) ub[q] = (double)UB[q];
  if (!isfinite(chk + (double)sbar)) atomicOr(status, 1u);
}
