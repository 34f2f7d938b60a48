// vjp_link.cuh — one link of one interval of the discrete-adjoint VJP, shared
// by the single-instance and the batched kernels (see vjp.cu).
#pragma once
#include "common.cuh"

namespace ciscvx {

template <typename TP, bool FOOT>
__device__ __forceinline__ void vjp_link(const DevModel& M, int b, int nsub, double sd,
                                         const double* __restrict__ xk,
                                         const double* __restrict__ xk1,
                                         const double* __restrict__ uL,
                                         const double* __restrict__ uR,
                                         const double* __restrict__ wk,
                                         const double* __restrict__ wkm1, double rho_c,
                                         double* __restrict__ gXk, double* __restrict__ gXN,
                                         double* __restrict__ part, double* __restrict__ ps,
                                         double* __restrict__ pL, unsigned* status) {
  const DevBody& B = M.body[b];
  const int nb = M.nb;
  const double g = M.g;
  const int nin = B.nin;
  double AxL = 0, AxR = 0, AyL = 0, AyR = 0, PL = 0, PR = 0, QL = 0, QR = 0, TL = 0, TR = 0;
  for (int i = 0; i < nin; ++i) {
    const int q = B.idx[i];
    const double a = uL[q], c = uR[q];
    AxL = fma(B.ax[i], a, AxL); AxR = fma(B.ax[i], c, AxR);
    AyL = fma(B.ay[i], a, AyL); AyR = fma(B.ay[i], c, AyR);
    PL = fma(B.p[i], a, PL); PR = fma(B.p[i], c, PR);
    QL = fma(B.q[i], a, QL); QR = fma(B.q[i], c, QR);
    TL = fma(B.t[i], a, TL); TR = fma(B.t[i], c, TR);
  }
  const int rpx = 3 * b, rpy = rpx + 1, rth = rpx + 2;
  const int rvx = 3 * nb + 3 * b, rvy = rvx + 1, rom = rvx + 2;
  const double px0 = xk[rpx], py0 = xk[rpy], th0 = xk[rth];
  const double vx0 = xk[rvx], vy0 = xk[rvy], om0 = xk[rom];
  const double axm = 0.5 * (AxL + AxR), ax3 = AxL * (1.0 / 3.0) + AxR * (1.0 / 6.0);
  const double aym = 0.5 * (AyL + AyR) - g, ay3 = AyL * (1.0 / 3.0) + AyR * (1.0 / 6.0) - 0.5 * g;
  const double px1 = px0 + sd * vx0 + sd * sd * ax3, vx1 = vx0 + sd * axm;
  const double py1 = py0 + sd * vy0 + sd * sd * ay3, vy1 = vy0 + sd * aym;
  const double dP = PR - PL, dQ = QR - QL, dT = TR - TL, dAy = AyR - AyL;
  const int cin = B.cin;
  double lnL = 0, lnD = 0, tpL = 0, tpD = 0, tmL = 0, tmD = 0;
  if (FOOT) {
    lnL = uL[cin]; lnD = uR[cin] - lnL;
    tpL = uL[cin + 1]; tpD = uR[cin + 1] - tpL;
    tmL = uL[cin + 2]; tmD = uR[cin + 2] - tmL;
  }
  const double mu = B.mu, crx = B.crho[0], cry = B.crho[1];
  const double h = 1.0 / nsub;

  // ---- forward sweep: checkpoints and x~(1) ----
  double ck_th[MAXSUB_VJP], ck_om[MAXSUB_VJP], ck_py[FOOT ? MAXSUB_VJP : 1],
      ck_vy[FOOT ? MAXSUB_VJP : 1];
  double th = th0, om = om0, py = py0, vy = vy0, Yom = 0.0;
  for (int i = 0; i < nsub; ++i) {
    ck_th[i] = th; ck_om[i] = om;
    if (FOOT) { ck_py[i] = py; ck_vy[i] = vy; }
    double kth = 0, kom = 0, ath = 0, aom = 0, kpy = 0, kvy = 0, apy = 0, avy = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double cj = rk_c(j), wj = rk_w(j), tj = (i + cj) * h;
      const double ths = (j == 0) ? th : fma(cj * h, kth, th);
      const double ws = (j == 0) ? om : fma(cj * h, kom, om);
      double sn, cs;
      sincos(ths, &sn, &cs);
      const double wdot = fma(cs, fma(tj, dP, PL), fma(-sn, fma(tj, dQ, QL), fma(tj, dT, TL)));
      kth = sd * ws; kom = sd * wdot;
      ath = fma(wj, kth, ath); aom = fma(wj, kom, aom);
      if (FOOT) {
        const double pys = (j == 0) ? py : fma(cj * h, kpy, py);
        const double vs = (j == 0) ? vy : fma(cj * h, kvy, vy);
        kpy = sd * vs; kvy = sd * (fma(tj, dAy, AyL) - g);
        apy = fma(wj, kpy, apy); avy = fma(wj, kvy, avy);
        const double ry = sn * crx + cs * cry;
        const double ln = fma(tj, lnD, lnL), ltp = fma(tj, tpD, tpL), ltm = fma(tj, tmD, tmL);
        double H1, D1, H2, D2, H3, D3, H4, D4, H5, D5;
        huber(-ln, H1, D1); huber(-ltp, H2, D2); huber(-ltm, H3, D3);
        huber(-(pys + ry), H4, D4); huber(ltp + ltm - mu * ln, H5, D5);
        Yom = fma(h * wj, H1 + H2 + H3 + H4 + H5, Yom);
      }
    }
    th = fma(h, ath, th); om = fma(h, aom, om);
    if (FOOT) { py = fma(h, apy, py); vy = fma(h, avy, vy); }
  }

  // cotangents of x~(1): w_k (+ rho on the penalty state)
  const double wpx = wk[rpx], wpy = wk[rpy], wth = wk[rth], wvx = wk[rvx], wvy = wk[rvy], wom = wk[rom];
  int ry_ = -1;
  double wy = 0.0, lam_y = 0.0;
  if (FOOT) { ry_ = 6 * nb + B.contact; wy = wk[ry_]; lam_y = wy + rho_c; }

  // L share: w . defect over this link's rows (+ rho . penalty)
  double Lp = wpx * (px1 - xk1[rpx]) + wpy * (py1 - xk1[rpy]) + wth * (th - xk1[rth]) +
              wvx * (vx1 - xk1[rvx]) + wvy * (vy1 - xk1[rvy]) + wom * (om - xk1[rom]);
  if (FOOT) {
    const double pen = sd * Yom;
    Lp += wy * (xk[ry_] + pen - xk1[ry_]) + rho_c * pen;
  }

  // ---- backward sweep ----
  TP lth = TP(wth), lom = TP(wom), lpy = TP(0), lvy = TP(0);
  const TP ly = TP(lam_y), sdP = TP(sd), hP = TP(h);
  TP gsd = TP(0), gPL = TP(0), gPR = TP(0), gQL = TP(0), gQR = TP(0), gTL = TP(0), gTR = TP(0);
  TP gAyL = TP(0), gAyR = TP(0), gd[6] = {TP(0), TP(0), TP(0), TP(0), TP(0), TP(0)};
  for (int i = nsub - 1; i >= 0; --i) {
    // recompute the four stages of substep i from its checkpoint
    TP cs_[4], sn_[4], sath[4], oms[4], wdt[4], tau[4];
    TP gr[4], gp[4], vys[4], ays[4], om_pen[4], dl0[4], dl1[4], dl2[4];
    {
      const double thc = ck_th[i], omc = ck_om[i];
      double pyc = 0, vyc = 0;
      if (FOOT) { pyc = ck_py[i]; vyc = ck_vy[i]; }
      double kth = 0, kom = 0, kpy = 0, kvy = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double cj = rk_c(j), tj = (i + cj) * h;
        const double ths = (j == 0) ? thc : fma(cj * h, kth, thc);
        const double ws = (j == 0) ? omc : fma(cj * h, kom, omc);
        double sn, cs;
        sincos(ths, &sn, &cs);
        const double P = fma(tj, dP, PL), Q = fma(tj, dQ, QL), T = fma(tj, dT, TL);
        const double wdot = fma(cs, P, fma(-sn, Q, T));
        kth = sd * ws; kom = sd * wdot;
        cs_[j] = TP(cs); sn_[j] = TP(sn);
        sath[j] = TP(-sd * fma(sn, P, cs * Q));
        oms[j] = TP(ws); wdt[j] = TP(wdot); tau[j] = TP(tj);
        if (FOOT) {
          const double pys = (j == 0) ? pyc : fma(cj * h, kpy, pyc);
          const double vs = (j == 0) ? vyc : fma(cj * h, kvy, vyc);
          const double ay = fma(tj, dAy, AyL) - g;
          kpy = sd * vs; kvy = sd * ay;
          const double rx = cs * crx - sn * cry, ry = sn * crx + cs * cry;
          const double ln = fma(tj, lnD, lnL), ltp = fma(tj, tpD, tpL), ltm = fma(tj, tmD, tmL);
          double H1, D1, H2, D2, H3, D3, H4, D4, H5, D5;
          huber(-ln, H1, D1); huber(-ltp, H2, D2); huber(-ltm, H3, D3);
          huber(-(pys + ry), H4, D4); huber(ltp + ltm - mu * ln, H5, D5);
          gp[j] = TP(-sd * D4);
          gr[j] = TP(-sd * D4 * rx);
          vys[j] = TP(vs); ays[j] = TP(ay);
          om_pen[j] = TP(H1 + H2 + H3 + H4 + H5);
          dl0[j] = TP(sd * (-D1 - mu * D5));
          dl1[j] = TP(sd * (-D2 + D5));
          dl2[j] = TP(sd * (-D3 + D5));
        }
      }
    }
    // transposed stages j = 3..0
    TP mth = TP(0), mom = TP(0), mpy = TP(0), mvy = TP(0);  // mu_{j+1}
    TP sth = TP(0), som = TP(0), spy = TP(0), svy = TP(0);  // sum of mu_j
#pragma unroll
    for (int j = 3; j >= 0; --j) {
      const TP hw = hP * TP(rk_w(j));
      const TP cnext = (j == 3) ? TP(0) : TP(rk_c(j + 1)) * hP;
      const TP gth = hw * lth + cnext * mth;   // dL/dk_j (theta)
      const TP gom = hw * lom + cnext * mom;   // dL/dk_j (omega)
      TP nth = sath[j] * gom;                  // J_j^T: theta <- s a_theta g_omega
      const TP nom = sdP * gth;                // omega <- s g_theta
      const TP wl = TP(1) - tau[j], wr = tau[j];
      gsd += gth * oms[j] + gom * wdt[j];
      const TP gc = gom * sdP * cs_[j], gs_ = -gom * sdP * sn_[j], g1 = gom * sdP;
      gPL += gc * wl; gPR += gc * wr;
      gQL += gs_ * wl; gQR += gs_ * wr;
      gTL += g1 * wl; gTR += g1 * wr;
      if (FOOT) {
        const TP inj = hw * ly;
        nth += inj * gr[j];
        const TP gpy = hw * lpy + cnext * mpy;
        const TP gvy = hw * lvy + cnext * mvy;
        const TP npy = inj * gp[j];
        const TP nvy = sdP * gpy;
        gsd += gpy * vys[j] + gvy * ays[j] + inj * om_pen[j];
        gAyL += gvy * sdP * wl; gAyR += gvy * sdP * wr;
        gd[0] += inj * dl0[j] * wl; gd[3] += inj * dl0[j] * wr;
        gd[1] += inj * dl1[j] * wl; gd[4] += inj * dl1[j] * wr;
        gd[2] += inj * dl2[j] * wl; gd[5] += inj * dl2[j] * wr;
        mpy = npy; mvy = nvy; spy += npy; svy += nvy;
      }
      mth = nth; mom = nom; sth += nth; som += nom;
    }
    lth += sth; lom += som;
    if (FOOT) { lpy += spy; lvy += svy; }
  }

  // ---- translation: transposed closed forms ----
  const double s2_3 = sd * sd / 3.0, s2_6 = sd * sd / 6.0, s_2 = 0.5 * sd;
  const double gAxL = wpx * s2_3 + wvx * s_2, gAxR = wpx * s2_6 + wvx * s_2;
  const double gAyLt = wpy * s2_3 + wvy * s_2 + double(gAyL), gAyRt = wpy * s2_6 + wvy * s_2 + double(gAyR);
  const double gsd_t = wpx * (vx0 + 2.0 * sd * ax3) + wvx * axm + wpy * (vy0 + 2.0 * sd * ay3) +
                       wvy * aym + double(gsd);

  // node-state gradient of this link's rows: own part minus w_{k-1} (defect_{k-1} subtracts x~_k)
  const double own[6] = {wpx, wpy + double(lpy), double(lth), wpx * sd + wvx,
                         wpy * sd + wvy + double(lvy), double(lom)};
  const int rows[6] = {rpx, rpy, rth, rvx, rvy, rom};
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int r = rows[t];
    gXk[r] = own[t] - (wkm1 ? wkm1[r] : 0.0);
    if (gXN) gXN[r] = -wk[r];
  }
  if (FOOT) {
    gXk[ry_] = wy - (wkm1 ? wkm1[ry_] : 0.0);  // y(1) = y_k + ..., minus rho for penalty_k
    if (gXN) gXN[ry_] = -wk[ry_];
  }
  // per-input partials of this link
  double* pp = part + 2 * B.slot0;
  for (int i = 0; i < nin; ++i) {
    double gl = B.ax[i] * gAxL + B.ay[i] * gAyLt + B.p[i] * double(gPL) + B.q[i] * double(gQL) +
                B.t[i] * double(gTL);
    double gr_ = B.ax[i] * gAxR + B.ay[i] * gAyRt + B.p[i] * double(gPR) + B.q[i] * double(gQR) +
                 B.t[i] * double(gTR);
    if (FOOT) {
      const int d = B.idx[i] - cin;
      if (d >= 0 && d < 3) { gl += double(gd[d]); gr_ += double(gd[3 + d]); }
    }
    pp[2 * i] = gl;
    pp[2 * i + 1] = gr_;
  }
  ps[b] = gsd_t;
  pL[b] = Lp;
  if (!finite_d(Lp + gsd_t + double(lth) + double(lom))) atomicOr(status, ST_NONFINITE);
}

}  // namespace ciscvx
