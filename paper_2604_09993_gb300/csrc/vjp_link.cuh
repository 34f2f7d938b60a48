// vjp_link.cuh — one link of one interval of the discrete-adjoint VJP, shared
// by the single-instance and the batched kernels (see vjp.cu).
//
// Forward sweep: the FP64 state, checkpointed at every substep start.
// Backward sweep: per substep, the four stages are recomputed from the
// checkpoint and the transposed stage Jacobians are applied in the adjoint
// precision TP.
//  * FP64 adjoint: the checkpoints are (theta, omega, sin theta, cos theta),
//    and (p_y, v_y) for a foot link; the stages are recomputed in FP64
//    (sin/cos chained as in the forward kernel) and the penalty quadrature
//    (for L) is taken there.
//  * FP32 adjoint: the checkpoints are the FP32 anchors of the stage
//    recursion (theta, omega, and p_y, v_y for a foot link, narrowed on the
//    integer pipe), the penalty quadrature is taken in the forward sweep on
//    the FP64 stages, and the backward sweep recomputes the stages in FP32
//    from the anchors with tau in FP32, so it issues no FP64 instruction per
//    substep.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "disc_link.cuh"

namespace ciscvx {

// FUSED: the forward sweep was run by the discretization (disc_link with CK);
// its checkpoints, end state and penalty quadrature come in through *ckin.
// CROSS: a foot link of the Eq. (12) model (Sec. IV-A).  Its contact adds
// four cross-complementarity rows (phi_n, lambda^c, gamma, rho^c) and its
// path-penalty row takes the input terms of that model (input_cross in
// disc_link.cuh).  Of these only lambda^c depends on the link's state: its
// integrand v_x - omega (R rho)_y + G(u) puts sources on the stage values of
// theta, omega and v_x in the backward sweep (v_x gets an adjoint channel of
// its own, forced like v_y); the other rows are integrals of the inputs
// alone, whose gradients are their quadrature weights times the slopes.  The
// forward sweep is the FP64 one in both precisions and takes all quadratures
// (fused: the discretization's sweep, handed over in the checkpoints).
template <typename TP, bool FOOT, bool FUSED = false, bool CROSS = false>
__device__ __forceinline__ void vjp_link(const DevModel& M, int b, int nsub, double sd,
                                         const double* __restrict__ xk,
                                         const double* __restrict__ xk1,
                                         const double* __restrict__ uL,
                                         const double* __restrict__ uR,
                                         const double* __restrict__ wk,
                                         const double* __restrict__ wkm1, double rho_c,
                                         double* __restrict__ gXk, double* __restrict__ gXN,
                                         double* __restrict__ part, double* __restrict__ ps,
                                         double* __restrict__ pL, unsigned* status,
                                         const Checkpoints* ckin = nullptr) {
  constexpr bool F32 = std::is_same<TP, float>::value;
  constexpr bool cross = FOOT && CROSS;
  const unsigned amask = __activemask();  // lanes running this link (they stay converged)
  const DevBody& B = M.body[b];
  const int nb = M.nb;
  const double g = M.g;
  const int nin = B.nin;
  double AxL = 0, AxR = 0, AyL = 0, AyR = 0, PL = 0, PR = 0, QL = 0, QR = 0, TL = 0, TR = 0;
  if constexpr (FUSED) {  // formed by the discretization's forward sweep
    AxL = ckin->ins[0]; AxR = ckin->ins[1]; AyL = ckin->ins[2]; AyR = ckin->ins[3];
    PL = ckin->ins[4]; PR = ckin->ins[5]; QL = ckin->ins[6]; QR = ckin->ins[7];
    TL = ckin->ins[8]; TR = ckin->ins[9];
  } else {
    for (int i = 0; i < nin; ++i) {
      const int q = B.idx[i];
      const double a = uL[q], c = uR[q];
      AxL = fma(B.ax[i], a, AxL); AxR = fma(B.ax[i], c, AxR);
      AyL = fma(B.ay[i], a, AyL); AyR = fma(B.ay[i], c, AyR);
      PL = fma(B.p[i], a, PL); PR = fma(B.p[i], c, PR);
      QL = fma(B.q[i], a, QL); QR = fma(B.q[i], c, QR);
      TL = fma(B.t[i], a, TL); TR = fma(B.t[i], c, TR);
    }
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
  double cL[3] = {0, 0, 0}, cD[3] = {0, 0, 0};
  TP cLP[3], cDP[3];
  if (FOOT) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      cL[m] = uL[cin + m];
      cD[m] = uR[cin + m] - cL[m];
      cLP[m] = anchor<TP>(cL[m]);
      cDP[m] = anchor<TP>(cD[m]);
    }
  }
  const double mu = B.mu, crx = B.crho[0], cry = B.crho[1];
  const TP muP = anchor<TP>(mu), crxP = anchor<TP>(crx), cryP = anchor<TP>(cry);
  // FP32 copies narrowed on the integer pipe (see to_f32_rz)
  const TP PLP = anchor<TP>(PL), dPP = anchor<TP>(dP), QLP = anchor<TP>(QL), dQP = anchor<TP>(dQ),
           TLP = anchor<TP>(TL), dTP = anchor<TP>(dT);
  const TP AyLP = anchor<TP>(AyL), dAyP = anchor<TP>(dAy), gP = anchor<TP>(g);
  const double h = FUSED ? ckin->h : 1.0 / nsub, h2 = 0.5 * h;
  const TP sdP = anchor<TP>(sd), hP = anchor<TP>(h), h2P = anchor<TP>(h2);
  const TP cjhP[4] = {TP(0), h2P, h2P, hP};
  // input-only terms of the path penalty (Eq. (12) model: and of the cross
  // rows) at one time; H64: FP64 values (the cross terms always have them)
  using IP = typename std::conditional<cross, InputCross<TP>, InputPenalty<TP>>::type;
  auto ipen = [&](auto h64, double t, TP tP) -> IP {
    if constexpr (cross) return input_cross<TP>(t, tP, sdP, mu, muP, cL, cD, cLP, cDP);
    else return input_penalty<TP, decltype(h64)::value>(t, tP, sd, sdP, mu, muP, cL, cD, cLP, cDP);
  };
  using H64 = std::true_type;
  using HP = std::integral_constant<bool, !F32>;
  // Eq. (12) model: x-acceleration sums (lambda^c's v_x stages)
  const double dAx = AxR - AxL, sAxL = sd * AxL, sdAxs = sd * dAx;
  const TP AxLP = anchor<TP>(AxL), dAxP = anchor<TP>(dAx);
  double Il = 0.0, Ir = 0.0, Ig = 0.0;  // lambda^c state part, rho^c, lambda^c input part

  // ---- forward sweep: FP64 state and checkpoints ----
  Checkpoints ckl;  // own forward sweep (unused when FUSED)
  ckl.sm = nullptr;
  const Checkpoints& ck = FUSED ? *ckin : ckl;
  double th = th0, om = om0, py = py0, vy = vy0;
  // FP32 adjoint: the penalty quadrature is taken here, on the FP64 forward
  // stages, so that the backward sweep needs no FP64 work at all.
  constexpr bool PEN_FWD = FOOT && (F32 || cross);
  double Yom = 0.0;
  if constexpr (FUSED) {
    th = ck.th_end;
    om = ck.om_end;
    Yom = ck.Yom;
    if constexpr (cross) { Il = ck.Il; Ir = ck.Ir; Ig = ck.Ig; }
  } else if constexpr (F32 && !cross) {
    // FP32 adjoint: stage values in float-float, the state accumulated in FP64
    // (state_df.cuh); the anchors at every substep start are the checkpoints,
    // and the penalty quadrature is taken here.
    const DfLink C = df_link(sd, nsub, PL, dP, QL, dQ, TL, dT, AyL, dAy, g, FOOT, crx, cry, mu, cL, cD);
    DfState S = df_state_init<FOOT>(C, th0, om0, py0, vy0);
    for (int i = 0; i < nsub; ++i) {
      ckl.thf[i] = anchor<TP>(S.th); ckl.omf[i] = anchor<TP>(S.om);
      if (FOOT) { ckl.pyf[i] = anchor<TP>(S.py); ckl.vyf[i] = anchor<TP>(S.vy); }
      df_substep<FOOT, false>(C, i, amask, S, nullptr);
    }
    df_state_finish<FOOT>(C, S);
    th = S.th;
    om = S.om;
    Yom = S.Y;
  } else {
  double sth, cth;
  sincos(th, &sth, &cth);
  IP fp0, fpm, fp1;
  // input-only penalty terms as Simpson per substep (see disc_link.cuh)
  const double h3 = h * (1.0 / 3.0), h23 = 2.0 * h3, h6 = 0.5 * h3;
  if (PEN_FWD) {
    fp0 = ipen(H64(), 0.0, TP(0));
    Yom = h6 * fp0.H;
    if constexpr (cross) { Ir = h6 * fp0.R; Ig = h6 * fp0.G; }
  }
  double vx = vx0;  // Eq. (12) model: v_x for lambda^c
  // The forward sweep needs only the state: slopes from s-scaled input sums
  // (k_theta = s omega_stage, k_omega = s (cos P - sin Q + T)), s P, s Q, s T
  // carried from each substep end to the next start.
  const double sPL = sd * PL, sdPs = sd * dP, sQL = sd * QL, sdQs = sd * dQ;
  const double sTL = sd * TL, sdTs = sd * dT;
  const double sAyg = sd * (AyL - g), sdAys = sd * dAy;
  const double sc2 = sd * h2, sc3 = sd * h;
  double sPi = sPL, sQi = sQL, sTi = sTL;
  double ti = 0.0;  // tau at the substep start (running sum)
  TP tiP = TP(0);
  for (int i = 0; i < nsub; ++i) {
    if constexpr (F32) {  // the FP32 backward sweep needs only the FP32 anchors
      ckl.thf[i] = anchor<TP>(th); ckl.omf[i] = anchor<TP>(om);
      if (FOOT) { ckl.pyf[i] = anchor<TP>(py); ckl.vyf[i] = anchor<TP>(vy); }
    } else {
      ckl.th[i] = th; ckl.om[i] = om; ckl.s[i] = sth; ckl.c[i] = cth;
      if (FOOT) { ckl.py[i] = py; ckl.vy[i] = vy; }
    }
    const double tm = ti + h2, te = ti + h;
    if (PEN_FWD) {
      fpm = ipen(H64(), tm, tiP + h2P);
      fp1 = ipen(H64(), te, tiP + hP);
    }
    double kth = 0, kom = 0, ath = 0, aom = 0, kpy = 0, kvy = 0, apy = 0, avy = 0, kvx = 0, avx = 0;
    const double som = sd * om, svy = FOOT ? sd * vy : 0.0;
    double sPm = 0, sQm = 0, sTm = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double wj = rk_w(j);
      const double cjh = (j == 0) ? 0.0 : (j == 3 ? h : h2);
      const double tj = (j == 0) ? ti : (j == 3 ? te : tm);
      const double dth = cjh * kth;
      double sn, cs;
      if (j == 0) { sn = sth; cs = cth; }
      else sincos_step(th, sth, cth, dth, amask, sn, cs);
      double sP, sQ, sT;
      if (j == 0) { sP = sPi; sQ = sQi; sT = sTi; }
      else if (j == 3) {
        sPi = fma(te, sdPs, sPL); sQi = fma(te, sdQs, sQL); sTi = fma(te, sdTs, sTL);
        sP = sPi; sQ = sQi; sT = sTi;
      } else {
        if (j == 1) { sPm = fma(tm, sdPs, sPL); sQm = fma(tm, sdQs, sQL); sTm = fma(tm, sdTs, sTL); }
        sP = sPm; sQ = sQm; sT = sTm;
      }
      const double wst = cross ? ((j == 0) ? om : fma(cjh, kom, om)) : 0.0;  // stage omega
      kth = (j == 0) ? som : fma(j == 3 ? sc3 : sc2, kom, som);
      kom = fma(cs, sP, fma(-sn, sQ, sT));
      ath = fma(wj, kth, ath); aom = fma(wj, kom, aom);
      if (FOOT) {
        if (PEN_FWD) {
          const double pys = (j == 0) ? py : fma(cjh, kpy, py);
          const double ry = fma(sn, crx, cs * cry);
          Yom = fma(h * wj, huber_value(-(pys + ry)), Yom);
          if constexpr (cross) {  // lambda^c's state part v_x - omega (R rho)_y
            const double vxs = (j == 0) ? vx : fma(cjh, kvx, vx);
            kvx = fma(tj, sdAxs, sAxL);
            avx = fma(wj, kvx, avx);
            Il = fma(h * wj, fma(-wst, ry, vxs), Il);
          }
        }
        kpy = (j == 0) ? svy : fma(j == 3 ? sc3 : sc2, kvy, svy);
        kvy = fma(tj, sdAys, sAyg);
        apy = fma(wj, kpy, apy); avy = fma(wj, kvy, avy);
      }
    }
    if (PEN_FWD) {
      Yom = fma(h3, fp1.H, fma(h23, fpm.H, Yom));
      if constexpr (cross) {
        Ir = fma(h3, fp1.R, fma(h23, fpm.R, Ir));
        Ig = fma(h3, fp1.G, fma(h23, fpm.G, Ig));
        vx = fma(h, avx, vx);
      }
      fp0 = fp1;
    }
    const double Dth = h * ath;
    double s1, c1;
    sincos_step(th, sth, cth, Dth, amask, s1, c1);
    sth = s1; cth = c1;
    th += Dth;
    om = fma(h, aom, om);
    if (FOOT) { py = fma(h, apy, py); vy = fma(h, avy, vy); }
    ti = te;
    tiP = tiP + hP;
  }
  if (PEN_FWD) {  // the end point was counted with h/3
    Yom = fma(-h6, fp0.H, Yom);
    if constexpr (cross) { Ir = fma(-h6, fp0.R, Ir); Ig = fma(-h6, fp0.G, Ig); }
  }
  }  // own forward sweep

  // cotangents of x~(1): w_k (+ rho on the penalty state)
  const double wpx = wk[rpx], wpy = wk[rpy], wth = wk[rth], wvx = wk[rvx], wvy = wk[rvy], wom = wk[rom];
  int ry_ = -1;
  double wy = 0.0, lam_y = 0.0;
  if (FOOT) { ry_ = 6 * nb + (cross ? 4 * M.nc : 0) + B.contact; wy = wk[ry_]; lam_y = wy + rho_c; }
  // Eq. (12) model: cotangents of the contact's rows phi_n, lambda^c, gamma, rho^c
  const int yb = cross ? 6 * nb + 4 * B.contact : 0;
  double wc[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (cross) {
#pragma unroll
    for (int t = 0; t < 4; ++t) wc[t] = wk[yb + t];
  }
  const TP wlP = anchor<TP>(wc[1]), wrP = anchor<TP>(wc[3]);

  // ---- backward sweep ----
  TP lth = anchor<TP>(wth), lom = anchor<TP>(wom), lpy = TP(0), lvy = TP(0);
  const TP ly = anchor<TP>(lam_y);
  TP gsd = TP(0), gPL = TP(0), gPR = TP(0), gQL = TP(0), gQR = TP(0), gTL = TP(0), gTR = TP(0);
  TP gAyL = TP(0), gAyR = TP(0), gd[6] = {TP(0), TP(0), TP(0), TP(0), TP(0), TP(0)};
  TP lvx = TP(0), gAxLc = TP(0), gAxRc = TP(0);  // Eq. (12) model: v_x channel
  // input penalty at the end of the current substep (FP64 values only for the
  // FP64 adjoint, which takes the penalty quadrature here, last substep first)
  IP ipE;
  if (FOOT) ipE = ipen(HP(), 1.0, TP(1));
  double di = (double)(nsub - 1);
  TP fi = TP(nsub - 1);  // substep index in the tangent precision (exact)
  for (int i = nsub - 1; i >= 0; --i, di -= 1.0, fi -= TP(1)) {
    TP cs_[4], sn_[4], sath[4], oms[4], wdt[4], tau[4];
    TP gr[4], gp[4], vys[4], ays[4], om_pen[4], dl0[4], dl1[4], dl2[4];
    // Eq. (12) model: lambda^c's sources on theta and omega (s-scaled), the
    // x acceleration, and the input-only slopes of lambda^c (q) and rho^c (r)
    TP lsth[4], lsom[4], axs[4], q0[4], q2[4], r0[4], r1[4];
    // substep start / midpoint / end: FP64 for the FP64 adjoint; the FP32
    // adjoint takes them in FP32 and issues no FP64 instruction per substep
    const double tsb = di * h, tmb = tsb + h2, teb = tsb + h;
    const TP tsP = F32 ? fi * hP : TP(tsb), tmP = tsP + h2P, teP = tsP + hP;
    IP ipS, ipM;
    if (FOOT) {
      ipM = ipen(HP(), tmb, tmP);
      ipS = ipen(HP(), tsb, tsP);
    }
    {
      // FP64 adjoint: the FP64 checkpoint; FP32 adjoint: the FP32 anchors
      double thc = 0, omc = 0, stc = 0, ctc = 1, pyc = 0, vyc = 0;
      TP thA = TP(0), omA = TP(0), pyA = TP(0), vyA = TP(0);
      if constexpr (F32) {
        thA = ck.get_f(i, 0); omA = ck.get_f(i, 1);
        if (FOOT) { pyA = ck.get_f(i, 2); vyA = ck.get_f(i, 3); }
      } else {
        thc = ck.th[i]; omc = ck.om[i]; stc = ck.s[i]; ctc = ck.c[i];
        if (FOOT) { pyc = ck.py[i]; vyc = ck.vy[i]; }
      }
      TP kthA = TP(0), komA = TP(0), kpyA = TP(0), kvyA = TP(0);
      double kth = 0, kom = 0, kpy = 0, kvy = 0;
      // FP32 adjoint: sin/cos of the anchor once per substep, the stages by angle addition
      float sA = 0.0f, cA = 1.0f;
      if constexpr (F32) sincos_f32_far(thA, &sA, &cA);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double wj = rk_w(j);
        const double cjd = (j == 0) ? 0.0 : (j == 3 ? h : h2);
        const double tj = (j == 0) ? tsb : (j == 3 ? teb : tmb);
        const TP cjh = cjhP[j];
        // FP64 stage state (FP64 adjoint only)
        double cs = ctc, sn = stc, P = 0, Q = 0, T = 0, ws = omc, wdot = 0, pys = pyc, vs = vyc;
        if (!F32) {
          const double dth = cjd * kth;
          ws = (j == 0) ? omc : fma(cjd, kom, omc);
          if (j > 0) sincos_step(thc, stc, ctc, dth, amask, sn, cs);
          P = fma(tj, dP, PL); Q = fma(tj, dQ, QL); T = fma(tj, dT, TL);
          wdot = fma(cs, P, fma(-sn, Q, T));
          kth = sd * ws; kom = sd * wdot;
          if (FOOT) {
            pys = (j == 0) ? pyc : fma(cjd, kpy, pyc);
            vs = (j == 0) ? vyc : fma(cjd, kvy, vyc);
            kpy = sd * vs; kvy = sd * (fma(tj, dAy, AyL) - g);
            const double ry = fma(sn, crx, cs * cry);
            const IP& ipj = (j == 0) ? ipS : (j == 3 ? ipE : ipM);
            const double Om = ipj.H + huber_value(-(pys + ry));
            // fused: taken by the discretization; Eq. (12) model: by the forward sweep
            if constexpr (!FUSED && !PEN_FWD) Yom = fma(h * wj, Om, Yom);
            om_pen[j] = TP(Om);
            dl0[j] = ipj.d0; dl1[j] = ipj.d1; dl2[j] = ipj.d2;
          }
        }
        TP csP, snP, PP, QP, TT, wsP, pysP = TP(0), vsP = TP(0);
        if constexpr (F32) {
          const TP tP = (j == 0) ? tsP : (j == 3 ? teP : tmP);
          wsP = (j == 0) ? omA : omA + cjh * komA;
          if (j == 0) { snP = sA; csP = cA; }
          else sincos_f32_step(thA, sA, cA, cjh * kthA, snP, csP);
          PP = PLP + tP * dPP; QP = QLP + tP * dQP; TT = TLP + tP * dTP;
          tau[j] = tP;
          if (FOOT) {
            pysP = (j == 0) ? pyA : pyA + cjh * kpyA;
            vsP = (j == 0) ? vyA : vyA + cjh * kvyA;
          }
        } else {
          csP = cs; snP = sn; PP = P; QP = Q; TT = T; wsP = ws; pysP = pys; vsP = vs;
          tau[j] = tj;
        }
        const TP wdP = csP * PP - snP * QP + TT;
        cs_[j] = csP; sn_[j] = snP;
        sath[j] = -sdP * (snP * PP + csP * QP);
        oms[j] = wsP; wdt[j] = wdP;
        if constexpr (F32) { kthA = sdP * wsP; komA = sdP * wdP; }
        if (FOOT) {
          const TP ayP = AyLP + tau[j] * dAyP - gP;
          if constexpr (F32) { kpyA = sdP * vsP; kvyA = sdP * ayP; }
          const TP rxP = csP * crxP - snP * cryP, ryP = snP * crxP + csP * cryP;
          const TP D4 = huber_slope(-(pysP + ryP));
          gp[j] = -sdP * D4;
          gr[j] = -sdP * D4 * rxP;
          vys[j] = vsP; ays[j] = ayP;
          if constexpr (F32) {
            const IP& ipj = (j == 0) ? ipS : (j == 3 ? ipE : ipM);
            if constexpr (cross) om_pen[j] = TP(ipj.H) + huber_value(-(pysP + ryP));
            else om_pen[j] = ipj.Hp + huber_value(-(pysP + ryP));
            dl0[j] = ipj.d0; dl1[j] = ipj.d1; dl2[j] = ipj.d2;
          }
          if constexpr (cross) {
            const IP& ipj = (j == 0) ? ipS : (j == 3 ? ipE : ipM);
            lsth[j] = -sdP * wsP * rxP;  // s d(lambda^c integrand)/d theta
            lsom[j] = -sdP * ryP;        // s d(...)/d omega
            axs[j] = AxLP + tau[j] * dAxP;
            q0[j] = ipj.q0; q2[j] = ipj.q2; r0[j] = ipj.r0; r1[j] = ipj.r1;
          }
        }
      }
    }
    if (FOOT) ipE = ipS;
    // transposed stages j = 3..0
    TP mth = TP(0), mom = TP(0), mpy = TP(0), mvy = TP(0), mvx = TP(0);  // mu_{j+1}
    TP sth_ = TP(0), som = TP(0), spy = TP(0), svy = TP(0), svx = TP(0);  // sum of mu_j
#pragma unroll
    for (int j = 3; j >= 0; --j) {
      const TP hw = hP * TP(rk_w(j));
      const TP cnext = (j == 3) ? TP(0) : TP(rk_c(j + 1)) * hP;
      const TP gth = hw * lth + cnext * mth;   // dL/dk_j (theta)
      const TP gom = hw * lom + cnext * mom;   // dL/dk_j (omega)
      TP nth = sath[j] * gom;                  // J_j^T: theta <- s a_theta g_omega
      TP nom = sdP * gth;                      // omega <- s g_theta
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
        if constexpr (cross) {
          // lambda^c: sources on the stage theta, omega, v_x; its input part
          // G (phi_t, gamma) and rho^c's R (phi_t, phi_n) by their slopes
          const TP inl = hw * wlP, inr = hw * wrP;
          nth += inl * lsth[j];
          nom += inl * lsom[j];
          const TP gvx = hw * lvx + cnext * mvx;  // dL/dk_j (v_x)
          const TP nvx = inl * sdP;
          gsd += gvx * axs[j];
          gAxLc += gvx * sdP * wl; gAxRc += gvx * sdP * wr;
          const TP e0 = inl * q0[j] + inr * r0[j], e1 = inr * r1[j], e2 = inl * q2[j];
          gd[0] += e0 * wl; gd[3] += e0 * wr;
          gd[1] += e1 * wl; gd[4] += e1 * wr;
          gd[2] += e2 * wl; gd[5] += e2 * wr;
          mvx = nvx; svx += nvx;
        }
      }
      mth = nth; mom = nom; sth_ += nth; som += nom;
    }
    lth += sth_; lom += som;
    if (FOOT) { lpy += spy; lvy += svy; }
    if constexpr (cross) lvx += svx;
  }

  // L share: w . defect over this link's rows (+ rho . penalty)
  double Lp = wpx * (px1 - xk1[rpx]) + wpy * (py1 - xk1[rpy]) + wth * (th - xk1[rth]) +
              wvx * (vx1 - xk1[rvx]) + wvy * (vy1 - xk1[rvy]) + wom * (om - xk1[rom]);
  if (FOOT) {
    const double pen = sd * Yom;
    Lp += wy * (xk[ry_] + pen - xk1[ry_]) + rho_c * pen;
  }
  // Eq. (12) model: the contact's rows x_k + s (mean phi_n, Il + Ig, mean gamma, Ir)
  double fn_m = 0.0, ga_m = 0.0;
  if constexpr (cross) {
    fn_m = fma(0.5, cD[1], cL[1]);
    ga_m = fma(0.5, cD[2], cL[2]);
    const double inc[4] = {fn_m, Il + Ig, ga_m, Ir};
#pragma unroll
    for (int t = 0; t < 4; ++t) Lp += wc[t] * (fma(sd, inc[t], xk[yb + t]) - xk1[yb + t]);
  }

  // ---- translation: transposed closed forms ----
  const double s2_3 = sd * sd * (1.0 / 3.0), s2_6 = sd * sd * (1.0 / 6.0), s_2 = 0.5 * sd;
  const double gAxL = wpx * s2_3 + wvx * s_2 + widen(gAxLc), gAxR = wpx * s2_6 + wvx * s_2 + widen(gAxRc);
  const double gAyLt = wpy * s2_3 + wvy * s_2 + widen(gAyL), gAyRt = wpy * s2_6 + wvy * s_2 + widen(gAyR);
  double gsd_t = wpx * (vx0 + 2.0 * sd * ax3) + wvx * axm + wpy * (vy0 + 2.0 * sd * ay3) +
                 wvy * aym + widen(gsd);
  // Eq. (12) model: the explicit factor s of the contact's rows
  if constexpr (cross) gsd_t += wc[0] * fn_m + wc[1] * (Il + Ig) + wc[2] * ga_m + wc[3] * Ir;

  // node-state gradient of this link's rows: own part minus w_{k-1} (defect_{k-1} subtracts x~_k)
  const double own[6] = {wpx, wpy + widen(lpy), widen(lth), wpx * sd + wvx + widen(lvx),
                         wpy * sd + wvy + widen(lvy), widen(lom)};
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
  if constexpr (cross) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      gXk[yb + t] = wc[t] - (wkm1 ? wkm1[yb + t] : 0.0);
      if (gXN) gXN[yb + t] = -wc[t];
    }
  }
  // per-input partials of this link
  double* pp = part + 2 * B.slot0;
  for (int i = 0; i < nin; ++i) {
    double gl = B.ax[i] * gAxL + B.ay[i] * gAyLt + B.p[i] * widen(gPL) + B.q[i] * widen(gQL) +
                B.t[i] * widen(gTL);
    double gr_ = B.ax[i] * gAxR + B.ay[i] * gAyRt + B.p[i] * widen(gPR) + B.q[i] * widen(gQR) +
                 B.t[i] * widen(gTR);
    if (FOOT) {
      const int d = B.idx[i] - cin;
      if (d >= 0 && d < 3) { gl += widen(gd[d]); gr_ += widen(gd[3 + d]); }
      if (cross && (d == 1 || d == 2)) {  // the means of phi_n and gamma: weight s/2 at each end
        const double e = s_2 * wc[d == 1 ? 0 : 2];
        gl += e;
        gr_ += e;
      }
    }
    pp[2 * i] = gl;
    pp[2 * i + 1] = gr_;
  }
  ps[b] = gsd_t;
  pL[b] = Lp;
  if (!finite_d(Lp + gsd_t + widen(lth) + widen(lom))) atomicOr(status, ST_NONFINITE);
}

}  // namespace ciscvx
