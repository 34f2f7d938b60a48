// disc_link.cuh — one link of one interval of the linearized discretization
// (Sec. IV-B Eqs. (14)-(15), Eq. (17b); IND + FOH, Sec. VI), shared by the
// single-instance and the batched kernels.  See common.cuh for the structure
// it exploits and disc.cu for the thread mapping.
//
// FP64 work is what bounds these kernels on this GPU, so the state side avoids
// every FP64 instruction it can:
//  * sin/cos of the stage angles are chained by angle addition from the
//    substep start (rotate_small), with sincos only for large increments;
//  * the four penalty terms that depend on the inputs alone are evaluated once
//    per distinct stage time (two per substep: the midpoint serves stages 2
//    and 3, the end point serves stage 4 and the next substep's stage 1);
//  * derivatives of the penalty terms are evaluated in the tangent precision;
//  * in FP32-Phi mode the tangent recursion takes its stage data from an FP32
//    copy of the stage recursion that is re-anchored on the FP64 state at the
//    start of every substep; the anchors are narrowed on the integer pipe
//    (to_f32_rz), so no conversion instruction takes an FP64-pipe slot;
//  * with checkpoints (CK) in FP32-Phi mode those anchors are the checkpoints,
//    so the FP32 adjoint's backward sweep issues no FP64 instruction per
//    substep.
// CROSS (a foot link of the Eq. (12) model): the contact's four
// cross-complementarity states and its path-penalty state.  The lambda^c row
// integrates v_x - omega (R rho)_y + gamma phi_t / sqrt(1 + phi_t^2) over the
// stages; its tangents reuse the rotation tangents and the v_y channel's
// unit-forcing tangents (v_x obeys the same equation), plus the tangent of
// v_x with respect to s.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "state_df.cuh"

namespace ciscvx {

template <typename TP>
struct Tangents {
  TP Pt[9], Pw[9];         // rotation tangents: theta row, omega row
  TP Qp[5], Qv[5];         // foot p_y/v_y tangents: columns py0, vy0, s, L, R
  TP Yr[9], Yp[5], Yd[6];  // foot penalty row: rotation columns, p_y columns, direct contact inputs
  // Eq. (12) model (CROSS) only:
  TP Yl[9];                // lambda^c row: rotation columns
  TP Ylv[3];               // lambda^c row: v_x channel columns u_L forcing, u_R forcing, s
  TP Vxs;                  // tangent of v_x with respect to s (substep start)
  TP Yld[4], Yrd[4];       // direct terms: lambda^c row (phi_t L/R, gamma L/R), rho^c row (phi_t L/R, phi_n L/R)
};

// Penalty terms that depend on the inputs alone, at one stage time.
template <typename TP>
struct InputPenalty {
  double H;       // sum of the four h(g) values (FP64; 0 unless requested)
  TP Hp;          // the same sum in the tangent precision (adjoint weights)
  TP d0, d1, d2;  // s * dOmega/d(lambda_n, lambda_t+, lambda_t-) (tangent precision)
};

// H64: evaluate the FP64 values (the penalty state); the tangent-precision
// slopes (and values, for FP32) are always evaluated.
template <typename TP, bool H64 = true>
__device__ __forceinline__ InputPenalty<TP> input_penalty(double t, TP tP, double sd, TP sdP,
                                                          double mu, TP muP, const double* L,
                                                          const double* D, const TP* LP,
                                                          const TP* DP) {
  InputPenalty<TP> r;
  r.H = 0.0;
  if (H64) {
    const double ln = fma(t, D[0], L[0]), ltp = fma(t, D[1], L[1]), ltm = fma(t, D[2], L[2]);
    r.H = huber_value(-ln) + huber_value(-ltp) + huber_value(-ltm) +
          huber_value(ltp + ltm - mu * ln);
  }
  const TP lnP = LP[0] + tP * DP[0], ltpP = LP[1] + tP * DP[1], ltmP = LP[2] + tP * DP[2];
  if constexpr (std::is_same<TP, float>::value)
    r.Hp = huber_value(-lnP) + huber_value(-ltpP) + huber_value(-ltmP) +
           huber_value(ltpP + ltmP - muP * lnP);
  else
    r.Hp = TP(r.H);
  const TP D1 = huber_slope(-lnP), D2 = huber_slope(-ltpP), D3 = huber_slope(-ltmP);
  const TP D5 = huber_slope(ltpP + ltmP - muP * lnP);
  r.d0 = sdP * (-D1 - muP * D5);
  r.d1 = sdP * (-D2 + D5);
  r.d2 = sdP * (-D3 + D5);
  (void)sd;
  return r;
}

// The input-only terms of the Eq. (12) auxiliary state at one stage time, for
// contact inputs (phi_t, phi_n, gamma) = L + t D:
//   H   = h(-phi_n) + h(-gamma) + h(-rho^c)   (path penalty, input-only part)
//   R   = rho^c = |mu phi_n|~ - |phi_t|~      (rho^c state)
//   G   = gamma phi_t / sqrt(1 + phi_t^2)      (input part of lambda^c)
// FP64 values and s-scaled slopes in the tangent precision.
template <typename TP>
struct InputCross {
  double H, R, G;
  TP d0, d1, d2;  // s dH/d(phi_t, phi_n, gamma)
  TP r0, r1;      // s dR/d(phi_t, phi_n)
  TP q0, q2;      // s dG/d(phi_t, gamma)
};

// pseudo-Huber absolute value sqrt(1 + x^2) - 1 (as a rsqrt(a) - 1, a = 1 + x^2)
__device__ __forceinline__ double sabs_value(double x) {
  const double a = fma(x, x, 1.0);
  return fma(a, rsqrt(a), -1.0);
}

template <typename TP>
__device__ __forceinline__ InputCross<TP> input_cross(double t, TP tP, TP sdP, double mu, TP muP,
                                                      const double* L, const double* D,
                                                      const TP* LP, const TP* DP) {
  InputCross<TP> r;
  const double ft = fma(t, D[0], L[0]), fn = fma(t, D[1], L[1]), ga = fma(t, D[2], L[2]);
  const double at = fma(ft, ft, 1.0), rt = rsqrt(at);
  r.R = sabs_value(mu * fn) - fma(at, rt, -1.0);
  r.H = huber_value(-fn) + huber_value(-ga) + huber_value(-r.R);
  r.G = ga * (ft * rt);
  const TP ftP = LP[0] + tP * DP[0], fnP = LP[1] + tP * DP[1], gaP = LP[2] + tP * DP[2];
  const TP rtP = TP(1) / sqrt(TP(1) + ftP * ftP);
  const TP mfn = muP * fnP;
  const TP dmn = mfn / sqrt(TP(1) + mfn * mfn);  // d|x|~/dx at mu phi_n
  const TP dft = ftP * rtP;                      // d|x|~/dx at phi_t (= phi_t / sqrt(1 + phi_t^2))
  const TP RP = (sqrt(TP(1) + mfn * mfn) - TP(1)) - (sqrt(TP(1) + ftP * ftP) - TP(1));
  const TP hR = huber_slope(-RP);
  r.r0 = -sdP * dft;
  r.r1 = sdP * muP * dmn;
  r.d0 = -hR * r.r0;
  r.d1 = -sdP * huber_slope(-fnP) - hR * r.r1;
  r.d2 = -sdP * huber_slope(-gaP);
  r.q0 = sdP * gaP * rtP * rtP * rtP;
  r.q2 = sdP * dft;
  return r;
}

// Stage data of one substep for the tangent recursion (tangent precision).
template <typename TP>
struct StageT {
  TP cw[4], sw[4], sath[4], oms[4], wdt[4], tau[4];
  TP gr[4], gp[4], vys[4], ays[4], dl0[4], dl1[4], dl2[4];
  TP lry[4], lrx[4], axs[4], cq0[4], cq2[4], cr0[4], cr1[4];  // Eq. (12) model
};

// One substep of the tangent recursion (IND, Sec. VI) of one link from its
// stage data: the nine rotation columns, the foot's p_y channel and penalty
// row, and (CROSS) the lambda^c row.
template <typename TP, bool FOOT, bool CROSS>
__device__ __forceinline__ void tangent_substep(Tangents<TP>& tg, const StageT<TP>& st, TP sdP, TP hP,
                                                const TP* cjhP) {
  constexpr bool foot = FOOT;
  constexpr bool cross = FOOT && CROSS;
  // ---- rotation tangents: 9 columns, 4 stages each ----
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const TP T0 = tg.Pt[c], W0 = tg.Pw[c];
    TP kT = TP(0), kW = TP(0), aT = TP(0), aW = TP(0), ya = TP(0), yl = TP(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const TP cjh = cjhP[j], wj = TP(rk_w(j));
      const TP Ts = (j == 0) ? T0 : T0 + cjh * kT;
      const TP Ws = (j == 0) ? W0 : W0 + cjh * kW;
      const TP wl = TP(1) - st.tau[j], wr = st.tau[j];
      TP fT = TP(0), fW = TP(0);
      if (c == 2) { fT = st.oms[j]; fW = st.wdt[j]; }
      else if (c == 3) fW = sdP * st.cw[j] * wl;
      else if (c == 4) fW = -sdP * st.sw[j] * wl;
      else if (c == 5) fW = sdP * wl;
      else if (c == 6) fW = sdP * st.cw[j] * wr;
      else if (c == 7) fW = -sdP * st.sw[j] * wr;
      else if (c == 8) fW = sdP * wr;
      kT = sdP * Ws + fT;
      kW = st.sath[j] * Ts + fW;
      aT += wj * kT;
      aW += wj * kW;
      if (foot) ya += wj * st.gr[j] * Ts;
      if constexpr (cross) yl += wj * (st.lry[j] * Ws + st.lrx[j] * Ts);
    }
    tg.Pt[c] = T0 + hP * aT;
    tg.Pw[c] = W0 + hP * aW;
    if (foot) tg.Yr[c] += hP * ya;
    if constexpr (cross) tg.Yl[c] += hP * yl;
  }

  // ---- foot: p_y channel tangents and the penalty row ----
  if (foot) {
    TP y0 = TP(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) y0 += TP(rk_w(j)) * st.gp[j];
    tg.Yp[0] += hP * y0;  // p_y0 column: stage tangent of p_y is 1
#pragma unroll
    for (int c = 1; c < 5; ++c) {
      const TP P0 = tg.Qp[c], V0 = tg.Qv[c];
      TP kP = TP(0), kV = TP(0), aP = TP(0), aV = TP(0), ya = TP(0), yv = TP(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const TP cjh = cjhP[j], wj = TP(rk_w(j));
        const TP Ps = (j == 0) ? P0 : P0 + cjh * kP;
        const TP Vs = (j == 0) ? V0 : V0 + cjh * kV;
        TP fP = TP(0), fV = TP(0);
        if (c == 2) { fP = st.vys[j]; fV = st.ays[j]; }
        else if (c == 3) fV = sdP * (TP(1) - st.tau[j]);
        else if (c == 4) fV = sdP * st.tau[j];
        kP = sdP * Vs + fP;
        kV = fV;
        aP += wj * kP;
        aV += wj * kV;
        ya += wj * st.gp[j] * Ps;
        // unit-forcing tangents of v_y equal those of v_x (same equation v' = s a)
        if constexpr (cross) yv += wj * sdP * Vs;
      }
      tg.Qp[c] = P0 + hP * aP;
      tg.Qv[c] = V0 + hP * aV;
      tg.Yp[c] += hP * ya;
      if constexpr (cross) {
        if (c >= 3) tg.Ylv[c - 3] += hP * yv;
      }
    }
    if constexpr (cross) {
      // v_x tangent with respect to s (forcing a_x(tau)); lambda^c's s column
      const TP V0 = tg.Vxs;
      TP kV = TP(0), aV = TP(0), yv = TP(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const TP wj = TP(rk_w(j));
        const TP Vs = (j == 0) ? V0 : V0 + cjhP[j] * kV;
        kV = st.axs[j];
        aV += wj * kV;
        yv += wj * sdP * Vs;
      }
      tg.Vxs = V0 + hP * aV;
      tg.Ylv[2] += hP * yv;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const TP hw = hP * TP(rk_w(j));
      const TP wl = TP(1) - st.tau[j], wr = st.tau[j];
      tg.Yd[0] += hw * st.dl0[j] * wl; tg.Yd[3] += hw * st.dl0[j] * wr;
      tg.Yd[1] += hw * st.dl1[j] * wl; tg.Yd[4] += hw * st.dl1[j] * wr;
      tg.Yd[2] += hw * st.dl2[j] * wl; tg.Yd[5] += hw * st.dl2[j] * wr;
      if constexpr (cross) {
        tg.Yld[0] += hw * st.cq0[j] * wl; tg.Yld[1] += hw * st.cq0[j] * wr;
        tg.Yld[2] += hw * st.cq2[j] * wl; tg.Yld[3] += hw * st.cq2[j] * wr;
        tg.Yrd[0] += hw * st.cr0[j] * wl; tg.Yrd[1] += hw * st.cr0[j] * wr;
        tg.Yrd[2] += hw * st.cr1[j] * wl; tg.Yrd[3] += hw * st.cr1[j] * wr;
      }
    }
  }
}

// One link of one interval.  xk/xk1: node states k and k+1; uL/uR: FOH
// controls; A/Bm/Bp/S/defect/pen/z: this interval's output blocks.
// CMP: A, Bm, Bp point at this interval's compact values (structural
// nonzeros only, at the link's offsets; see common.cuh) instead of its dense
// blocks.  CK: also record the FP64 state at every substep start (and the end
// state and penalty quadrature) in *ck, for the adjoint's backward sweep.
template <typename TP, bool FOOT, bool CMP = false, bool CK = false, bool CROSS = false>
__device__ __forceinline__ void disc_link(const DevModel& M, int b, int nsub, double sd,
                                          const double* __restrict__ xk,
                                          const double* __restrict__ xk1,
                                          const double* __restrict__ uL,
                                          const double* __restrict__ uR, TP* __restrict__ A,
                                          TP* __restrict__ Bm, TP* __restrict__ Bp,
                                          TP* __restrict__ S, double* __restrict__ defect,
                                          double* __restrict__ pen, double* __restrict__ z,
                                          unsigned* status, Checkpoints* ck = nullptr) {
  constexpr bool F32 = std::is_same<TP, float>::value;
  // CROSS: the link carries a contact of the Eq. (12) model (see the header
  // comment of input_cross); the kernels form no z for it (callers form it
  // from the stored outputs).  Its checkpoints add the quadratures Il, Ir,
  // Ig of the contact's rows.
  constexpr bool cross = FOOT && CROSS;
  const unsigned amask = __activemask();  // lanes running this link (they stay converged)
  const DevBody& B = M.body[b];
  const int nb = M.nb, nxt = M.nxt, nu = M.nu;
  const double g = M.g;
  const int nin = B.nin;

  // Input sums at the interval ends (the forces/torques are linear in u).
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

  // Translation in closed form (exact for RK4: polynomial of degree <= 3 in tau).
  // (explicit fma: the same rounding in every instantiation of this function)
  const double axm = 0.5 * (AxL + AxR), ax3 = fma(AxL, 1.0 / 3.0, AxR * (1.0 / 6.0));
  const double aym = fma(0.5, AyL + AyR, -g), ay3 = fma(AyL, 1.0 / 3.0, fma(AyR, 1.0 / 6.0, -0.5 * g));
  const double sd2 = sd * sd;
  const double px1 = fma(sd2, ax3, fma(sd, vx0, px0)), vx1 = fma(sd, axm, vx0);
  const double py1 = fma(sd2, ay3, fma(sd, vy0, py0)), vy1 = fma(sd, aym, vy0);

  constexpr bool foot = FOOT;  // B.contact >= 0; warp-uniform, dispatched by the kernel
  const int cin = B.cin;
  double cL[3] = {0, 0, 0}, cD[3] = {0, 0, 0};  // contact inputs at tau = 0 and their increments
  TP cLP[3], cDP[3];
  if (foot) {
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
  const double dP = PR - PL, dQ = QR - QL, dT = TR - TL, dAy = AyR - AyL;
  // tangent-precision copies of the input sums (FP32: narrowed on the integer
  // pipe, like every FP32 copy of a per-interval constant below)
  const TP PLP = anchor<TP>(PL), dPP = anchor<TP>(dP), QLP = anchor<TP>(QL), dQP = anchor<TP>(dQ),
           TLP = anchor<TP>(TL), dTP = anchor<TP>(dT);
  const TP AyLP = anchor<TP>(AyL), dAyP = anchor<TP>(dAy), gP = anchor<TP>(g);

  Tangents<TP> tg;
#pragma unroll
  for (int c = 0; c < 9; ++c) { tg.Pt[c] = TP(0); tg.Pw[c] = TP(0); tg.Yr[c] = TP(0); }
#pragma unroll
  for (int c = 0; c < 5; ++c) { tg.Qp[c] = TP(0); tg.Qv[c] = TP(0); tg.Yp[c] = TP(0); }
#pragma unroll
  for (int c = 0; c < 6; ++c) tg.Yd[c] = TP(0);
  tg.Pt[0] = TP(1); tg.Pw[1] = TP(1);
  tg.Qp[0] = TP(1); tg.Qv[1] = TP(1);
  if constexpr (cross) {
#pragma unroll
    for (int c = 0; c < 9; ++c) tg.Yl[c] = TP(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) { tg.Yld[c] = TP(0); tg.Yrd[c] = TP(0); }
    tg.Ylv[0] = tg.Ylv[1] = tg.Ylv[2] = TP(0);
    tg.Vxs = TP(0);
  }
  // Eq. (12) model: x-velocity stages for lambda^c (s-scaled slopes, as for v_y)
  const double dAx = AxR - AxL, sAxL = sd * AxL, sdAxs = sd * dAx;
  const TP AxLP = anchor<TP>(AxL), dAxP = anchor<TP>(dAx);
  double vx = vx0, Il = 0.0, Ir = 0.0, Ig = 0.0;  // lambda^c state part, rho^c, gamma g integrals

  const double h = 1.0 / nsub, h2 = 0.5 * h;
  if constexpr (CK) {  // the backward sweep of the fused pass takes these over
    ck->h = h;
    ck->ins[0] = AxL; ck->ins[1] = AxR; ck->ins[2] = AyL; ck->ins[3] = AyR; ck->ins[4] = PL;
    ck->ins[5] = PR; ck->ins[6] = QL; ck->ins[7] = QR; ck->ins[8] = TL; ck->ins[9] = TR;
  }
  const TP hP = anchor<TP>(h), sdP = anchor<TP>(sd), h2P = anchor<TP>(h2);
  const TP cjhP[4] = {TP(0), h2P, h2P, hP};
  double th = th0, om = om0, py = py0, vy = vy0, Yom = 0.0;
  double ti = 0.0;  // tau at the substep start (running sum; rounding ~1e-16 per step)
  TP tiP = TP(0);
  double sth, cth;  // sin/cos of th at the substep start (chained)
  sincos(th, &sth, &cth);
  InputPenalty<TP> ip0;  // input penalty at the substep start
  InputCross<TP> ic0;    // Eq. (12) model: input-only terms at the substep start
  if constexpr (cross) ic0 = input_cross<TP>(0.0, TP(0), sdP, mu, muP, cL, cD, cLP, cDP);
  else if (foot) ip0 = input_penalty<TP>(0.0, TP(0), sd, sdP, mu, muP, cL, cD, cLP, cDP);
  // Penalty quadrature: the input-only terms H(tau) enter every substep as
  // Simpson's rule (h/6 H(t_i) + 2h/3 H(t_i + h/2) + h/6 H(t_i + h)); they are
  // accumulated as 2h/3 H(mid) + h/3 H(end) per substep, with h/6 H(0) added
  // first and h/6 H(1) taken off at the end.
  const double h3 = h * (1.0 / 3.0), h23 = 2.0 * h3, h6 = 0.5 * h3;
  if constexpr (cross) {
    Yom = h6 * ic0.H;
    Ir = h6 * ic0.R;
    Ig = h6 * ic0.G;
  } else if (foot) {
    Yom = h6 * ip0.H;
  }
  // FP32-Phi mode: the FP64 state needs only the s-scaled stage slopes
  // k_theta = s omega_stage and k_omega = s (cos P - sin Q + T), so the input
  // sums are pre-scaled by s (one FMA per slope instead of an FMA and a
  // multiply) and s P, s Q, s T at the substep end carry over to the next start.
  const double sPL = sd * PL, sdPs = sd * dP, sQL = sd * QL, sdQs = sd * dQ;
  const double sTL = sd * TL, sdTs = sd * dT;
  const double sAyg = sd * (AyL - g), sdAys = sd * dAy;
  const double sc2 = sd * h2, sc3 = sd * h;
  double sPi = sPL, sQi = sQL, sTi = sTL;

  // FP32-Phi mode of the default model: stage values in float-float on the
  // FP32 pipe, the state accumulated in FP64 (state_df.cuh); the tangent
  // recursion takes its FP32 stage data from the same pass.
  constexpr bool DF = F32 && !CROSS;
  if constexpr (DF) {
    const DfLink C = df_link(sd, nsub, PL, dP, QL, dQ, TL, dT, AyL, dAy, g, foot, crx, cry, mu, cL, cD);
    DfState S = df_state_init<FOOT>(C, th0, om0, py0, vy0);
    InputPenalty<TP> ipA, ipB;  // FP32 slopes of the input-only terms at the substep start / end
    if (foot) ipA = input_penalty<TP, false>(0.0, TP(0), sd, sdP, mu, muP, cL, cD, cLP, cDP);
    for (int i = 0; i < nsub; ++i) {
      if constexpr (CK) {  // FP32 anchors at the substep start: the backward sweep's checkpoints
        ck->put_f(i, 0, anchor<TP>(S.th)); ck->put_f(i, 1, anchor<TP>(S.om));
        if (foot) { ck->put_f(i, 2, anchor<TP>(S.py)); ck->put_f(i, 3, anchor<TP>(S.vy)); }
      }
      StageF sf[4];
      df_substep<FOOT, true>(C, i, amask, S, sf);
      StageT<TP> st;
      InputPenalty<TP> ipM;
      if (foot) {
        ipM = input_penalty<TP, false>(0.0, TP(sf[1].tau), sd, sdP, mu, muP, cL, cD, cLP, cDP);
        ipB = input_penalty<TP, false>(0.0, TP(sf[3].tau), sd, sdP, mu, muP, cL, cD, cLP, cDP);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const TP tP = sf[j].tau, csP = sf[j].cs, snP = sf[j].sn;
        const TP PP = PLP + tP * dPP, QP = QLP + tP * dQP, TT = TLP + tP * dTP;
        st.cw[j] = csP;
        st.sw[j] = snP;
        st.sath[j] = -sdP * (snP * PP + csP * QP);  // s * d(omega')/d(theta)
        st.oms[j] = sf[j].ws;
        st.wdt[j] = csP * PP - snP * QP + TT;
        st.tau[j] = tP;
        if (foot) {
          const TP rxP = csP * crxP - snP * cryP, ryP = snP * crxP + csP * cryP;
          const TP D4 = huber_slope(-(TP(sf[j].pys) + ryP));
          st.gp[j] = -sdP * D4;        // s dOmega/dp_y
          st.gr[j] = -sdP * D4 * rxP;  // s dOmega/dtheta
          st.vys[j] = sf[j].vys;
          st.ays[j] = AyLP + tP * dAyP - gP;
          const InputPenalty<TP>& ipj = (j == 0) ? ipA : (j == 3 ? ipB : ipM);
          st.dl0[j] = ipj.d0; st.dl1[j] = ipj.d1; st.dl2[j] = ipj.d2;
        }
      }
      tangent_substep<TP, FOOT, false>(tg, st, sdP, hP, cjhP);
      if (foot) ipA = ipB;
    }
    df_state_finish<FOOT>(C, S);
    th = S.th;
    om = S.om;
    Yom = S.Y;
  } else {
    for (int i = 0; i < nsub; ++i) {
      if constexpr (CK && !F32) {
        ck->th[i] = th; ck->om[i] = om; ck->s[i] = sth; ck->c[i] = cth;
        if (foot) { ck->py[i] = py; ck->vy[i] = vy; }
      }
      // ---- state stages (FP64) ----
      StageT<TP> st;
      TP (&cw)[4] = st.cw, (&sw)[4] = st.sw, (&sath)[4] = st.sath, (&oms)[4] = st.oms;
      TP (&wdt)[4] = st.wdt, (&tau)[4] = st.tau, (&gr)[4] = st.gr, (&gp)[4] = st.gp;
      TP (&vys)[4] = st.vys, (&ays)[4] = st.ays, (&dl0)[4] = st.dl0, (&dl1)[4] = st.dl1, (&dl2)[4] = st.dl2;
      TP (&lry)[4] = st.lry, (&lrx)[4] = st.lrx, (&axs)[4] = st.axs, (&cq0)[4] = st.cq0;
      TP (&cq2)[4] = st.cq2, (&cr0)[4] = st.cr0, (&cr1)[4] = st.cr1;
      TP vxP[4];  // Eq. (12) model
      const double tm = ti + h2, te = ti + h;
      const TP tmP = tiP + h2P, teP = tiP + hP;
      InputPenalty<TP> ipm, ip1;
      InputCross<TP> icm, ic1;
      if constexpr (cross) {
        icm = input_cross<TP>(tm, tmP, sdP, mu, muP, cL, cD, cLP, cDP);
        ic1 = input_cross<TP>(te, teP, sdP, mu, muP, cL, cD, cLP, cDP);
      } else if (foot) {
        ipm = input_penalty<TP>(tm, tmP, sd, sdP, mu, muP, cL, cD, cLP, cDP);
        ip1 = input_penalty<TP>(te, teP, sd, sdP, mu, muP, cL, cD, cLP, cDP);
      }
      // FP32 copy of the stage recursion, anchored on the FP64 state (FP32-Phi
      // mode; the anchors are narrowed on the integer pipe).  With CK the
      // anchors are the checkpoints: the FP32 backward sweep starts from them.
      const TP thA = anchor<TP>(th), omA = anchor<TP>(om), pyA = anchor<TP>(py), vyA = anchor<TP>(vy);
      const TP vxA = cross ? anchor<TP>(vx) : TP(0);
      if constexpr (CK && F32) {
        ck->put_f(i, 0, thA); ck->put_f(i, 1, omA);
        if (foot) { ck->put_f(i, 2, pyA); ck->put_f(i, 3, vyA); }
      }
      TP kthA = TP(0), komA = TP(0), kpyA = TP(0), kvyA = TP(0), kvxA = TP(0);
      double kth = 0, kom = 0, ath_ = 0, aom_ = 0, kpy = 0, kvy = 0, apy = 0, avy = 0;
      double kvx = 0, avx = 0;  // Eq. (12) model: s a_x at the stage, its RK4 sum
      const double som = sd * om, svy = foot ? sd * vy : 0.0;
      double sPm = 0, sQm = 0, sTm = 0;
      double ws = 0, P = 0, Q = 0, T = 0;  // FP64 stage data (FP64 mode only)
  #pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double wj = rk_w(j);
        const double cjh = (j == 0) ? 0.0 : (j == 3 ? h : h2);
        const double tj = (j == 0) ? ti : (j == 3 ? te : tm);
        const double dth = cjh * kth;
        double sn, cs;
        if (j == 0) { sn = sth; cs = cth; }
        else sincos_step(th, sth, cth, dth, amask, sn, cs);
        // Eq. (12) model: omega at the stage (kom is still the previous stage's slope)
        const double wst = cross ? ((j == 0) ? om : fma(cjh, kom, om)) : 0.0;
        if constexpr (F32) {
          double sP, sQ, sT;
          if (j == 0) { sP = sPi; sQ = sQi; sT = sTi; }
          else if (j == 3) {
            sPi = fma(te, sdPs, sPL); sQi = fma(te, sdQs, sQL); sTi = fma(te, sdTs, sTL);
            sP = sPi; sQ = sQi; sT = sTi;
          } else {
            if (j == 1) { sPm = fma(tm, sdPs, sPL); sQm = fma(tm, sdQs, sQL); sTm = fma(tm, sdTs, sTL); }
            sP = sPm; sQ = sQm; sT = sTm;
          }
          kth = (j == 0) ? som : fma(j == 3 ? sc3 : sc2, kom, som);
          kom = fma(cs, sP, fma(-sn, sQ, sT));
        } else {
          ws = (j == 0) ? om : fma(cjh, kom, om);
          P = fma(tj, dP, PL); Q = fma(tj, dQ, QL); T = fma(tj, dT, TL);
          kth = sd * ws;
          kom = sd * fma(cs, P, fma(-sn, Q, T));
        }
        ath_ = fma(wj, kth, ath_);
        aom_ = fma(wj, kom, aom_);
        double pys = 0.0, vs = 0.0;
        if (foot) {
          pys = (j == 0) ? py : fma(cjh, kpy, py);
          if constexpr (F32) {
            kpy = (j == 0) ? svy : fma(j == 3 ? sc3 : sc2, kvy, svy);
            kvy = fma(tj, sdAys, sAyg);
          } else {
            vs = (j == 0) ? vy : fma(cjh, kvy, vy);
            kpy = sd * vs;
            kvy = sd * (fma(tj, dAy, AyL) - g);
          }
          apy = fma(wj, kpy, apy);
          avy = fma(wj, kvy, avy);
          if constexpr (cross) {
            // ground term h(-phi); lambda^c's state part v_x - omega (R rho)_y
            const double ry = fma(sn, crx, cs * cry);
            Yom = fma(h * wj, huber_value(-(pys + ry)), Yom);
            const double vxs = (j == 0) ? vx : fma(cjh, kvx, vx);
            kvx = fma(tj, sdAxs, sAxL);
            avx = fma(wj, kvx, avx);
            Il = fma(h * wj, fma(-wst, ry, vxs), Il);
            vxP[j] = F32 ? ((j == 0) ? vxA : vxA + cjhP[j] * kvxA) : TP(vxs);
            const InputCross<TP>& icj = (j == 0) ? ic0 : (j == 3 ? ic1 : icm);
            dl0[j] = icj.d0; dl1[j] = icj.d1; dl2[j] = icj.d2;
            cq0[j] = icj.q0; cq2[j] = icj.q2; cr0[j] = icj.r0; cr1[j] = icj.r1;
          } else {
            // ground term h(-phi), phi = p_y + (R rho)_y at the stage
            Yom = fma(h * wj, huber_value(-fma(sn, crx, fma(cs, cry, pys))), Yom);
            const InputPenalty<TP>& ipj = (j == 0) ? ip0 : (j == 3 ? ip1 : ipm);
            dl0[j] = ipj.d0; dl1[j] = ipj.d1; dl2[j] = ipj.d2;
          }
        }
        // stage data for the tangent recursion
        const TP cjhT = cjhP[j];
        TP csP, snP, PP, QP, TT, wsP, pysP = TP(0), vsP = TP(0);
        if constexpr (F32) {
          const TP tP = (j == 0) ? tiP : (j == 3 ? teP : tmP);
          const TP thsP = (j == 0) ? thA : thA + cjhT * kthA;
          wsP = (j == 0) ? omA : omA + cjhT * komA;
          sincosf(thsP, &snP, &csP);
          PP = PLP + tP * dPP; QP = QLP + tP * dQP; TT = TLP + tP * dTP;
          tau[j] = tP;
          if (foot) {
            pysP = (j == 0) ? pyA : pyA + cjhT * kpyA;
            vsP = (j == 0) ? vyA : vyA + cjhT * kvyA;
          }
        } else {
          csP = cs; snP = sn; PP = P; QP = Q; TT = T; wsP = ws; pysP = pys; vsP = vs;
          tau[j] = tj;
        }
        const TP wdP = csP * PP - snP * QP + TT;
        cw[j] = csP;
        sw[j] = snP;
        sath[j] = -sdP * (snP * PP + csP * QP);  // s * d(omega')/d(theta)
        oms[j] = wsP;
        wdt[j] = wdP;
        if constexpr (F32) { kthA = sdP * wsP; komA = sdP * wdP; }
        if (foot) {
          const TP ayP = AyLP + tau[j] * dAyP - gP;
          if constexpr (F32) { kpyA = sdP * vsP; kvyA = sdP * ayP; }
          const TP rxP = csP * crxP - snP * cryP;
          const TP ryP = snP * crxP + csP * cryP;
          const TP D4 = huber_slope(-(pysP + ryP));
          gp[j] = -sdP * D4;        // s dOmega/dp_y
          gr[j] = -sdP * D4 * rxP;  // s dOmega/dtheta
          vys[j] = vsP;
          ays[j] = ayP;
          if constexpr (cross) {
            lry[j] = -sdP * ryP;        // s d(lambda^c)/d omega
            lrx[j] = -sdP * wsP * rxP;  // s d(lambda^c)/d theta
            axs[j] = AxLP + tau[j] * dAxP;
            if constexpr (F32) kvxA = sdP * axs[j];
          }
        }
      }
      const double Dth = h * ath_;
      {
        double s1, c1;
        sincos_step(th, sth, cth, Dth, amask, s1, c1);
        sth = s1;
        cth = c1;
      }
      th += Dth;
      om = fma(h, aom_, om);
      if (foot) {
        py = fma(h, apy, py);
        vy = fma(h, avy, vy);
        if constexpr (cross) {
          vx = fma(h, avx, vx);
          Yom = fma(h3, ic1.H, fma(h23, icm.H, Yom));
          Ir = fma(h3, ic1.R, fma(h23, icm.R, Ir));
          Ig = fma(h3, ic1.G, fma(h23, icm.G, Ig));
          ic0 = ic1;
        } else {
          Yom = fma(h3, ip1.H, fma(h23, ipm.H, Yom));
          ip0 = ip1;
        }
      }
      ti = te;
      tiP = teP;

      tangent_substep<TP, FOOT, CROSS>(tg, st, sdP, hP, cjhP);
    }

    // the end point was counted with h/3
    if constexpr (cross) {
      Yom = fma(-h6, ic0.H, Yom);
      Ir = fma(-h6, ic0.R, Ir);
      Ig = fma(-h6, ic0.G, Ig);
    } else if (foot) {
      Yom = fma(-h6, ip0.H, Yom);
    }
  }
  if constexpr (CK) {
    ck->th_end = th; ck->om_end = om; ck->Yom = Yom;
    if constexpr (cross) { ck->Il = Il; ck->Ir = Ir; ck->Ig = Ig; }
  }

  // ------------------------------------------------------------ outputs ---
  const TP one = TP(1);
  const TP sdT = anchor<TP>(sd), s2_3 = anchor<TP>(sd2 * (1.0 / 3.0)), s2_6 = anchor<TP>(sd2 * (1.0 / 6.0)),
           s_2 = anchor<TP>(0.5 * sd);
  // the contact's path-penalty row (after the Eq. (12) model's four cross states per contact)
  const int ry = foot ? 6 * nb + (cross ? 4 * M.nc : 0) + B.contact : -1;
  if constexpr (!CMP) {
    // Zero this link's rows of A, B-, B+ (and the contact's row) cooperatively,
    // then write the structural entries.
    warp_zero_chunks(A + (size_t)rpx * nxt, 3 * nxt, amask);
    warp_zero_chunks(A + (size_t)rvx * nxt, 3 * nxt, amask);
    if (nu > 0) {
      warp_zero_chunks(Bm + (size_t)rpx * nu, 3 * nu, amask);
      warp_zero_chunks(Bm + (size_t)rvx * nu, 3 * nu, amask);
      warp_zero_chunks(Bp + (size_t)rpx * nu, 3 * nu, amask);
      warp_zero_chunks(Bp + (size_t)rvx * nu, 3 * nu, amask);
    }
    if (foot) {
      warp_zero_chunks(A + (size_t)ry * nxt, nxt, amask);
      if (nu > 0) {
        warp_zero_chunks(Bm + (size_t)ry * nu, nu, amask);
        warp_zero_chunks(Bp + (size_t)ry * nu, nu, amask);
      }
    }
    if constexpr (cross) {  // the contact's four cross-complementarity rows
      const int yb = 6 * nb + 4 * B.contact;
      warp_zero_chunks(A + (size_t)yb * nxt, 4 * nxt, amask);
      if (nu > 0) {
        warp_zero_chunks(Bm + (size_t)yb * nu, 4 * nu, amask);
        warp_zero_chunks(Bp + (size_t)yb * nu, 4 * nu, amask);
      }
    }
    __syncwarp(amask);
  }
  // Entry (r, c) of A, the j-th compact A entry of this link (order in common.cuh).
  TP* const Ac = A + (CMP ? B.a_off : 0);
  auto a_put = [&](int r, int c, int j, TP v) {
    if constexpr (CMP) Ac[j] = v; else A[(size_t)r * nxt + c] = v;
  };
  a_put(rpx, rpx, 0, one); a_put(rpx, rvx, 1, sdT);
  a_put(rpy, rpy, 2, one); a_put(rpy, rvy, 3, sdT);
  a_put(rth, rth, 4, tg.Pt[0]); a_put(rth, rom, 5, tg.Pt[1]);
  a_put(rvx, rvx, 6, one);
  a_put(rvy, rvy, 7, one);
  a_put(rom, rth, 8, tg.Pw[0]); a_put(rom, rom, 9, tg.Pw[1]);
  // S
  const double Spx = fma(2.0 * sd, ax3, vx0), Spy = fma(2.0 * sd, ay3, vy0);
  S[rpx] = TP(Spx); S[rvx] = TP(axm);
  S[rpy] = TP(Spy); S[rvy] = TP(aym);
  S[rth] = tg.Pt[2]; S[rom] = tg.Pw[2];

  // Optional affine term z = x~(1) - A x~_k - B- u_L - B+ u_R - S s, formed from
  // the stored (rounded) block values: rows px, py, th, vx, vy, om, y.
  const bool wz = (z != nullptr);
  double zr[7];
  if (wz) {
    zr[0] = px1 - double(S[rpx]) * sd - xk[rpx] - double(sdT) * xk[rvx];
    zr[1] = py1 - double(S[rpy]) * sd - xk[rpy] - double(sdT) * xk[rvy];
    zr[2] = th - double(S[rth]) * sd - double(tg.Pt[0]) * xk[rth] - double(tg.Pt[1]) * xk[rom];
    zr[3] = vx1 - double(S[rvx]) * sd - xk[rvx];
    zr[4] = vy1 - double(S[rvy]) * sd - xk[rvy];
    zr[5] = om - double(S[rom]) * sd - double(tg.Pw[0]) * xk[rth] - double(tg.Pw[1]) * xk[rom];
  }
  // B-, B+: per input q of this link (slot order), entries in rows px (if the
  // input pushes along x), py (along y), th (if it exerts a torque), vx, vy,
  // om (torque), then y for a foot.  nzx/nzy/tq: the input has an x / y force
  // component / a torque (tested on the bit patterns).
  auto torque = [&](int i) { return (abs_bits(B.p[i]) | abs_bits(B.q[i]) | abs_bits(B.t[i])) != 0ull; };
  if (nu > 0) {
    int o = B.b_off;
    for (int i = 0; i < nin; ++i) {
      const int q = B.idx[i];
      const bool nzx = abs_bits(B.ax[i]) != 0ull, nzy = abs_bits(B.ay[i]) != 0ull, tq = torque(i);
      const TP ax = anchor<TP>(B.ax[i]), ay = anchor<TP>(B.ay[i]), pc = anchor<TP>(B.p[i]),
               qc = anchor<TP>(B.q[i]), tc = anchor<TP>(B.t[i]);
      const TP bmpx = ax * s2_3, bppx = ax * s2_6, bvx = ax * s_2;
      const TP bmpy = ay * s2_3, bppy = ay * s2_6, bvy = ay * s_2;
      const TP bmth = pc * tg.Pt[3] + qc * tg.Pt[4] + tc * tg.Pt[5];
      const TP bpth = pc * tg.Pt[6] + qc * tg.Pt[7] + tc * tg.Pt[8];
      const TP bmom = pc * tg.Pw[3] + qc * tg.Pw[4] + tc * tg.Pw[5];
      const TP bpom = pc * tg.Pw[6] + qc * tg.Pw[7] + tc * tg.Pw[8];
      if constexpr (CMP) {
        if (nzx) { Bm[o] = bmpx; Bp[o] = bppx; ++o; }
        if (nzy) { Bm[o] = bmpy; Bp[o] = bppy; ++o; }
        if (tq) { Bm[o] = bmth; Bp[o] = bpth; ++o; }
        if (nzx) { Bm[o] = bvx; Bp[o] = bvx; ++o; }
        if (nzy) { Bm[o] = bvy; Bp[o] = bvy; ++o; }
        if (tq) { Bm[o] = bmom; Bp[o] = bpom; ++o; }
        if (foot) ++o;  // the y entry, written below
      } else {
        Bm[(size_t)rpx * nu + q] = bmpx; Bp[(size_t)rpx * nu + q] = bppx;
        Bm[(size_t)rvx * nu + q] = bvx;  Bp[(size_t)rvx * nu + q] = bvx;
        Bm[(size_t)rpy * nu + q] = bmpy; Bp[(size_t)rpy * nu + q] = bppy;
        Bm[(size_t)rvy * nu + q] = bvy;  Bp[(size_t)rvy * nu + q] = bvy;
        Bm[(size_t)rth * nu + q] = bmth; Bp[(size_t)rth * nu + q] = bpth;
        Bm[(size_t)rom * nu + q] = bmom; Bp[(size_t)rom * nu + q] = bpom;
      }
      if (wz) {
        const double a = uL[q], c = uR[q];
        zr[0] -= double(bmpx) * a + double(bppx) * c;
        zr[1] -= double(bmpy) * a + double(bppy) * c;
        zr[2] -= double(bmth) * a + double(bpth) * c;
        zr[3] -= double(bvx) * a + double(bvx) * c;
        zr[4] -= double(bvy) * a + double(bvy) * c;
        zr[5] -= double(bmom) * a + double(bpom) * c;
      }
    }
  }
  // defect (Eq. (17b))
  defect[rpx] = px1 - xk1[rpx]; defect[rpy] = py1 - xk1[rpy]; defect[rth] = th - xk1[rth];
  defect[rvx] = vx1 - xk1[rvx]; defect[rvy] = vy1 - xk1[rvy]; defect[rom] = om - xk1[rom];
  double chk = px1 + py1 + th + vx1 + vy1 + om + Spx + Spy;
  TP chkP = TP(0);  // the tangent values, summed in their own precision (finite check only)
#pragma unroll
  for (int c = 0; c < 9; ++c) chkP += tg.Pt[c] + tg.Pw[c];

  double y1 = 0.0;
  if (foot) {
    const double y0 = xk[ry];
    y1 = fma(sd, Yom, y0);
    pen[B.contact] = sd * Yom;
    defect[ry] = y1 - xk1[ry];
    a_put(ry, rpy, 10, tg.Yp[0]);
    a_put(ry, rth, 11, tg.Yr[0]);
    a_put(ry, rvy, 12, tg.Yp[1]);
    a_put(ry, rom, 13, tg.Yr[1]);
    a_put(ry, ry, 14, one);
    const TP Sy = TP(Yom) + tg.Yr[2] + tg.Yp[2];
    S[ry] = Sy;
    if (wz)
      zr[6] = y1 - double(Sy) * sd - double(tg.Yp[0]) * xk[rpy] - double(tg.Yr[0]) * xk[rth] -
              double(tg.Yp[1]) * xk[rvy] - double(tg.Yr[1]) * xk[rom] - xk[ry];
    if (nu > 0) {
      int o = B.b_off;
      for (int i = 0; i < nin; ++i) {
        const int q = B.idx[i];
        const TP ay = anchor<TP>(B.ay[i]), pc = anchor<TP>(B.p[i]), qc = anchor<TP>(B.q[i]),
                 tc = anchor<TP>(B.t[i]);
        TP vm = pc * tg.Yr[3] + qc * tg.Yr[4] + tc * tg.Yr[5] + ay * tg.Yp[3];
        TP vp = pc * tg.Yr[6] + qc * tg.Yr[7] + tc * tg.Yr[8] + ay * tg.Yp[4];
        const int d = q - cin;
        if (d >= 0 && d < 3) { vm += tg.Yd[d]; vp += tg.Yd[3 + d]; }
        if constexpr (CMP) {
          o += 1 + (torque(i) ? 2 : 0) + (abs_bits(B.ax[i]) != 0ull ? 2 : 0) + (abs_bits(B.ay[i]) != 0ull ? 2 : 0);
          Bm[o - 1] = vm;
          Bp[o - 1] = vp;
        } else {
          Bm[(size_t)ry * nu + q] = vm;
          Bp[(size_t)ry * nu + q] = vp;
        }
        if (wz) zr[6] -= double(vm) * uL[q] + double(vp) * uR[q];
      }
    }
    chk += y1;
    chkP += Sy;
  }
  if constexpr (cross) {
    // Eq. (12) cross-complementarity rows of the contact: phi_n, lambda^c, gamma, rho^c
    const int yb = 6 * nb + 4 * B.contact;
    const double fn_m = fma(0.5, cD[1], cL[1]), ga_m = fma(0.5, cD[2], cL[2]);  // tau-averages
    const double Ilg = Il + Ig;
    const double y1v[4] = {fma(sd, fn_m, xk[yb]), fma(sd, Ilg, xk[yb + 1]), fma(sd, ga_m, xk[yb + 2]),
                           fma(sd, Ir, xk[yb + 3])};
    // compact: after the foot's 15 A entries (c_t,c_t) for t = 0..3, then
    // (c1,vx) (c1,th) (c1,om)
    constexpr int JA = A_PER_LINK + A_PER_FOOT;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      defect[yb + t] = y1v[t] - xk1[yb + t];
      a_put(yb + t, yb + t, JA + t, one);
      chk += y1v[t];
    }
    a_put(yb + 1, rvx, JA + 4, sdT);
    a_put(yb + 1, rth, JA + 5, tg.Yl[0]);
    a_put(yb + 1, rom, JA + 6, tg.Yl[1]);
    const TP Sl = TP(Ilg) + tg.Yl[2] + tg.Ylv[2];
    S[yb] = TP(fn_m); S[yb + 1] = Sl; S[yb + 2] = TP(ga_m); S[yb + 3] = TP(Ir);
    chkP += Sl;
    if (nu > 0) {
      // compact: after the link's input groups, (c1,q) for the inputs that
      // enter lambda^c, then (c0,phi_n) (c2,gamma) (c3,phi_t) (c3,phi_n)
      int o = B.b_off;
      if constexpr (CMP)
        for (int i = 0; i < nin; ++i)
          o += 1 + (torque(i) ? 2 : 0) + (abs_bits(B.ax[i]) != 0ull ? 2 : 0) + (abs_bits(B.ay[i]) != 0ull ? 2 : 0);
      auto b_put = [&](int r, int q, TP vm, TP vp) {
        if constexpr (CMP) {
          Bm[o] = vm;
          Bp[o] = vp;
          ++o;
        } else {
          Bm[(size_t)r * nu + q] = vm;
          Bp[(size_t)r * nu + q] = vp;
        }
      };
      for (int i = 0; i < nin; ++i) {
        const int q = B.idx[i];
        const TP ax = anchor<TP>(B.ax[i]), pc = anchor<TP>(B.p[i]), qc = anchor<TP>(B.q[i]),
                 tc = anchor<TP>(B.t[i]);
        TP vm = ax * tg.Ylv[0] + pc * tg.Yl[3] + qc * tg.Yl[4] + tc * tg.Yl[5];
        TP vp = ax * tg.Ylv[1] + pc * tg.Yl[6] + qc * tg.Yl[7] + tc * tg.Yl[8];
        const int d = q - cin;
        if (d == 0) { vm += tg.Yld[0]; vp += tg.Yld[1]; }
        else if (d == 2) { vm += tg.Yld[2]; vp += tg.Yld[3]; }
        if (!CMP || abs_bits(B.ax[i]) != 0ull || torque(i) || d == 0 || d == 2) b_put(yb + 1, q, vm, vp);
      }
      b_put(yb, cin + 1, s_2, s_2);
      b_put(yb + 2, cin + 2, s_2, s_2);
      b_put(yb + 3, cin, tg.Yrd[0], tg.Yrd[1]);
      b_put(yb + 3, cin + 1, tg.Yrd[2], tg.Yrd[3]);
    }
  }
  if (!finite_d(chk) || !isfinite(chkP)) atomicOr(status, ST_NONFINITE);

  if (wz) {
    z[rpx] = zr[0]; z[rpy] = zr[1]; z[rth] = zr[2];
    z[rvx] = zr[3]; z[rvy] = zr[4]; z[rom] = zr[5];
    if (foot) z[ry] = zr[6];
  }
}

}  // namespace ciscvx
