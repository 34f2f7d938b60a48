// state_df.cuh — one RK4 substep of one link's FP64 state with the stage
// right-hand sides evaluated in float-float arithmetic (dfloat.cuh), for the
// FP32-Phi kernels (the linearization, the adjoint's forward sweep, and the
// fused pass of both).  Sec. IV-B Eqs. (14)-(15): the time-dilated rotation
//   theta' = s omega,  omega' = s (cos(theta) P(tau) - sin(theta) Q(tau) + T(tau)),
// with P, Q, T affine in tau under the first-order hold (common.cuh), and for
// a foot link the penalty integrand of its contact (Sec. IV-A):
//   y' = s (h(-phi) + h(-lambda_n) + h(-lambda_t+) + h(-lambda_t-)
//          + h(lambda_t+ + lambda_t- - mu lambda_n)),  phi = p_y + (R(theta) rho)_y.
//
// What stays FP64: theta, omega, sin/cos(theta) at the substep start, the
// foot's p_y, v_y and the penalty quadrature; each is advanced once per
// substep by the float-float increment (two FP64 additions per value).
// What moves to the FP32 pipe: every stage value.  With (s0, c0) the sin and
// cos of theta at the substep start and d_j = c_j h k_theta,j-1 the stage's
// angle increment,
//   cos(theta_j) sP - sin(theta_j) sQ = G - sin(d_j) H - (1 - cos(d_j)) G,
//   G = c0 sP - s0 sQ,  H = s0 sP + c0 sQ   (sP = s P etc. at the stage time),
// so each stage costs one sin / 1-cos pair of a small increment (Taylor
// series, dfloat.cuh) and two float-float products.  The state then matches
// the FP64 recursion to ~1e-14 relative: every stage slope carries a
// relative error of a few 2^-48, which the substep accumulates like FP64
// rounding, far below the 1e-10 state tolerance.
//
// The same pass hands the FP32 stage data to the tangent recursion (the high
// parts of the float-float stage values), which replaces the separate FP32
// copy of the stage recursion the tangents used before.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace ciscvx {

// x += d (two FP64 additions of the widened parts; the widening is exact and
// runs on the integer pipe).
__device__ __forceinline__ void add_df(double& x, dflt d) { x = (x + widen(d.h)) + widen(d.l); }

// sin(d) and 1 - cos(d) of a stage's angle increment: the short Taylor tier
// when every lane of the warp has |d| <= 0.02, else (out of line, so that
// the rare paths do not crowd the instruction cache) the long tier per lane
// (|d| <= 0.2), else FP64 sincos of d (also taken by NaN).
static __device__ __noinline__ void rot_inc_slow(dflt d, dflt& sn, dflt& vc) {
  if (fabsf(d.h) <= 0.2f) {
    sin_vers_long(d, sn, vc);
  } else {
    double s, c;
    sincos(widen(d.h) + widen(d.l), &s, &c);
    sn = df_split(s);
    vc = df_split(1.0 - c);
  }
}

__device__ __forceinline__ void rot_inc(dflt d, unsigned amask, dflt& sn, dflt& vc) {
  if (__all_sync(amask, fabsf(d.h) <= 0.02f)) sin_vers_short(d, sn, vc);
  else rot_inc_slow(d, sn, vc);
}

// Per-interval constants of one link (float-float).
struct DfLink {
  dflt s;                             // dilation s_k
  dflt h, h2, h3, h6;                 // h = 1/n_sub, h/2, h/3, h/6
  dflt sc2, sc3;                      // s h / 2, s h
  dflt sPL, sdP, sQL, sdQ, sTL, sdT;  // s P, s Q, s T at tau = 0 and their increments over [0, 1]
  // foot link only
  dflt sAyg, sdAy;                    // s (A_y(0) - g) and its increment
  dflt crx, cry, mu;                  // contact point (body frame), friction coefficient
  dflt cL[3], cD[3];                  // contact inputs at tau = 0 and their increments
};

__device__ __forceinline__ DfLink df_link(double sd, int nsub, double PL, double dP, double QL, double dQ,
                                          double TL, double dT, double AyL, double dAy, double g, bool foot,
                                          double crx, double cry, double mu, const double* cL,
                                          const double* cD) {
  DfLink C;
  C.s = df_split(sd);
  // h = 1/n_sub: exact for a power of two, else the float-float quotient
  const float nf = (float)nsub;
  const float hh = 1.0f / nf;
  C.h = dflt{hh, f_mul(f_fma(-hh, nf, 1.0f), hh)};  // residual of 1 - hh n, divided by n
  C.h = fast_two_sum(C.h.h, C.h.l);
  C.h2 = df_scale(C.h, 0.5f);
  C.h3 = df_mul(C.h, DF_CONST(1.0 / 3.0));
  C.h6 = df_scale(C.h3, 0.5f);
  C.sc2 = df_mul(C.s, C.h2);
  C.sc3 = df_mul(C.s, C.h);
  C.sPL = df_mul(C.s, df_split(PL)); C.sdP = df_mul(C.s, df_split(dP));
  C.sQL = df_mul(C.s, df_split(QL)); C.sdQ = df_mul(C.s, df_split(dQ));
  C.sTL = df_mul(C.s, df_split(TL)); C.sdT = df_mul(C.s, df_split(dT));
  if (foot) {
    C.sAyg = df_mul(C.s, df_sub(df_split(AyL), df_split(g)));
    C.sdAy = df_mul(C.s, df_split(dAy));
    C.crx = df_split(crx); C.cry = df_split(cry); C.mu = df_split(mu);
#pragma unroll
    for (int m = 0; m < 3; ++m) { C.cL[m] = df_split(cL[m]); C.cD[m] = df_split(cD[m]); }
  }
  return C;
}

// The input-only penalty terms at stage time t (float-float).
__device__ __forceinline__ dflt input_penalty_df(const DfLink& C, dflt t) {
  const dflt ln = df_add(C.cL[0], df_mul(t, C.cD[0]));
  const dflt ltp = df_add(C.cL[1], df_mul(t, C.cD[1]));
  const dflt ltm = df_add(C.cL[2], df_mul(t, C.cD[2]));
  const dflt cone = df_sub(df_add(ltp, ltm), df_mul(C.mu, ln));
  return df_add(df_add(huber_df(df_neg(ln)), huber_df(df_neg(ltp))),
                df_add(huber_df(df_neg(ltm)), huber_df(cone)));
}

// FP64 state of one link between substeps, plus the float-float values the
// next substep takes over from the last (stage time t = end of this substep).
struct DfState {
  double th, om, sth, cth;  // theta, omega, sin/cos(theta) at the substep start
  double py, vy, Y;         // foot: p_y, v_y, penalty quadrature
  dflt sP, sQ, sT;          // s P, s Q, s T at the substep start
  dflt kvy, H;              // foot: s a_y and the input-only penalty at the substep start
};

// FP32 stage data for the tangent recursion (per stage j of a substep).
struct StageF {
  float cs, sn, ws, tau;  // cos / sin of the stage angle, omega, tau
  float pys, vys;         // foot: p_y, v_y at the stage
};

// Initial state: x_k of the link, its sin/cos, the input sums and (foot) the
// penalty quadrature's h/6 H(0) term.
template <bool FOOT>
__device__ __forceinline__ DfState df_state_init(const DfLink& C, double th, double om, double py, double vy) {
  DfState S;
  S.th = th; S.om = om; S.py = py; S.vy = vy; S.Y = 0.0;
  sincos(th, &S.sth, &S.cth);
  S.sP = C.sPL; S.sQ = C.sQL; S.sT = C.sTL;
  if (FOOT) {
    S.kvy = C.sAyg;
    S.H = input_penalty_df(C, dflt{0.0f, 0.0f});
    add_df(S.Y, df_mul(C.h6, S.H));
  }
  return S;
}

// Substep i: advances S by one RK4 step; SD: fill sd[0..3] for the tangents.
template <bool FOOT, bool SD>
__device__ __forceinline__ void df_substep(const DfLink& C, int i, unsigned amask, DfState& S, StageF* sd) {
  const dflt s0 = df_split(S.sth), c0 = df_split(S.cth), w0 = df_split(S.om);
  const dflt som = df_mul(C.s, w0);
  const float fi = (float)i;
  const dflt tm = df_mul_f(C.h, fi + 0.5f), te = df_mul_f(C.h, fi + 1.0f);
  const dflt sPm = df_add(C.sPL, df_mul(tm, C.sdP)), sQm = df_add(C.sQL, df_mul(tm, C.sdQ));
  const dflt sTm = df_add(C.sTL, df_mul(tm, C.sdT));
  const dflt sPe = df_add(C.sPL, df_mul(te, C.sdP)), sQe = df_add(C.sQL, df_mul(te, C.sdQ));
  const dflt sTe = df_add(C.sTL, df_mul(te, C.sdT));
  const dflt GT0 = df_add(df_sub(df_mul(c0, S.sP), df_mul(s0, S.sQ)), S.sT);
  const dflt Gm = df_sub(df_mul(c0, sPm), df_mul(s0, sQm)), Hm = df_add(df_mul(s0, sPm), df_mul(c0, sQm));
  const dflt Ge = df_sub(df_mul(c0, sPe), df_mul(s0, sQe)), He = df_add(df_mul(s0, sPe), df_mul(c0, sQe));
  const dflt GTm = df_add(Gm, sTm), GTe = df_add(Ge, sTe);

  // foot: translation channel, lever arm at the substep start, input penalty
  dflt py0{0.f, 0.f}, vy0{0.f, 0.f}, svy{0.f, 0.f}, kvym{0.f, 0.f}, kvye{0.f, 0.f};
  dflt Rx0{0.f, 0.f}, Ry0{0.f, 0.f}, Hm_{0.f, 0.f}, He_{0.f, 0.f};
  dflt kpy{0.f, 0.f}, kvy{0.f, 0.f}, apy{0.f, 0.f}, avy{0.f, 0.f}, ay{0.f, 0.f};
  if (FOOT) {
    py0 = df_split(S.py);
    vy0 = df_split(S.vy);
    svy = df_mul(C.s, vy0);
    kvym = df_add(C.sAyg, df_mul(tm, C.sdAy));
    kvye = df_add(C.sAyg, df_mul(te, C.sdAy));
    Rx0 = df_sub(df_mul(c0, C.crx), df_mul(s0, C.cry));
    Ry0 = df_add(df_mul(s0, C.crx), df_mul(c0, C.cry));
    Hm_ = input_penalty_df(C, tm);
    He_ = input_penalty_df(C, te);
  }

  // stage 0
  dflt kth = som, kom = GT0;
  dflt ath = kth, aom = kom;  // k_0 + 2 k_1 + 2 k_2 + k_3
  if (SD) {
    sd[0].cs = c0.h; sd[0].sn = s0.h; sd[0].ws = w0.h; sd[0].tau = df_mul_f(C.h, fi).h;
  }
  if (FOOT) {
    kpy = svy;
    kvy = S.kvy;
    apy = kpy;
    avy = kvy;
    ay = huber_df(df_neg(df_add(py0, Ry0)));
    if (SD) { sd[0].pys = py0.h; sd[0].vys = vy0.h; }
  }
#pragma unroll
  for (int j = 1; j < 4; ++j) {
    const dflt& ch = (j == 3) ? C.h : C.h2;
    const dflt d = df_mul(ch, kth);
    dflt sdj, vdj;
    rot_inc(d, amask, sdj, vdj);
    const dflt& G = (j == 3) ? Ge : Gm;
    const dflt& H = (j == 3) ? He : Hm;
    const dflt& GT = (j == 3) ? GTe : GTm;
    if (SD) {
      const float omv = 1.0f - vdj.h;
      sd[j].cs = c0.h * omv - s0.h * sdj.h;
      sd[j].sn = s0.h * omv + c0.h * sdj.h;
      sd[j].ws = w0.h + ch.h * kom.h;  // omega at the stage (kom: the previous stage's slope)
      sd[j].tau = (j == 3) ? te.h : tm.h;
    }
    if (FOOT) {
      const dflt pys = df_add(py0, df_mul(ch, kpy));  // kpy, kvy: the previous stage's slopes
      if (SD) { sd[j].pys = pys.h; sd[j].vys = vy0.h + ch.h * kvy.h; }
      kpy = df_add(svy, df_mul((j == 3) ? C.sc3 : C.sc2, kvy));
      kvy = (j == 3) ? kvye : kvym;
      const dflt Ry = df_sub(df_add(Ry0, df_mul(sdj, Rx0)), df_mul(vdj, Ry0));
      const dflt hj = huber_df(df_neg(df_add(pys, Ry)));
      if (j == 3) { apy = df_add(apy, kpy); avy = df_add(avy, kvy); ay = df_add(ay, hj); }
      else {
        apy = df_add(apy, df_scale(kpy, 2.0f));
        avy = df_add(avy, df_scale(kvy, 2.0f));
        ay = df_add(ay, df_scale(hj, 2.0f));
      }
    }
    kth = df_add(som, df_mul((j == 3) ? C.sc3 : C.sc2, kom));
    kom = df_sub(df_sub(GT, df_mul(sdj, H)), df_mul(vdj, G));
    if (j == 3) { ath = df_add(ath, kth); aom = df_add(aom, kom); }
    else { ath = df_add(ath, df_scale(kth, 2.0f)); aom = df_add(aom, df_scale(kom, 2.0f)); }
  }
  // substep update: theta, omega and sin/cos(theta) (FP64 accumulation)
  const dflt Dth = df_mul(C.h6, ath);
  dflt sdD, vdD;
  rot_inc(Dth, amask, sdD, vdD);
  const dflt ds = df_sub(df_mul(c0, sdD), df_mul(s0, vdD));
  const dflt dc = df_neg(df_add(df_mul(s0, sdD), df_mul(c0, vdD)));
  add_df(S.th, Dth);
  add_df(S.om, df_mul(C.h6, aom));
  add_df(S.sth, ds);
  add_df(S.cth, dc);
  S.sP = sPe; S.sQ = sQe; S.sT = sTe;
  if (FOOT) {
    add_df(S.py, df_mul(C.h6, apy));
    add_df(S.vy, df_mul(C.h6, avy));
    // penalty: h/6 (stage terms) + Simpson's h/3 (2 H(t_m) + H(t_e)) for the input-only terms
    add_df(S.Y, df_add(df_mul(C.h6, ay), df_mul(C.h3, df_add(df_scale(Hm_, 2.0f), He_))));
    S.kvy = kvye;
    S.H = He_;
  }
}

// End of the last substep: the input-only terms' end point was counted with
// h/3 (Simpson's h/6 at each end of the interval).
template <bool FOOT>
__device__ __forceinline__ void df_state_finish(const DfLink& C, DfState& S) {
  if (FOOT) add_df(S.Y, df_neg(df_mul(C.h6, S.H)));
}

}  // namespace ciscvx
