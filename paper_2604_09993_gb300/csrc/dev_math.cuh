// dev_math.cuh — scalar device math shared by the library's kernels and by
// the sources the library compiles at run time (NVRTC): no host headers, only
// CUDA built-ins.
#pragma once

namespace ciscvx {

// FP64 -> FP32 rounded toward zero, on the integer pipe (a conversion
// instruction takes an FP64-pipe slot on this GPU).  From the two IEEE
// formats: keep the sign, rebias the exponent (1023 -> 127), keep the top 23
// of the 52 mantissa bits.  Magnitudes below the smallest normal FP32 number
// give a signed zero, larger finite magnitudes than the largest FP32 number
// give that number, infinities stay infinite and NaNs stay NaN.  Used for the
// FP32 anchors of the tangent recursion and for the FP32 stage data of the
// coupled path's nominal pass, which tolerate one FP32 ulp.
__device__ __forceinline__ float to_f32_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;          // FP32 biased exponent
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 mantissa bits
  unsigned r = sign | ((unsigned)e << 23) | m;
  if (e <= 0) r = sign;
  if (e >= 255) {
    const bool special = (hi & 0x7ff00000u) == 0x7ff00000u;
    const bool nan = special && (((hi & 0xfffffu) | lo) != 0u);
    r = special ? (sign | (nan ? 0x7fc00000u : 0x7f800000u)) : (sign | 0x7f7fffffu);
  }
  return __uint_as_float(r);
}

// Pseudo-Huber ramp h(z) = sqrt(1 + p^2) - 1 = p^2 / (1 + sqrt(1 + p^2)),
// p = max(z, 0), and its derivative h'(z) = p / sqrt(1 + p^2).
__device__ __forceinline__ void huber(double z, double& H, double& D) {
  const double p = fmax(z, 0.0);
  const double r = sqrt(fma(p, p, 1.0));
  H = (p * p) / (1.0 + r);
  D = p / r;
}

// Value only: h(z) in FP64 for the penalty state, as a rsqrt(a) - 1 with
// a = 1 + z^2 (about 7 FP64 issue slots on this GPU against about 18 for
// z^2 / (1 + sqrt(a))).  Its absolute error is a few ulp of a, i.e. ~1e-15
// for |z| <= 10; the cancellation for small z only affects the relative error
// of values far below the penalty's magnitude.  Lanes with z <= 0 skip it.
__device__ __forceinline__ double huber_value(double z) {
  double H = 0.0;
  if (__double_as_longlong(z) > 0) {  // z > 0, tested on the bit pattern
    const double a = fma(z, z, 1.0);
    H = fma(a, rsqrt(a), -1.0);
  }
  return H;
}

// Value in FP32 (adjoint weights only; the penalty state itself uses the FP64
// value): p^2 / (1 + sqrt(1 + p^2)) with the square root as a rsqrt(a) and
// the fast division, a few ulp.
__device__ __forceinline__ float huber_value(float z) {
  const float p = fmaxf(z, 0.0f);
  const float a = fmaf(p, p, 1.0f);
  return __fdividef(p * p, fmaf(a, rsqrtf(a), 1.0f));
}

// (sin, cos) of theta0 + d in FP32 from (s0, c0) = (sin, cos)(theta0):
// Taylor series of sin d through d^7 and of cos d through d^8 (truncation
// below 6e-9 for |d| <= 0.5, under FP32 rounding), then angle addition; for
// |d| > 0.5 (or NaN) sincosf of theta0 + d, out of line.
static __device__ __noinline__ void sincos_f32_far(float th, float* s, float* c) { sincosf(th, s, c); }

__device__ __forceinline__ void sincos_f32_step(float th0, float s0, float c0, float d, float& s, float& c) {
  if (fabsf(d) <= 0.5f) {
    const float x = d * d;
    const float sd = d * fmaf(x, fmaf(x, fmaf(x, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    const float cm = x * fmaf(x, fmaf(x, fmaf(x, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f);
    s = fmaf(s0, cm, fmaf(c0, sd, s0));  // s0 cos d + c0 sin d
    c = fmaf(c0, cm, fmaf(-s0, sd, c0));  // c0 cos d - s0 sin d
  } else {
    sincos_f32_far(th0 + d, &s, &c);
  }
}

// Derivative only, in the tangent precision: h'(z) = p / sqrt(1 + p^2).
__device__ __forceinline__ float huber_slope(float z) {
  const float p = fmaxf(z, 0.0f);
  return p * rsqrtf(fmaf(p, p, 1.0f));
}
__device__ __forceinline__ double huber_slope(double z) {
  const double p = fmax(z, 0.0);
  return p * rsqrt(fma(p, p, 1.0));
}

// (sin, cos) of theta + d from (s0, c0) = (sin theta, cos theta) by angle
// addition, with sin d and cos d from their Taylor series.  Two tiers, chosen
// per warp so that no FP64 instruction runs partly masked:
//  * short, used when every active lane has |d| <= 0.02:
//    sin d through d^5, cos d through d^6 (truncation <= 2.6e-16 absolute);
//  * long, |d| <= 0.2: sin d through d^9, cos d through d^10 (<= 5e-16).
// Lanes with |d| > 0.2 (or a NaN) return false; the caller uses sincos.
constexpr double ROT_SHORT = 0.02;
constexpr double ROT_DMAX = 0.2;

__device__ __forceinline__ unsigned long long abs_bits(double d) {
  return (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ bool rotate_small(double s0, double c0, double d, bool short_tier,
                                             double& s, double& c) {
  if (abs_bits(d) > (unsigned long long)__double_as_longlong(ROT_DMAX)) return false;
  const double x = d * d;
  double ps, pc;
  if (short_tier) {
    ps = fma(x, 1.0 / 120.0, -1.0 / 6.0);
    ps = fma(ps, x, 1.0);
    pc = fma(x, -1.0 / 720.0, 1.0 / 24.0);
    pc = fma(pc, x, -0.5);
  } else {
    ps = fma(x, 1.0 / 362880.0, -1.0 / 5040.0);
    ps = fma(ps, x, 1.0 / 120.0);
    ps = fma(ps, x, -1.0 / 6.0);
    ps = fma(ps, x, 1.0);
    pc = fma(x, -1.0 / 3628800.0, 1.0 / 40320.0);
    pc = fma(pc, x, -1.0 / 720.0);
    pc = fma(pc, x, 1.0 / 24.0);
    pc = fma(pc, x, -0.5);
  }
  const double sd = d * ps;
  const double cd = fma(pc, x, 1.0);
  s = fma(s0, cd, c0 * sd);
  c = fma(c0, cd, -(s0 * sd));
  return true;
}

// (sin, cos) of theta0 + d given those of theta0; `active` is the mask of
// lanes executing this call (they vote on the tier); falls back to
// sincos(theta0 + d), the sum formed only on that path.
__device__ __forceinline__ void sincos_step(double th0, double s0, double c0, double d,
                                            unsigned active, double& s, double& c) {
  const bool short_tier =
      __all_sync(active, abs_bits(d) <= (unsigned long long)__double_as_longlong(ROT_SHORT));
  if (!rotate_small(s0, c0, d, short_tier, s, c)) sincos(th0 + d, &s, &c);
}

// Contact surface y = ta sin(tk x) at the world point (xc, yc) (Sec. VI-B;
// ta = 0: flat ground y = 0): approximate signed distance phi = h^c /
// ||grad h^c||, h^c = y - ta sin(tk x); unit normal n = grad h^c / ||grad h^c||
// (grad phi on the surface); tangent t = (n_y, -n_x); their derivatives along
// x (nothing depends on y but phi).
struct SurfFrame {
  double phi, tx, ty, nx, ny, phix, phiy, dtx, dty, dnx, dny;
};

// The same frame from (sk, ck) = (sin, cos)(tk xc), for callers that chain
// those across stages instead of evaluating them (ta != 0).
__device__ __forceinline__ SurfFrame contact_surface_sc(double ta, double tk, double yc, double sk,
                                                       double ck) {
  SurfFrame f;
  const double hc = fma(-ta, sk, yc);
  const double gx = -(ta * tk) * ck;       // dh^c/dx
  const double gp = (ta * tk * tk) * sk;   // d gx / dx
  const double w = rsqrt(fma(gx, gx, 1.0));
  const double w3g = gp * w * w * w;
  f.phi = hc * w;
  f.nx = gx * w; f.ny = w;
  f.tx = w; f.ty = -f.nx;
  f.phix = f.nx * fma(-hc * w * w, gp, 1.0);  // gx w (1 - h^c w^2 gp)
  f.phiy = w;
  f.dnx = w3g; f.dny = -gx * w3g;             // dn/dx = gp w^3 (1, -gx)
  f.dtx = -gx * w3g; f.dty = -w3g;            // dt/dx = gp w^3 (-gx, -1)
  return f;
}

__device__ __forceinline__ SurfFrame contact_surface(double ta, double tk, double xc, double yc) {
  if (ta == 0.0) {
    SurfFrame f;
    f.phi = yc;
    f.tx = 1.0; f.ty = 0.0; f.nx = 0.0; f.ny = 1.0;
    f.phix = 0.0; f.phiy = 1.0;
    f.dtx = f.dty = f.dnx = f.dny = 0.0;
    return f;
  }
  double sk, ck;
  sincos(tk * xc, &sk, &ck);
  return contact_surface_sc(ta, tk, yc, sk, ck);
}

// Where interval e's data live (the library's batch instance table has this
// layout): for a single instance (entries null) interval e itself; in a batch,
// entry e = (instance, k).
struct InstRec {
  int model, N, nsub, pad_;
  long long x, u, s, a, b, v, p;  // element offsets: X, U, s, A, Bm/Bp, S/defect, penalty
  long long part, pb;
};

struct IvRef {
  long long x, u, s, a, b, v, p;
};

// a_stride: elements of A per interval (n_x~^2 dense; the compact pattern's
// size for compact outputs).
__device__ __forceinline__ IvRef iv_ref(long long e, int nxt, int nu, int nc, int layout,
                                        const int2* entries, const InstRec* inst,
                                        long long a_stride) {
  IvRef r;
  long long k = e;
  long long x = 0, u = 0, sv = 0, a = 0, b = 0, v = 0, p = 0;
  if (entries) {
    const int2 en = entries[e];
    const InstRec& I = inst[en.x];
    k = en.y;
    x = I.x; u = I.u; sv = I.s; a = I.a; b = I.b; v = I.v; p = I.p;
  }
  r.x = x + k * nxt;
  r.u = u + (layout == 0 ? k : 2 * k) * nu;
  r.s = sv + k;
  r.a = a + k * a_stride;
  r.b = b + k * nxt * nu;
  r.v = v + k * nxt;
  r.p = p + k * nc;
  return r;
}

// FP32 -> FP64 (exact) from the IEEE-754 binary32 and binary64 layouts on the
// integer pipe: exponent rebiased by 1023 - 127, the 23 fraction bits moved
// to the top of the 52.  Zeros keep their sign; subnormals, infinities and
// NaNs take the conversion instruction.  On this part the conversion
// instruction occupies the FP64 pipe, which bounds the kernels that read FP32
// blocks into FP64 sums.
__device__ __forceinline__ double widen(unsigned u) {
  const unsigned e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e == 0u || e == 0xFFu) return (double)__uint_as_float(u);
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double widen(float f) { return widen(__float_as_uint(f)); }
__device__ __forceinline__ double widen(double d) { return d; }

}  // namespace ciscvx
