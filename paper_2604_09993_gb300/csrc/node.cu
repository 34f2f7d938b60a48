// node.cu — node constraints of the transcription (Sec. IV-C, Eqs. (17e)-(17f)):
// the impact map G~ with the joint impulse eliminated (Eq. (6a), Sec. II-B)
// and the Fischer-Burmeister-relaxed impulse conditions Theta^delta
// (Eqs. (6b)-(6e) relaxed by Eq. (16)), with their Jacobians.
//
// Impact map (all kinematics at the pre-impact pose q-; M = diag(m, m, I)):
//   w  = v- + M^-1 J_c^T Phi,   K = C' M^-1 C'^T,   mu = K^-1 C' w
//   v rows of G~:  M (v+ - v-) - J_c^T Phi + C'^T mu        (Lambda = -mu)
// with C' = grad C the revolute-joint constraint Jacobian.  Its derivatives:
//   d/dv-    : column c = -M e_c + C'^T K^-1 C' e_c             (= -M P)
//   d/dPhi   : column   = -f + C'^T K^-1 C' M^-1 f,  f = J_c^T e (one impulse component)
//   d/dtheta_b: with v^ = w - M^-1 C'^T mu (the post-impact velocity the map
//     implies) and a_b = -sum_i r_i . Phi_i + sum_j s_jb r_jb . mu_j (theta_b
//     component of dJ_c^T Phi - dC'^T mu), column = -a_b e_theta_b + C'^T K^-1 t,
//     t_j = s_jb (-r_jb omega^_b + perp(r_jb) a_b / I_b) for the joints j on link b,
//   where r are world lever arms, perp(r) = (-r_y, r_x) = d(R rho)/dtheta and
//   s_jb = +1 (child) / -1 (parent).
// On the sinusoidal surface (Sec. VI-B) the contact frame [t n] is taken at
// the pre-impact contact point x_c = p_x- + r_x, so the world impulse
// I = t Phi_t + n Phi_n moves with p_x- and theta- of the contact's link:
// dI/dx_c = (dt/dx) Phi_t + (dn/dx) Phi_n =: D.  With h = F' - C''^T mu for a
// coordinate the generalized impulse F = J_c^T R_c Phi depends on, the v rows'
// column is -h + C'^T K^-1 (C'' v^ + C' M^-1 h):
//   d/dtheta_b: h = a_b e_theta + g, g = (dI, r x dI), dI = -r_y D;
//   d/dp_x-   : h = (D, r x D) (C' does not depend on positions);
//   d/dPhi    : h = (t or n, r x (t or n)).
// Theta's pairs read the contact point's distance phi and its velocity in the
// contact frame: c = n . (v_c+ + e v_c-), lambda^c = t . v_c+ + Gamma
// dPhi_t/..., with v_c = (v_x - omega r_y, v_y + omega r_x).
//
// Mapping: lane = node.  The joint impulse couples every link of a node, so
// one thread owns one node; a warp's 32 lanes run the same program on 32
// nodes of one model, so no FP64 instruction runs partly masked.  K's
// L D L^T factor, the lever arms and the solve vectors sit in shared memory,
// element major ([element][lane]), so a warp's access to one element is one
// contiguous 256-byte row; products with C' and C'^T go through per-link
// joint lists, so no dense C' is formed.  FP64 throughout (the state
// precision).
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace ciscvx {

namespace {

// What the node kernel reads of a model, passed by value as a kernel
// parameter (constant bank: uniform loads are broadcast from the constant
// cache instead of going through L1).
struct NodeTab {
  int nb, nj, nc, nxt;
  int nadj[MAXB];
  unsigned char adj[MAXB][NODE_MAXADJ];  // (joint << 1) | (1 if the link is the joint's parent)
  int npos[NODE_MAXJ], nord[NODE_MAXJ], jchi[NODE_MAXJ], jpar[NODE_MAXJ];
  int nf[2 * NODE_MAXJ], noff[2 * NODE_MAXJ + 1];
  int lmin[MAXB], contact[MAXB];
  double jrc[NODE_MAXJ][2], jrp[NODE_MAXJ][2];
  double mass[MAXB], inertia[MAXB], minv[MAXB], iinv[MAXB];
  double crho[MAXB][2], mu[MAXB];
  double delta, e[MAXB];
  double ta, tk;  // contact surface y = ta sin(tk x)
};

// Per-lane scratch layout (in doubles; each element is a row of 32 lanes).
struct NodeLayout {
  int arm, carm, fr, K, wh, mu, x, total;
};

// per-contact contact-frame slots (at the pre-impact contact point)
constexpr int FR_TX = 0, FR_TY = 1, FR_NX = 2, FR_NY = 3, FR_DTX = 4, FR_DTY = 5, FR_DNX = 6,
              FR_DNY = 7, FR_PHI = 8, FR_PHIX = 9, FR_PHIY = 10, FR_N = 11;

__host__ __device__ inline NodeLayout node_layout(int nb, int nj, int nc, int nsky, bool terrain) {
  const int nk = 2 * nj;
  NodeLayout L;
  L.arm = 0;                       // perp lever arms per joint: child x, y; parent x, y (4 nj)
  L.carm = L.arm + 4 * nj;         // world lever arm r of each contact point          (2 nc)
  L.fr = L.carm + 2 * nc;          // contact frame, its x-derivatives, phi (FR_N nc; sinusoidal surface only)
  L.K = L.fr + (terrain ? FR_N * nc : 0);  // K = L D L^T in skyline rows: unit L left of the diagonal, 1/D on it (nsky)
  L.wh = L.K + nsky;               // omega^ of every link (post-impact velocity the map implies) (nb)
  L.mu = L.wh + nb;                // mu = K^-1 C' w                                    (nk)
  L.x = L.mu + nk;                 // right-hand side / solution of one solve          (nk)
  L.total = L.x + nk;
  return L;
}

#define SM(e) sm[(e) * 32]
// entry (i, k) of K / its factor, f_i <= k <= i (skyline storage)
#define LK(i, k) SM(Ly.K + M.noff[i] + (k) - M.nf[i])

// Solves K x = x in place with the L D L^T factor (one multiply per row);
// x is zero in rows before i0 (the caller zeroes them), so the forward pass
// starts at row i0.
__device__ __forceinline__ void ldl_solve(const NodeTab& M, double* sm, const NodeLayout& Ly,
                                          int nk, int i0) {
  for (int i = (i0 > 1 ? i0 : 1); i < nk; ++i) {
    double acc = SM(Ly.x + i);
    const int k0 = M.nf[i] > i0 ? M.nf[i] : i0;
    for (int k = k0; k < i; ++k) acc = fma(-LK(i, k), SM(Ly.x + k), acc);
    SM(Ly.x + i) = acc;
  }
  for (int i = nk - 1; i >= 0; --i) {
    double acc = SM(Ly.x + i) * LK(i, i);
    for (int k = i + 1; k < nk; ++k)
      if (M.nf[k] <= i) acc = fma(-LK(k, i), SM(Ly.x + k), acc);
    SM(Ly.x + i) = acc;
  }
}

// (C'^T y) on link b, components 0..2, for the vector y at element offset yo.
__device__ __forceinline__ void ct_link(const NodeTab& M, const double* sm, const NodeLayout& Ly,
                                        int yo, int b, double& o0, double& o1, double& o2) {
  o0 = o1 = o2 = 0.0;
  for (int t = 0; t < M.nadj[b]; ++t) {
    const int code = M.adj[b][t], j = code >> 1, role = code & 1, r = 2 * M.npos[j];
    const double y0 = SM(yo + r), y1 = SM(yo + r + 1);
    const double px = SM(Ly.arm + 4 * j + 2 * role), py = SM(Ly.arm + 4 * j + 2 * role + 1);
    if (t == 0) {
      o0 = role ? -y0 : y0;
      o1 = role ? -y1 : y1;
      o2 = role ? -fma(px, y0, py * y1) : fma(px, y0, py * y1);
    } else if (role) {
      o0 -= y0; o1 -= y1; o2 = fma(-px, y0, fma(-py, y1, o2));
    } else {
      o0 += y0; o1 += y1; o2 = fma(px, y0, fma(py, y1, o2));
    }
  }
}

// x <- 0 except, for the joints on link b, s (e0 + perp . (0, 0) ...) as given by the
// generalized vector (f0, f1, f2) on link b: x_j = s (f0, f1) + s perp_jb f2.
__device__ __forceinline__ void c_link(const NodeTab& M, double* sm, const NodeLayout& Ly, int nk,
                                       int b, double f0, double f1, double f2) {
  for (int r = 0; r < nk; ++r) SM(Ly.x + r) = 0.0;
  for (int t = 0; t < M.nadj[b]; ++t) {
    const int code = M.adj[b][t], j = code >> 1, role = code & 1, r = 2 * M.npos[j];
    const double px = SM(Ly.arm + 4 * j + 2 * role), py = SM(Ly.arm + 4 * j + 2 * role + 1);
    const double v0 = fma(px, f2, f0), v1 = fma(py, f2, f1);
    SM(Ly.x + r) = role ? -v0 : v0;
    SM(Ly.x + r + 1) = role ? -v1 : v1;
  }
}

__device__ __forceinline__ double fb(double a, double b, double delta, double& da, double& db) {
  const double r = sqrt(fma(a, a, fma(b, b, delta)));
  const double ir = 1.0 / r;
  da = 1.0 - a * ir;
  db = 1.0 - b * ir;
  return a + b - r;
}

// pseudo-Huber absolute value sqrt(1 + x^2) - 1 and its slope x / sqrt(1 + x^2)
__device__ __forceinline__ double sabs(double x, double& d) {
  const double r = sqrt(fma(x, x, 1.0));
  d = x / r;
  return r - 1.0;
}

__global__ void __launch_bounds__(256) k_node(const __grid_constant__ NodeTab M, int n,
                                              const double* __restrict__ Xp,
                                              const double* __restrict__ Xm,
                                              const double* __restrict__ Phi,
                                              const double* __restrict__ Gam, double* g,
                                              double* Gvm, double* Gth, double* Gphi, double* Gpx,
                                              double* theta, double* dtheta, unsigned* status) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int nb = M.nb, nj = M.nj, nc = M.nc, nxt = M.nxt, nq = 3 * nb, nk = 2 * nj;
  const bool terrain = M.ta != 0.0;
  const NodeLayout Ly = node_layout(nb, nj, nc, M.noff[2 * nj], terrain);
  double* sm = smem + (size_t)warp * Ly.total * 32 + lane;
  const double* xp = Xp + k * nxt;
  const double* xm = Xm + k * nxt;
  const double* ph = Phi ? Phi + k * 2 * nc : nullptr;
  const double* gm = Gam ? Gam + k * nc : nullptr;
  double chk = 0.0;

  // lever arms: perp(R rho) = d(R rho)/dtheta per joint end, R rho per contact
  for (int b = 0; b < nb; ++b) {
    double s, c;
    sincos(xm[3 * b + 2], &s, &c);
    for (int t = 0; t < M.nadj[b]; ++t) {
      const int code = M.adj[b][t], j = code >> 1, role = code & 1;
      const double* rho = role ? M.jrp[j] : M.jrc[j];
      const double rx = c * rho[0] - s * rho[1], ry = s * rho[0] + c * rho[1];
      SM(Ly.arm + 4 * j + 2 * role) = -ry;
      SM(Ly.arm + 4 * j + 2 * role + 1) = rx;
    }
    const int ci = M.contact[b];
    if (ci >= 0) {
      const double rx = c * M.crho[b][0] - s * M.crho[b][1], ry = s * M.crho[b][0] + c * M.crho[b][1];
      SM(Ly.carm + 2 * ci) = rx;
      SM(Ly.carm + 2 * ci + 1) = ry;
      if (terrain) {
        const SurfFrame f = contact_surface(M.ta, M.tk, xm[3 * b] + rx, xm[3 * b + 1] + ry);
        double* F = &SM(Ly.fr + FR_N * ci);
        F[FR_TX * 32] = f.tx; F[FR_TY * 32] = f.ty; F[FR_NX * 32] = f.nx; F[FR_NY * 32] = f.ny;
        F[FR_DTX * 32] = f.dtx; F[FR_DTY * 32] = f.dty; F[FR_DNX * 32] = f.dnx; F[FR_DNY * 32] = f.dny;
        F[FR_PHI * 32] = f.phi; F[FR_PHIX * 32] = f.phix; F[FR_PHIY * 32] = f.phiy;
      }
    }
  }
  // contact-frame value `slot` of contact ci: stored on the sinusoid; on flat
  // ground t = (1, 0), n = (0, 1) and nothing depends on x (phi is formed at its use)
#define FRV(ci, slot) \
  (terrain ? SM(Ly.fr + FR_N * (ci) + (slot)) \
           : ((slot) == FR_TX || (slot) == FR_NY || (slot) == FR_PHIY ? 1.0 : 0.0))

  // K = C' M^-1 C'^T (skyline rows, joints in the children-first order), then K = L D L^T
  for (int r1 = 0; r1 < nk; ++r1) {
    const int j1 = M.nord[r1 >> 1], a1 = r1 & 1;
    for (int r2 = M.nf[r1]; r2 <= r1; ++r2) {
      const int j2 = M.nord[r2 >> 1], a2 = r2 & 1;
      double acc = 0.0;
      for (int u = 0; u < 2; ++u) {
        const int b1 = u ? M.jpar[j1] : M.jchi[j1];
        const double p1 = SM(Ly.arm + 4 * j1 + 2 * u + a1);
        for (int v = 0; v < 2; ++v) {
          const int b2 = v ? M.jpar[j2] : M.jchi[j2];
          if (b1 != b2) continue;
          const double p2 = SM(Ly.arm + 4 * j2 + 2 * v + a2);
          const double e = fma(p1 * p2, M.iinv[b1], (a1 == a2) ? M.minv[b1] : 0.0);
          acc = (u == v) ? acc + e : acc - e;
        }
      }
      LK(r1, r2) = acc;
    }
  }
  // Cholesky L_c by rows within the envelopes (diagonal slot: 1 / L_c,ii), then
  // unit L = L_c diag(1 / L_c,kk) and 1/D = (1 / L_c,ii)^2
  for (int i = 0; i < nk; ++i) {
    const int fi = M.nf[i];
    for (int kk = fi; kk < i; ++kk) {
      double acc = LK(i, kk);
      const int m0 = fi > M.nf[kk] ? fi : M.nf[kk];
      for (int m = m0; m < kk; ++m) acc = fma(-LK(i, m), LK(kk, m), acc);
      LK(i, kk) = acc * LK(kk, kk);
    }
    double d = LK(i, i);
    for (int m = fi; m < i; ++m) d = fma(-LK(i, m), LK(i, m), d);
    LK(i, i) = 1.0 / sqrt(d);
  }
  for (int i = 0; i < nk; ++i)
    for (int kk = M.nf[i]; kk < i; ++kk) LK(i, kk) *= LK(kk, kk);
  for (int i = 0; i < nk; ++i) LK(i, i) = LK(i, i) * LK(i, i);

  // w = v- + M^-1 J_c^T R_c Phi on link b (generalized impulse of its contact:
  // world impulse t Phi_t + n Phi_n at the contact point)
  auto impulse = [&](int b, double& f0, double& f1, double& f2) {
    f0 = f1 = f2 = 0.0;
    const int ci = M.contact[b];
    if (ci >= 0) {
      const double rx = SM(Ly.carm + 2 * ci), ry = SM(Ly.carm + 2 * ci + 1);
      const double pt = ph[2 * ci], pn = ph[2 * ci + 1];
      f0 = fma(FRV(ci, FR_TX), pt, FRV(ci, FR_NX) * pn);
      f1 = fma(FRV(ci, FR_TY), pt, FRV(ci, FR_NY) * pn);
      f2 = rx * f1 - ry * f0;
    }
  };
  // mu = K^-1 C' w
  for (int j = 0; j < nj; ++j) {
    double a0 = 0.0, a1 = 0.0;
    for (int role = 0; role < 2; ++role) {
      const int b = role ? M.jpar[j] : M.jchi[j];
      double f0, f1, f2;
      impulse(b, f0, f1, f2);
      const double w0 = fma(f0, M.minv[b], xm[nq + 3 * b]);
      const double w1 = fma(f1, M.minv[b], xm[nq + 3 * b + 1]);
      const double w2 = fma(f2, M.iinv[b], xm[nq + 3 * b + 2]);
      const double c0 = fma(SM(Ly.arm + 4 * j + 2 * role), w2, w0);
      const double c1 = fma(SM(Ly.arm + 4 * j + 2 * role + 1), w2, w1);
      if (role) { a0 -= c0; a1 -= c1; } else { a0 += c0; a1 += c1; }
    }
    SM(Ly.x + 2 * M.npos[j]) = a0;
    SM(Ly.x + 2 * M.npos[j] + 1) = a1;
  }
  ldl_solve(M, sm, Ly, nk, 0);
  for (int r = 0; r < nk; ++r) SM(Ly.mu + r) = SM(Ly.x + r);

  // residual G~ and omega^ = w_theta - (C'^T mu)_theta / I
  double* gk = g + k * nxt;
  for (int a = 0; a < nq; ++a) gk[a] = xp[a] - xm[a];
  for (int b = 0; b < nb; ++b) {
    double t0, t1, t2, f0, f1, f2;
    ct_link(M, sm, Ly, Ly.mu, b, t0, t1, t2);
    impulse(b, f0, f1, f2);
    const double* vp = xp + nq + 3 * b;
    const double* vm = xm + nq + 3 * b;
    const double g0 = fma(M.mass[b], vp[0] - vm[0], t0 - f0);
    const double g1 = fma(M.mass[b], vp[1] - vm[1], t1 - f1);
    const double g2 = fma(M.inertia[b], vp[2] - vm[2], t2 - f2);
    gk[nq + 3 * b] = g0;
    gk[nq + 3 * b + 1] = g1;
    gk[nq + 3 * b + 2] = g2;
    chk += g0 + g1 + g2;
    SM(Ly.wh + b) = fma(f2 - t2, M.iinv[b], vm[2]);
  }
  for (int a = 2 * nq; a < nxt; ++a) gk[a] = xp[a] - xm[a];  // auxiliary-state continuity

  // d/dv-: column c = -M e_c + C'^T K^-1 C' e_c, stored as row c (the block is symmetric)
  if (Gvm) {
    double* out = Gvm + (size_t)k * nq * nq;
    for (int c = 0; c < nq; ++c) {
      const int bc = c / 3, comp = c - 3 * bc;
      c_link(M, sm, Ly, nk, bc, comp == 0 ? 1.0 : 0.0, comp == 1 ? 1.0 : 0.0, comp == 2 ? 1.0 : 0.0);
      ldl_solve(M, sm, Ly, nk, M.lmin[bc]);
      double* row = out + (size_t)c * nq;
      for (int b = 0; b < nb; ++b) {
        double t0, t1, t2;
        ct_link(M, sm, Ly, Ly.x, b, t0, t1, t2);
        if (b == bc) {
          if (comp == 0) t0 -= M.mass[b];
          else if (comp == 1) t1 -= M.mass[b];
          else t2 -= M.inertia[b];
        }
        row[3 * b] = t0;
        row[3 * b + 1] = t1;
        row[3 * b + 2] = t2;
        chk += t0 + t1 + t2;
      }
    }
  }

  // d/dtheta_b: a_b = -sum_i r_i . Phi_i + sum_j s_jb r_jb . mu_j;
  // t_j = s_jb (-r_jb omega^_b + perp(r_jb) a_b / I_b); column = -a_b e_theta_b + C'^T K^-1 t
  if (Gth) {
    double* out = Gth + (size_t)k * nq * nb;
    for (int b = 0; b < nb; ++b) {
      double ab = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
      const int ci = M.contact[b];
      if (ci >= 0) {
        double i0, i1, i2;
        impulse(b, i0, i1, i2);
        const double rx = SM(Ly.carm + 2 * ci), ry = SM(Ly.carm + 2 * ci + 1);
        ab = -fma(rx, i0, ry * i1);
        // the frame turns with x_c: dI = -r_y (dt/dx Phi_t + dn/dx Phi_n)
        const double pt = ph[2 * ci], pn = ph[2 * ci + 1];
        g0 = -ry * fma(FRV(ci, FR_DTX), pt, FRV(ci, FR_DNX) * pn);
        g1 = -ry * fma(FRV(ci, FR_DTY), pt, FRV(ci, FR_DNY) * pn);
        g2 = rx * g1 - ry * g0;
      }
      for (int t = 0; t < M.nadj[b]; ++t) {
        const int code = M.adj[b][t], j = code >> 1, role = code & 1;
        const double px = SM(Ly.arm + 4 * j + 2 * role), py = SM(Ly.arm + 4 * j + 2 * role + 1);
        // r = (py, -px)
        const double rm = fma(py, SM(Ly.mu + 2 * M.npos[j]), -px * SM(Ly.mu + 2 * M.npos[j] + 1));
        ab = role ? ab - rm : ab + rm;
      }
      const double wb = SM(Ly.wh + b), ai = (ab + g2) * M.iinv[b];
      const double l0 = g0 * M.minv[b], l1 = g1 * M.minv[b];
      for (int r = 0; r < nk; ++r) SM(Ly.x + r) = 0.0;
      for (int t = 0; t < M.nadj[b]; ++t) {
        const int code = M.adj[b][t], j = code >> 1, role = code & 1, r = 2 * M.npos[j];
        const double px = SM(Ly.arm + 4 * j + 2 * role), py = SM(Ly.arm + 4 * j + 2 * role + 1);
        const double t0 = fma(px, ai, fma(-py, wb, l0)), t1 = fma(py, ai, fma(px, wb, l1));
        SM(Ly.x + r) = role ? -t0 : t0;
        SM(Ly.x + r + 1) = role ? -t1 : t1;
      }
      ldl_solve(M, sm, Ly, nk, M.lmin[b]);
      for (int bb = 0; bb < nb; ++bb) {
        double t0, t1, t2;
        ct_link(M, sm, Ly, Ly.x, bb, t0, t1, t2);
        if (bb == b) { t0 -= g0; t1 -= g1; t2 -= ab + g2; }
        out[(size_t)(3 * bb) * nb + b] = t0;
        out[(size_t)(3 * bb + 1) * nb + b] = t1;
        out[(size_t)(3 * bb + 2) * nb + b] = t2;
        chk += t0 + t1 + t2;
      }
    }
  }

  // d/dPhi: column = -f + C'^T K^-1 C' M^-1 f,  f = J_c^T e (one impulse component)
  if (Gphi && nc > 0) {
    double* out = Gphi + (size_t)k * nq * 2 * nc;
    for (int b = 0; b < nb; ++b) {
      const int ci = M.contact[b];
      if (ci < 0) continue;
      const double rx = SM(Ly.carm + 2 * ci), ry = SM(Ly.carm + 2 * ci + 1);
      for (int comp = 0; comp < 2; ++comp) {
        // world direction of the impulse component: t (Phi_t) or n (Phi_n)
        const double f0 = comp == 0 ? FRV(ci, FR_TX) : FRV(ci, FR_NX);
        const double f1 = comp == 0 ? FRV(ci, FR_TY) : FRV(ci, FR_NY);
        const double f2 = rx * f1 - ry * f0;
        c_link(M, sm, Ly, nk, b, f0 * M.minv[b], f1 * M.minv[b], f2 * M.iinv[b]);
        ldl_solve(M, sm, Ly, nk, M.lmin[b]);
        const int col = 2 * ci + comp;
        for (int bb = 0; bb < nb; ++bb) {
          double t0, t1, t2;
          ct_link(M, sm, Ly, Ly.x, bb, t0, t1, t2);
          if (bb == b) { t0 -= f0; t1 -= f1; t2 -= f2; }
          out[(size_t)(3 * bb) * 2 * nc + col] = t0;
          out[(size_t)(3 * bb + 1) * 2 * nc + col] = t1;
          out[(size_t)(3 * bb + 2) * 2 * nc + col] = t2;
          chk += t0 + t1 + t2;
        }
      }
    }
  }

  // d/dp_x- of each contact's link: column = -f + C'^T K^-1 C' M^-1 f, f = (D, r x D),
  // D = (dt/dx) Phi_t + (dn/dx) Phi_n (zero on flat ground)
  if (Gpx && nc > 0 && !terrain) {  // on flat ground the frame does not move: the block is 0
    double* out = Gpx + (size_t)k * nq * nc;
    for (int q = 0; q < nq * nc; ++q) out[q] = 0.0;
  } else if (Gpx && nc > 0) {
    double* out = Gpx + (size_t)k * nq * nc;
    for (int b = 0; b < nb; ++b) {
      const int ci = M.contact[b];
      if (ci < 0) continue;
      const double rx = SM(Ly.carm + 2 * ci), ry = SM(Ly.carm + 2 * ci + 1);
      const double pt = ph[2 * ci], pn = ph[2 * ci + 1];
      const double f0 = fma(FRV(ci, FR_DTX), pt, FRV(ci, FR_DNX) * pn);
      const double f1 = fma(FRV(ci, FR_DTY), pt, FRV(ci, FR_DNY) * pn);
      const double f2 = rx * f1 - ry * f0;
      c_link(M, sm, Ly, nk, b, f0 * M.minv[b], f1 * M.minv[b], f2 * M.iinv[b]);
      ldl_solve(M, sm, Ly, nk, M.lmin[b]);
      for (int bb = 0; bb < nb; ++bb) {
        double t0, t1, t2;
        ct_link(M, sm, Ly, Ly.x, bb, t0, t1, t2);
        if (bb == b) { t0 -= f0; t1 -= f1; t2 -= f2; }
        out[(size_t)(3 * bb) * nc + ci] = t0;
        out[(size_t)(3 * bb + 1) * nc + ci] = t1;
        out[(size_t)(3 * bb + 2) * nc + ci] = t2;
        chk += t0 + t1 + t2;
      }
    }
  }

  // Theta^delta per contact, and its Jacobian in the contact's local variables
  // (p_x-, p_y-, theta-, v_x+, v_y+, omega+, v_x-, v_y-, omega-, Phi_t, Phi_n, Gamma)
  // of its link.
  for (int b = 0; b < nb; ++b) {
    const int ci = M.contact[b];
    if (ci < 0) continue;
    const double rx = SM(Ly.carm + 2 * ci), ry = SM(Ly.carm + 2 * ci + 1);
    const double pt = ph[2 * ci], pn = ph[2 * ci + 1], ga = gm[ci], e = M.e[ci];
    const double mu = M.mu[b];
    const double tx = FRV(ci, FR_TX), ty = FRV(ci, FR_TY), nx = FRV(ci, FR_NX), ny = FRV(ci, FR_NY);
    const double wp = xp[nq + 3 * b + 2], wm = xm[nq + 3 * b + 2];
    const double phi = terrain ? FRV(ci, FR_PHI) : xm[3 * b + 1] + ry;  // flat: p_y- + r_y
    // contact-point velocities after (p) and before (m) the impact
    const double vxp = fma(-wp, ry, xp[nq + 3 * b]), vyp = fma(wp, rx, xp[nq + 3 * b + 1]);
    const double vxm = fma(-wm, ry, xm[nq + 3 * b]), vym = fma(wm, rx, xm[nq + 3 * b + 1]);
    const double Vx = fma(e, vxm, vxp), Vy = fma(e, vym, vyp);  // v_c+ + e v_c-
    const double cn = fma(nx, Vx, ny * Vy);
    const double vtp = fma(tx, vxp, ty * vyp);
    const double sq = sqrt(fma(pt, pt, 1.0));
    const double gn = pt / sq;
    const double lc = fma(ga, gn, vtp);
    double dcn, dlc, dmn, dpt;
    const double scn = sabs(cn, dcn), slc = sabs(lc, dlc);
    const double smn = sabs(mu * pn, dmn), spt = sabs(pt, dpt);
    const double rho = smn - spt;
    double f0a, f0b, f1a, f1b, f2a, f2b, f3a, f3b;
    double* th = theta + ((size_t)k * nc + ci) * 8;
    th[0] = fb(pn, phi, M.delta, f0a, f0b);
    th[1] = fb(pn, scn, M.delta, f1a, f1b);
    th[2] = fb(pn, slc, M.delta, f2a, f2b);
    th[3] = fb(ga, rho, M.delta, f3a, f3b);
    th[4] = -pn;
    th[5] = -phi;
    th[6] = -ga;
    th[7] = -rho;
    chk += th[0] + th[1] + th[2] + th[3] + rho + phi;
    if (dtheta) {
      // derivatives of the pair arguments in the local variables
      // (0 p_x, 1 p_y, 2 theta, 3 v_x+, 4 v_y+, 5 w+, 6 v_x-, 7 v_y-, 8 w-, 9 Phi_t, 10 Phi_n, 11 Gamma),
      // with dx_c = dp_x - r_y dtheta, dy_c = dp_y + r_x dtheta:
      //   phi: phi_x dx_c + phi_y dy_c
      //   cn = n . V: (dn/dx) . V dx_c + n . dV,  V = v_c+ + e v_c-
      //   lc = t . v_c+ + Gamma gn: (dt/dx) . v_c+ dx_c + t . dv_c+ + ...
      //   dv_c/dtheta = (-w r_x, -w r_y), dv_c/dw = (-r_y, r_x)
      constexpr int NT = CISCVX_NODE_THETA_COLS;
      double* D = dtheta + ((size_t)k * nc + ci) * 8 * NT;
      for (int q = 0; q < 8 * NT; ++q) D[q] = 0.0;
      const double phx = FRV(ci, FR_PHIX), phy = FRV(ci, FR_PHIY);
      const double dndx_V = fma(FRV(ci, FR_DNX), Vx, FRV(ci, FR_DNY) * Vy);
      const double dtdx_v = fma(FRV(ci, FR_DTX), vxp, FRV(ci, FR_DTY) * vyp);
      // argument derivatives: [px, py, theta]
      const double dphi[3] = {phx, phy, fma(-phx, ry, phy * rx)};
      const double dcn_x = dndx_V, dlc_x = dtdx_v;
      // theta: through x_c and through the lever arms of both velocities
      const double dcn_th = fma(-ry, dcn_x, -(wp + e * wm) * fma(nx, rx, ny * ry));
      const double dlc_th = fma(-ry, dlc_x, -wp * fma(tx, rx, ty * ry));
      const double dlc_pt = ga / (sq * sq * sq);
      const double c1 = f1b * dcn, c2 = f2b * dlc;
      // row 0: FB(Phi_n, phi)
      D[0 * NT + 10] = f0a;
      D[0 * NT + 0] = f0b * dphi[0]; D[0 * NT + 1] = f0b * dphi[1]; D[0 * NT + 2] = f0b * dphi[2];
      // row 1: FB(Phi_n, |cn|~)
      D[1 * NT + 10] = f1a;
      D[1 * NT + 0] = c1 * dcn_x; D[1 * NT + 2] = c1 * dcn_th;
      D[1 * NT + 3] = c1 * nx; D[1 * NT + 4] = c1 * ny; D[1 * NT + 5] = c1 * fma(-nx, ry, ny * rx);
      D[1 * NT + 6] = c1 * e * nx; D[1 * NT + 7] = c1 * e * ny; D[1 * NT + 8] = c1 * e * fma(-nx, ry, ny * rx);
      // row 2: FB(Phi_n, |lc|~)
      D[2 * NT + 10] = f2a;
      D[2 * NT + 0] = c2 * dlc_x; D[2 * NT + 2] = c2 * dlc_th;
      D[2 * NT + 3] = c2 * tx; D[2 * NT + 4] = c2 * ty; D[2 * NT + 5] = c2 * fma(-tx, ry, ty * rx);
      D[2 * NT + 9] = c2 * dlc_pt; D[2 * NT + 11] = c2 * gn;
      // row 3: FB(Gamma, rho)
      D[3 * NT + 11] = f3a; D[3 * NT + 9] = -f3b * dpt; D[3 * NT + 10] = f3b * mu * dmn;
      D[4 * NT + 10] = -1.0;
      D[5 * NT + 0] = -dphi[0]; D[5 * NT + 1] = -dphi[1]; D[5 * NT + 2] = -dphi[2];
      D[6 * NT + 11] = -1.0;
      D[7 * NT + 9] = dpt; D[7 * NT + 10] = -mu * dmn;
    }
  }
  if (!isfinite(chk)) atomicOr(status, ST_NONFINITE);
}

#undef FRV
#undef LK
#undef SM

}  // namespace

size_t node_smem_per_warp(const DevModel& M) {
  return (size_t)node_layout(M.nb, M.nj, M.nc, M.noff[2 * M.nj], M.ta != 0.0).total * 32 * sizeof(double);
}

cudaError_t launch_node(const DevModel& Mh, const DevModel* dM, int n, const double* Xp,
                        const double* Xm, const double* Phi, const double* Gam,
                        const NodeParams& P, double* g, double* Gvm, double* Gth, double* Gphi,
                        double* Gpx, double* theta, double* dtheta, unsigned* status,
                        cudaStream_t st) {
  const size_t per_warp = node_smem_per_warp(Mh);
  const size_t budget = 220u * 1024u;  // one CTA per SM, as many warps as fit (<= 8)
  int wpc = (int)std::min<size_t>(8, std::max<size_t>(1, budget / per_warp));
  const long warps = (n + 31) / 32;
  if (warps < wpc) wpc = (int)std::max<long>(1, warps);
  const size_t smem = per_warp * wpc;
  cudaError_t e = cudaSuccess;
  if (smem > 48u * 1024u)
    e = cudaFuncSetAttribute(k_node, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = 32 * wpc;
  const long blocks = (n + threads - 1) / threads;
  NodeTab T;
  std::memset(&T, 0, sizeof T);
  T.nb = Mh.nb; T.nj = Mh.nj; T.nc = Mh.nc; T.nxt = Mh.nxt;
  for (int b = 0; b < Mh.nb; ++b) {
    T.nadj[b] = Mh.nadj[b];
    for (int t = 0; t < Mh.nadj[b]; ++t) T.adj[b][t] = (unsigned char)Mh.adj[b][t];
    T.lmin[b] = Mh.lmin[b];
    T.contact[b] = Mh.body[b].contact;
    T.mass[b] = Mh.mass[b]; T.inertia[b] = Mh.inertia[b];
    T.minv[b] = Mh.minv[b]; T.iinv[b] = Mh.iinv[b];
    T.crho[b][0] = Mh.body[b].crho[0]; T.crho[b][1] = Mh.body[b].crho[1];
    T.mu[b] = Mh.body[b].mu;
  }
  for (int j = 0; j < Mh.nj; ++j) {
    T.npos[j] = Mh.npos[j]; T.nord[j] = Mh.nord[j];
    T.jchi[j] = Mh.jchi[j]; T.jpar[j] = Mh.jpar[j];
    T.jrc[j][0] = Mh.jrc[j][0]; T.jrc[j][1] = Mh.jrc[j][1];
    T.jrp[j][0] = Mh.jrp[j][0]; T.jrp[j][1] = Mh.jrp[j][1];
  }
  for (int i = 0; i <= 2 * Mh.nj; ++i) {
    if (i < 2 * Mh.nj) T.nf[i] = Mh.nf[i];
    T.noff[i] = Mh.noff[i];
  }
  T.delta = P.delta;
  T.ta = Mh.ta;
  T.tk = Mh.tk;
  for (int i = 0; i < Mh.nc; ++i) T.e[i] = P.e[i];
  k_node<<<(unsigned)blocks, threads, smem, st>>>(T, n, Xp, Xm, Phi, Gam, g, Gvm, Gth, Gphi, Gpx,
                                                  theta, dtheta, status);
  return cudaGetLastError();
}

}  // namespace ciscvx
