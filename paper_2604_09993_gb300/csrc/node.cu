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
//
// Mapping: lane = node.  The joint impulse couples every link of a node, so
// one thread owns one node; a warp's 32 lanes run the same program on 32
// nodes of one model, so no FP64 instruction runs partly masked.  K's
// Cholesky factor and the per-node vectors sit in shared memory, element
// major ([element][lane]), so a warp's access to one element is one
// contiguous 256-byte row.  FP64 throughout (the state precision).
#include <algorithm>

#include "common.cuh"

namespace ciscvx {

namespace {

// Per-lane scratch layout (in doubles; each element is a row of 32 lanes).
struct NodeLayout {
  int cs, arm, K, dinv, v, mu, x, col, total;
};

__host__ __device__ inline NodeLayout node_layout(int nb, int nj) {
  const int nk = 2 * nj;
  NodeLayout L;
  L.cs = 0;                        // cos, sin of every link angle           (2 nb)
  L.arm = L.cs + 2 * nb;           // perp lever arms (child x,y; parent x,y) (4 nj)
  L.K = L.arm + 4 * nj;            // packed lower Cholesky factor of K       (nk(nk+1)/2)
  L.dinv = L.K + nk * (nk + 1) / 2;  // reciprocal diagonal of the factor    (nk)
  L.v = L.dinv + nk;               // w, then the implied post-impact v^      (3 nb)
  L.mu = L.v + 3 * nb;             // mu = K^-1 C' w                          (nk)
  L.x = L.mu + nk;                 // solve right-hand side / solution        (nk)
  L.col = L.x + nk;                // output column accumulator               (3 nb)
  L.total = L.col + 3 * nb;
  return L;
}

__device__ __forceinline__ int tri(int i, int k) { return i * (i + 1) / 2 + k; }

// Solves K x = x in place (the factor is L L^T, L packed with reciprocal diagonal).
__device__ __forceinline__ void chol_solve(double* sm, const NodeLayout& Ly, int nk) {
#define SM(e) sm[(e) * 32]
  for (int i = 0; i < nk; ++i) {
    double acc = SM(Ly.x + i);
    for (int k = 0; k < i; ++k) acc = fma(-SM(Ly.K + tri(i, k)), SM(Ly.x + k), acc);
    SM(Ly.x + i) = acc * SM(Ly.dinv + i);
  }
  for (int i = nk - 1; i >= 0; --i) {
    double acc = SM(Ly.x + i);
    for (int k = i + 1; k < nk; ++k) acc = fma(-SM(Ly.K + tri(k, i)), SM(Ly.x + k), acc);
    SM(Ly.x + i) = acc * SM(Ly.dinv + i);
  }
#undef SM
}

// col = C'^T x (3 nb), from the solution in x.
__device__ __forceinline__ void ct_times_x(const DevModel& M, double* sm, const NodeLayout& Ly) {
#define SM(e) sm[(e) * 32]
  const int nb = M.nb, nj = M.nj;
  for (int a = 0; a < 3 * nb; ++a) SM(Ly.col + a) = 0.0;
  for (int j = 0; j < nj; ++j) {
    const double x0 = SM(Ly.x + 2 * j), x1 = SM(Ly.x + 2 * j + 1);
    const int c = M.jchi[j], p = M.jpar[j];
    SM(Ly.col + 3 * c) += x0;
    SM(Ly.col + 3 * c + 1) += x1;
    SM(Ly.col + 3 * c + 2) = fma(SM(Ly.arm + 4 * j), x0, fma(SM(Ly.arm + 4 * j + 1), x1, SM(Ly.col + 3 * c + 2)));
    SM(Ly.col + 3 * p) -= x0;
    SM(Ly.col + 3 * p + 1) -= x1;
    SM(Ly.col + 3 * p + 2) = fma(-SM(Ly.arm + 4 * j + 2), x0, fma(-SM(Ly.arm + 4 * j + 3), x1, SM(Ly.col + 3 * p + 2)));
  }
#undef SM
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

__global__ void __launch_bounds__(128) k_node(const DevModel* __restrict__ Mp, int n,
                                              const double* __restrict__ Xp,
                                              const double* __restrict__ Xm,
                                              const double* __restrict__ Phi,
                                              const double* __restrict__ Gam, NodeParams P,
                                              double* g, double* Gvm, double* Gth, double* Gphi,
                                              double* theta, double* dtheta, unsigned* status) {
  extern __shared__ double smem[];
  const DevModel& M = *Mp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int nb = M.nb, nj = M.nj, nc = M.nc, nxt = M.nxt, nq = 3 * nb, nk = 2 * nj;
  const NodeLayout Ly = node_layout(nb, nj);
  double* sm = smem + (size_t)warp * Ly.total * 32 + lane;
#define SM(e) sm[(e) * 32]
  const double* xp = Xp + k * nxt;
  const double* xm = Xm + k * nxt;
  const double* ph = Phi ? Phi + k * 2 * nc : nullptr;
  const double* gm = Gam ? Gam + k * nc : nullptr;
  double chk = 0.0;

  // link angles, joint lever arms (as perp(r) = d(R rho)/dtheta)
  for (int b = 0; b < nb; ++b) {
    double s, c;
    sincos(xm[3 * b + 2], &s, &c);
    SM(Ly.cs + 2 * b) = c;
    SM(Ly.cs + 2 * b + 1) = s;
  }
  for (int j = 0; j < nj; ++j) {
    const int cb = M.jchi[j], pb = M.jpar[j];
    const double cc = SM(Ly.cs + 2 * cb), sc = SM(Ly.cs + 2 * cb + 1);
    const double cp = SM(Ly.cs + 2 * pb), sp = SM(Ly.cs + 2 * pb + 1);
    const double rcx = cc * M.jrc[j][0] - sc * M.jrc[j][1], rcy = sc * M.jrc[j][0] + cc * M.jrc[j][1];
    const double rpx = cp * M.jrp[j][0] - sp * M.jrp[j][1], rpy = sp * M.jrp[j][0] + cp * M.jrp[j][1];
    SM(Ly.arm + 4 * j) = -rcy;
    SM(Ly.arm + 4 * j + 1) = rcx;
    SM(Ly.arm + 4 * j + 2) = -rpy;
    SM(Ly.arm + 4 * j + 3) = rpx;
  }

  // K = C' M^-1 C'^T and its Cholesky factor (packed lower, reciprocal diagonal)
  for (int r1 = 0; r1 < nk; ++r1) {
    const int j1 = r1 >> 1, a1 = r1 & 1;
    for (int r2 = 0; r2 <= r1; ++r2) {
      const int j2 = r2 >> 1, a2 = r2 & 1;
      double acc = 0.0;
      for (int u = 0; u < 2; ++u) {
        const int b1 = u ? M.jpar[j1] : M.jchi[j1];
        const double p1 = SM(Ly.arm + 4 * j1 + 2 * u + a1);
        for (int v = 0; v < 2; ++v) {
          const int b2 = v ? M.jpar[j2] : M.jchi[j2];
          if (b1 != b2) continue;
          const double p2 = SM(Ly.arm + 4 * j2 + 2 * v + a2);
          double e = p1 * p2 * M.iinv[b1];
          if (a1 == a2) e += M.minv[b1];
          acc += (u == v) ? e : -e;
        }
      }
      SM(Ly.K + tri(r1, r2)) = acc;
    }
  }
  for (int i = 0; i < nk; ++i) {
    double d = SM(Ly.K + tri(i, i));
    for (int kk = 0; kk < i; ++kk) d = fma(-SM(Ly.K + tri(i, kk)), SM(Ly.K + tri(i, kk)), d);
    const double di = 1.0 / sqrt(d);
    SM(Ly.dinv + i) = di;
    SM(Ly.K + tri(i, i)) = d * di;
    for (int jrow = i + 1; jrow < nk; ++jrow) {
      double acc = SM(Ly.K + tri(jrow, i));
      for (int kk = 0; kk < i; ++kk) acc = fma(-SM(Ly.K + tri(jrow, kk)), SM(Ly.K + tri(i, kk)), acc);
      SM(Ly.K + tri(jrow, i)) = acc * di;
    }
  }

  // w = v- + M^-1 J_c^T Phi
  for (int a = 0; a < nq; ++a) SM(Ly.v + a) = xm[nq + a];
  for (int b = 0; b < nb; ++b) {
    const int ci = M.body[b].contact;
    if (ci < 0) continue;
    const double c = SM(Ly.cs + 2 * b), s = SM(Ly.cs + 2 * b + 1);
    const double rx = c * M.body[b].crho[0] - s * M.body[b].crho[1];
    const double ry = s * M.body[b].crho[0] + c * M.body[b].crho[1];
    const double pt = ph[2 * ci], pn = ph[2 * ci + 1];
    SM(Ly.v + 3 * b) += pt * M.minv[b];
    SM(Ly.v + 3 * b + 1) += pn * M.minv[b];
    SM(Ly.v + 3 * b + 2) += (rx * pn - ry * pt) * M.iinv[b];
  }
  // mu = K^-1 C' w
  for (int j = 0; j < nj; ++j) {
    const int cb = M.jchi[j], pb = M.jpar[j];
    for (int a = 0; a < 2; ++a)
      SM(Ly.x + 2 * j + a) = fma(SM(Ly.arm + 4 * j + a), SM(Ly.v + 3 * cb + 2), SM(Ly.v + 3 * cb + a)) -
                             fma(SM(Ly.arm + 4 * j + 2 + a), SM(Ly.v + 3 * pb + 2), SM(Ly.v + 3 * pb + a));
  }
  chol_solve(sm, Ly, nk);
  for (int r = 0; r < nk; ++r) SM(Ly.mu + r) = SM(Ly.x + r);
  ct_times_x(M, sm, Ly);  // col = C'^T mu

  // residual G~; v^ = w - M^-1 C'^T mu
  double* gk = g + k * nxt;
  for (int a = 0; a < nq; ++a) gk[a] = xp[a] - xm[a];
  for (int b = 0; b < nb; ++b) {
    for (int a = 0; a < 3; ++a) {
      const int r = 3 * b + a;
      const double mm = (a < 2) ? M.mass[b] : M.inertia[b];
      const double mi = (a < 2) ? M.minv[b] : M.iinv[b];
      double f = 0.0;  // J_c^T Phi on this coordinate
      const int ci = M.body[b].contact;
      if (ci >= 0) {
        const double c = SM(Ly.cs + 2 * b), s = SM(Ly.cs + 2 * b + 1);
        const double rx = c * M.body[b].crho[0] - s * M.body[b].crho[1];
        const double ry = s * M.body[b].crho[0] + c * M.body[b].crho[1];
        const double pt = ph[2 * ci], pn = ph[2 * ci + 1];
        f = (a == 0) ? pt : (a == 1 ? pn : rx * pn - ry * pt);
      }
      const double gv = mm * (xp[nq + r] - xm[nq + r]) - f + SM(Ly.col + r);
      gk[nq + r] = gv;
      chk += gv;
      SM(Ly.v + r) = fma(-SM(Ly.col + r), mi, SM(Ly.v + r));
    }
  }
  for (int i = 0; i < nc; ++i) gk[2 * nq + i] = xp[2 * nq + i] - xm[2 * nq + i];

  // d/dv-: column c = -M e_c + C'^T K^-1 C' e_c (written as row c: the block is symmetric)
  if (Gvm) {
    double* out = Gvm + (size_t)k * nq * nq;
    for (int c = 0; c < nq; ++c) {
      const int bc = c / 3, comp = c - 3 * bc;
      for (int j = 0; j < nj; ++j) {
        for (int a = 0; a < 2; ++a) {
          double e = 0.0;
          if (M.jchi[j] == bc) e += (comp < 2) ? (comp == a ? 1.0 : 0.0) : SM(Ly.arm + 4 * j + a);
          if (M.jpar[j] == bc) e -= (comp < 2) ? (comp == a ? 1.0 : 0.0) : SM(Ly.arm + 4 * j + 2 + a);
          SM(Ly.x + 2 * j + a) = e;
        }
      }
      chol_solve(sm, Ly, nk);
      ct_times_x(M, sm, Ly);
      const double mc = (comp < 2) ? M.mass[bc] : M.inertia[bc];
      for (int r = 0; r < nq; ++r) {
        const double v = SM(Ly.col + r) - (r == c ? mc : 0.0);
        out[(size_t)c * nq + r] = v;
        chk += v;
      }
    }
  }

  // d/dtheta_b
  if (Gth) {
    double* out = Gth + (size_t)k * nq * nb;
    for (int b = 0; b < nb; ++b) {
      // a_b = -sum_i r_i . Phi_i + sum_j s_jb r_jb . mu_j  (r = R rho; perp(r) stored)
      double ab = 0.0;
      const int ci = M.body[b].contact;
      if (ci >= 0) {
        const double c = SM(Ly.cs + 2 * b), s = SM(Ly.cs + 2 * b + 1);
        const double rx = c * M.body[b].crho[0] - s * M.body[b].crho[1];
        const double ry = s * M.body[b].crho[0] + c * M.body[b].crho[1];
        ab -= rx * ph[2 * ci] + ry * ph[2 * ci + 1];
      }
      for (int j = 0; j < nj; ++j) {
        // r = (perp_y, -perp_x)
        if (M.jchi[j] == b)
          ab += SM(Ly.arm + 4 * j + 1) * SM(Ly.mu + 2 * j) - SM(Ly.arm + 4 * j) * SM(Ly.mu + 2 * j + 1);
        if (M.jpar[j] == b)
          ab -= SM(Ly.arm + 4 * j + 3) * SM(Ly.mu + 2 * j) - SM(Ly.arm + 4 * j + 2) * SM(Ly.mu + 2 * j + 1);
      }
      const double wb = SM(Ly.v + 3 * b + 2), ai = ab * M.iinv[b];
      for (int j = 0; j < nj; ++j) {
        double t0 = 0.0, t1 = 0.0;
        if (M.jchi[j] == b) {
          const double px = SM(Ly.arm + 4 * j), py = SM(Ly.arm + 4 * j + 1);  // r = (py, -px)
          t0 += -py * wb + px * ai;
          t1 += px * wb + py * ai;
        }
        if (M.jpar[j] == b) {
          const double px = SM(Ly.arm + 4 * j + 2), py = SM(Ly.arm + 4 * j + 3);
          t0 -= -py * wb + px * ai;
          t1 -= px * wb + py * ai;
        }
        SM(Ly.x + 2 * j) = t0;
        SM(Ly.x + 2 * j + 1) = t1;
      }
      chol_solve(sm, Ly, nk);
      ct_times_x(M, sm, Ly);
      for (int r = 0; r < nq; ++r) {
        const double v = SM(Ly.col + r) - (r == 3 * b + 2 ? ab : 0.0);
        out[(size_t)r * nb + b] = v;
        chk += v;
      }
    }
  }

  // d/dPhi: column = -f + C'^T K^-1 C' M^-1 f,  f = J_c^T e
  if (Gphi && nc > 0) {
    double* out = Gphi + (size_t)k * nq * 2 * nc;
    for (int b = 0; b < nb; ++b) {
      const int ci = M.body[b].contact;
      if (ci < 0) continue;
      const double c = SM(Ly.cs + 2 * b), s = SM(Ly.cs + 2 * b + 1);
      const double rx = c * M.body[b].crho[0] - s * M.body[b].crho[1];
      const double ry = s * M.body[b].crho[0] + c * M.body[b].crho[1];
      for (int comp = 0; comp < 2; ++comp) {
        const double f0 = (comp == 0) ? 1.0 : 0.0, f1 = (comp == 1) ? 1.0 : 0.0;
        const double f2 = (comp == 0) ? -ry : rx;
        const double g0 = f0 * M.minv[b], g1 = f1 * M.minv[b], g2 = f2 * M.iinv[b];
        for (int j = 0; j < nj; ++j) {
          for (int a = 0; a < 2; ++a) {
            double e = 0.0;
            const double ga = a ? g1 : g0;
            if (M.jchi[j] == b) e += ga + SM(Ly.arm + 4 * j + a) * g2;
            if (M.jpar[j] == b) e -= ga + SM(Ly.arm + 4 * j + 2 + a) * g2;
            SM(Ly.x + 2 * j + a) = e;
          }
        }
        chol_solve(sm, Ly, nk);
        ct_times_x(M, sm, Ly);
        const int col = 2 * ci + comp;
        for (int r = 0; r < nq; ++r) {
          double v = SM(Ly.col + r);
          if (r == 3 * b) v -= f0;
          else if (r == 3 * b + 1) v -= f1;
          else if (r == 3 * b + 2) v -= f2;
          out[(size_t)r * 2 * nc + col] = v;
          chk += v;
        }
      }
    }
  }

  // Theta^delta per contact, and its Jacobian in the contact's local variables
  // (p_y-, theta-, v_x+, v_y+, omega+, v_y-, omega-, Phi_t, Phi_n, Gamma) of its link.
  if (nc > 0) {
    for (int b = 0; b < nb; ++b) {
      const int ci = M.body[b].contact;
      if (ci < 0) continue;
      const double c = SM(Ly.cs + 2 * b), s = SM(Ly.cs + 2 * b + 1);
      const double rx = c * M.body[b].crho[0] - s * M.body[b].crho[1];
      const double ry = s * M.body[b].crho[0] + c * M.body[b].crho[1];
      const double pt = ph[2 * ci], pn = ph[2 * ci + 1], ga = gm[ci], e = P.e[ci];
      const double mu = M.body[b].mu;
      const double wp = xp[nq + 3 * b + 2], wm = xm[nq + 3 * b + 2];
      const double phi = xm[3 * b + 1] + ry;
      const double vtp = xp[nq + 3 * b] - wp * ry;
      const double vnp = xp[nq + 3 * b + 1] + wp * rx;
      const double vnm = xm[nq + 3 * b + 1] + wm * rx;
      const double cn = fma(e, vnm, vnp);
      const double sq = sqrt(fma(pt, pt, 1.0));
      const double gn = pt / sq;
      const double lc = fma(ga, gn, vtp);
      double dcn, dlc, dmn, dpt;
      const double scn = sabs(cn, dcn), slc = sabs(lc, dlc);
      const double smn = sabs(mu * pn, dmn), spt = sabs(pt, dpt);
      const double rho = smn - spt;
      double f0a, f0b, f1a, f1b, f2a, f2b, f3a, f3b;
      double* th = theta + ((size_t)k * nc + ci) * 8;
      th[0] = fb(pn, phi, P.delta, f0a, f0b);
      th[1] = fb(pn, scn, P.delta, f1a, f1b);
      th[2] = fb(pn, slc, P.delta, f2a, f2b);
      th[3] = fb(ga, rho, P.delta, f3a, f3b);
      th[4] = -pn;
      th[5] = -phi;
      th[6] = -ga;
      th[7] = -rho;
      chk += th[0] + th[1] + th[2] + th[3] + rho + phi;
      if (dtheta) {
        // derivatives of the pair arguments in the local variables:
        //   phi: p_y 1, theta r_x
        //   cn:  theta -(w+ + e w-) r_y, v_y+ 1, w+ r_x, v_y- e, w- e r_x
        //   lc:  theta -w+ r_x, v_x+ 1, w+ -r_y, Phi_t Gamma / sq^3, Gamma gn
        //   rho: Phi_t -dpt, Phi_n mu dmn
        double* D = dtheta + ((size_t)k * nc + ci) * 80;
        for (int q = 0; q < 80; ++q) D[q] = 0.0;
        const double dcn_th = -(wp + e * wm) * ry, dlc_th = -wp * rx;
        const double dlc_pt = ga / (sq * sq * sq);
        const double c1 = f1b * dcn, c2 = f2b * dlc;
        D[0 * 10 + 8] = f0a; D[0 * 10 + 0] = f0b; D[0 * 10 + 1] = f0b * rx;
        D[1 * 10 + 8] = f1a;
        D[1 * 10 + 1] = c1 * dcn_th; D[1 * 10 + 3] = c1; D[1 * 10 + 4] = c1 * rx;
        D[1 * 10 + 5] = c1 * e; D[1 * 10 + 6] = c1 * e * rx;
        D[2 * 10 + 8] = f2a;
        D[2 * 10 + 1] = c2 * dlc_th; D[2 * 10 + 2] = c2; D[2 * 10 + 4] = -c2 * ry;
        D[2 * 10 + 7] = c2 * dlc_pt; D[2 * 10 + 9] = c2 * gn;
        D[3 * 10 + 9] = f3a; D[3 * 10 + 7] = -f3b * dpt; D[3 * 10 + 8] = f3b * mu * dmn;
        D[4 * 10 + 8] = -1.0;
        D[5 * 10 + 0] = -1.0; D[5 * 10 + 1] = -rx;
        D[6 * 10 + 9] = -1.0;
        D[7 * 10 + 7] = dpt; D[7 * 10 + 8] = -mu * dmn;
      }
    }
  }
  if (!isfinite(chk)) atomicOr(status, ST_NONFINITE);
#undef SM
}

}  // namespace

size_t node_smem_per_warp(const DevModel& M) {
  return (size_t)node_layout(M.nb, M.nj).total * 32 * sizeof(double);
}

cudaError_t launch_node(const DevModel& Mh, const DevModel* dM, int n, const double* Xp,
                        const double* Xm, const double* Phi, const double* Gam,
                        const NodeParams& P, double* g, double* Gvm, double* Gth, double* Gphi,
                        double* theta, double* dtheta, unsigned* status, cudaStream_t st) {
  const size_t per_warp = node_smem_per_warp(Mh);
  const size_t budget = 200u * 1024u;
  int wpc = (int)std::min<size_t>(4, std::max<size_t>(1, budget / per_warp));
  const long warps = (n + 31) / 32;
  if (warps < wpc) wpc = (int)std::max<long>(1, warps);
  const size_t smem = per_warp * wpc;
  cudaError_t e = cudaSuccess;
  if (smem > 48u * 1024u)
    e = cudaFuncSetAttribute(k_node, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = 32 * wpc;
  const long blocks = (n + threads - 1) / threads;
  k_node<<<(unsigned)blocks, threads, smem, st>>>(dM, n, Xp, Xm, Phi, Gam, P, g, Gvm, Gth, Gphi,
                                                  theta, dtheta, status);
  return cudaGetLastError();
}

}  // namespace ciscvx
