// oracle.cpp — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow FP64 CPU implementation of the CI-SCvx per-interval
// discretization/linearization (Buckner & Elango, "GPU-Accelerated
// Continuous-Time Successive Convexification for Contact-Implicit Legged
// Locomotion").  It exists to check the CUDA library against.  Only tests/,
// __graft_entry__.smoke() and bench.py (its CPU-baseline and reference legs)
// may load it; the product package never links, imports or calls it, and it
// shares no code, header or table with the product.
//
// What is computed, and where it comes from:
//   rhs()       the augmented right-hand side (f, Omega): Newton-Euler per
//               link in maximal coordinates, Sec. II-A Eq. (1), with the joint
//               reaction forces either as inputs or eliminated at the
//               acceleration level (Eq. (3), eliminated_accel()); contact
//               frame and signed distance on flat ground y = 0 or on the
//               sinusoidal surface of Sec. VI-B (contact_frame());
//               integral path-constraint penalty Omega = M^g sabs+(g), Sec. IV-A
//               Eq. (12), with one auxiliary state per contact — or, for the
//               aux model 1, the full Eq. (12): four cross-complementarity
//               states per contact (phi_n, lambda^c, gamma, rho^c) before the
//               path-penalty states, with contact inputs (phi_t, phi_n, gamma).
//   rk_foh()    the time-dilated augmented system d x~/d tau = s (f, Omega) on
//               tau in [0,1], Sec. IV-B Eq. (14), integrated in integral form
//               Eq. (15) with a first-order-hold control u(tau) =
//               (1 - tau) u_L + tau u_R (Sec. VI: FOH), by n_sub fixed steps
//               of classical RK4 or of the Runge-Kutta-Fehlberg 4(5) pair
//               (Sec. VI), given by their Butcher tableaux.
//   interval()  Internal Numerical Differentiation (Sec. VI): the Jacobian of
//               the discrete RK4 map is obtained by running the very same RK4
//               arithmetic on forward-mode dual numbers seeded in
//               (x~_k, u_L, u_R, s).  Outputs A = dF/dx~, B- = dF/du_L,
//               B+ = dF/du_R, S = dF/ds.
//   discretize() every interval k of the multiple-shooting grid, independently:
//               defect_k = F~(x~_k, U_k, s_k) - x~_{k+1} (Eq. (17b)) and
//               penalty_k = y(1) - y_k (the increments that Eq. (13) bounds).
//   vjp()       gradient of L = sum_k w_k . defect_k + sum_k rho_k . penalty_k
//               contracted from the IND blocks (J^T times the cotangent).
//   linear_interval()  the same integrator and IND applied to a linear
//               right-hand side A_c x + B_c u (used only to pin the integrator).
//   node()      the node constraints of Eqs. (17e)-(17f): the impact map G~
//               (Eq. (6a) with the joint impulse eliminated, Sec. II-B) and the
//               Fischer-Burmeister-relaxed impulse conditions Theta^delta
//               (Eqs. (6b)-(6e), (16)), with Jacobians by dual numbers.
//   psi()       Psi^{delta,eps}(y-_{k+1}, y+_k) <= 0 of Eq. (17c) on every
//               interval: Fischer-Burmeister-relaxed (Eq. (16)) integral
//               cross-complementarity of the auxiliary-state increments
//               (Eq. (11) applied to the pairs of Eq. (12)) and the relaxed
//               path-constraint rows of Eq. (13), with Jacobians by dual numbers.
//
// Readings of points the paper leaves open (one auxiliary state per contact,
// pseudo-Huber ramp h(z) = sqrt(1 + max(z,0)^2) - 1, joint reaction forces and
// contact forces (lambda_n, lambda_t+, lambda_t-) as FOH inputs by default,
// N intervals on N+1 nodes, classical RK4 by default, the RKF step advanced
// with the fifth-order weights, the contact normal n = grad h^c / ||grad h^c||
// off the surface) are listed in the project's design notes; this file
// follows them.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -pthread oracle.cpp -o liboracle.so

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers with a run-time number of tangent directions.
// ---------------------------------------------------------------------------
constexpr int MAXC = 400;   // max tangent directions (n_x~ + 2 n_u + 1; 393 for a 32-link chain)
thread_local int g_nd = 0;  // active directions for this thread

struct Dual {
  double v;
  double d[MAXC];
  Dual() : v(0.0) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }  // NOLINT
};

inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v + b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v - b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r; r.v = -a.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = -a.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v * b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.v * b.d[i] + b.v * a.d[i];
  return r;
}
inline Dual operator*(double a, const Dual& b) {
  Dual r; r.v = a * b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a * b.d[i];
  return r;
}
inline Dual operator*(const Dual& a, double b) { return b * a; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v / b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
inline Dual operator/(const Dual& a, double b) {
  Dual r; r.v = a.v / b;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] / b;
  return r;
}
inline Dual operator+(double a, const Dual& b) { Dual r = b; r.v += a; return r; }
inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
inline Dual operator-(double a, const Dual& b) { Dual r = -b; r.v += a; return r; }

inline Dual sin(const Dual& a) {
  Dual r; r.v = std::sin(a.v);
  const double c = std::cos(a.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = c * a.d[i];
  return r;
}
inline Dual cos(const Dual& a) {
  Dual r; r.v = std::cos(a.v);
  const double s = -std::sin(a.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = s * a.d[i];
  return r;
}
inline Dual sqrt(const Dual& a) {
  Dual r; r.v = std::sqrt(a.v);
  const double k = 0.5 / r.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = k * a.d[i];
  return r;
}
inline double value(const Dual& a) { return a.v; }

inline double sin(double a) { return std::sin(a); }
inline double cos(double a) { return std::cos(a); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double value(double a) { return a; }

// ramp max(z, 0) (Sec. II notation); derivative 0 for z <= 0.
template <class T> T ramp(const T& z) { return value(z) > 0.0 ? z : T(0.0); }

// Pseudo-Huber ramp with unit steepness, h(z) = sqrt(1 + max(z,0)^2) - 1,
// written as p^2 / (1 + sqrt(1 + p^2)) with p = max(z,0), which is the same
// number without the cancellation near p = 0.  h = 0 exactly for z <= 0, as
// the CTCS condition y_{k+1} = y_k needs (Sec. IV-A).
template <class T> T sabs_plus(const T& z) {
  const T p = ramp(z);
  return (p * p) / (1.0 + sqrt(1.0 + p * p));
}

// Pseudo-Huber absolute value / norm with unit steepness (Sec. II notation):
// sqrt(1 + x^2) - 1 (in the plane the tangential force or impulse is a
// scalar, so the smooth norm and the smooth absolute value are the same
// function).
template <class T> T smooth_abs(const T& x) { return sqrt(1.0 + x * x) - 1.0; }

}  // namespace

// ---------------------------------------------------------------------------
// Model description (the oracle's own layout; filled in from Python).
// ---------------------------------------------------------------------------
extern "C" {
typedef struct {
  int nb, nj, nc;
  const double* mass;     // [nb]
  const double* inertia;  // [nb]  rotational inertia about the centre of mass
  const int* jparent;     // [nj]
  const int* jchild;      // [nj]
  const double* jrho_p;   // [nj][2] joint anchor in the parent body frame
  const double* jrho_c;   // [nj][2] joint anchor in the child body frame
  const int* cbody;       // [nc]
  const double* crho;     // [nc][2] contact point in the body frame
  const double* cmu;      // [nc] friction coefficient
  double g;               // gravity magnitude, acting along -y
  int aux;                // 0: one path-penalty state per contact, forces (lambda_n, lambda_t+, lambda_t-);
                          // 1: Eq. (12): four cross-complementarity states + one path-penalty
                          //    state per contact, forces (phi_t, phi_n) and multiplier gamma
  int jelim;              // 0: joint reaction forces are inputs; 1: eliminated at the
                          //    acceleration level, Eq. (3) (inputs: joint torques and contact inputs)
  int scheme;             // 0: classical RK4; 1: Runge-Kutta-Fehlberg 4(5), fifth-order weights
  double terrain_amp;     // contact surface y = terrain_amp sin(terrain_k x) (0: flat ground y = 0)
  double terrain_k;
} OracleModel;
}

namespace {

int nx_of(const OracleModel& M) { return 6 * M.nb; }
int nxt_of(const OracleModel& M) { return 6 * M.nb + (M.aux ? 5 : 1) * M.nc; }
// first path-penalty state (the states Eq. (13) bounds)
int pen_of(const OracleModel& M) { return 6 * M.nb + (M.aux ? 4 * M.nc : 0); }
int nu_of(const OracleModel& M) { return (M.jelim ? 1 : 3) * M.nj + 3 * M.nc; }

// World-frame lever arm r = R(theta) rho, R = [[cos, -sin], [sin, cos]].
template <class T>
void lever_arm(const T& theta, const double* rho, T& rx, T& ry) {
  const T c = cos(theta), s = sin(theta);
  rx = c * rho[0] - s * rho[1];
  ry = s * rho[0] + c * rho[1];
}

// Planar cross product r x F = r_x F_y - r_y F_x.
template <class T>
T cross2(const T& rx, const T& ry, const T& fx, const T& fy) { return rx * fy - ry * fx; }

// Solves the dense system K x = r (n x n, row-major, overwritten) by Gaussian
// elimination with partial pivoting on the values.
template <class T> void dense_solve(int n, std::vector<T>& K, std::vector<T>& r) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(value(K[i * n + c])) > std::fabs(value(K[piv * n + c]))) piv = i;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(K[c * n + j], K[piv * n + j]);
      std::swap(r[c], r[piv]);
    }
    for (int i = c + 1; i < n; ++i) {
      const T f = K[i * n + c] / K[c * n + c];
      for (int j = c; j < n; ++j) K[i * n + j] = K[i * n + j] - f * K[c * n + j];
      r[i] = r[i] - f * r[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    T acc = r[c];
    for (int j = c + 1; j < n; ++j) acc = acc - K[c * n + j] * r[j];
    r[c] = acc / K[c * n + c];
  }
}

// Contact surface and contact frame at a world point (p_x, p_y) (Sec. II-A;
// the sinusoidal surface of Sec. VI-B).  The surface is the zero set of
// h^c(p) = p_y - a sin(k p_x) (a = 0: flat ground y = 0).  The signed distance
// is approximated by h^c / ||grad h^c|| (Sec. VI-B), the unit normal is
// n = grad h^c / ||grad h^c|| (grad phi on the surface), and the tangent
// t = (n_y, -n_x) completes the right-handed frame R_c = [t n].
template <class T>
struct Frame {
  T phi, tx, ty, nx, ny;
};

template <class T>
Frame<T> contact_frame(const OracleModel& M, const T& px, const T& py) {
  Frame<T> f;
  if (M.terrain_amp == 0.0) {
    f.phi = py;
    f.tx = T(1.0); f.ty = T(0.0);
    f.nx = T(0.0); f.ny = T(1.0);
    return f;
  }
  const double a = M.terrain_amp, k = M.terrain_k;
  const T hc = py - a * sin(k * px);
  const T gx = -(a * k) * cos(k * px);  // dh^c/dp_x; dh^c/dp_y = 1
  const T inv = 1.0 / sqrt(1.0 + gx * gx);
  f.phi = hc * inv;
  f.nx = gx * inv;
  f.ny = inv;
  f.tx = f.ny;
  f.ty = -f.nx;
  return f;
}

// Generalized accelerations with the joint reaction forces eliminated at the
// acceleration level (Sec. II-A, Eq. (3)).  F = (F_x, F_y, torque) per link
// holds every other generalized force.  The joint constraints
// C_j = p_c + R_c rho_c - p_p - R_p rho_p = 0 differentiated twice give
// grad C v' + (v^T Hess C_j v)_j = 0, and with M v' = F + grad C^T lambda the
// pair (v', lambda) solves
//   [ M        -grad C^T ] [ v'     ]   [ F                      ]
//   [ grad C    0        ] [ lambda ] = [ -(v^T Hess C_j v)_j    ],
// solved here densely.  The only second derivative of C_j is
// d^2 (R rho) / d theta^2 = -R rho, so v^T Hess C_j v = -omega_c^2 r_c + omega_p^2 r_p.
template <class T>
std::vector<T> eliminated_accel(const OracleModel& M, const T* xt, const std::vector<T>& Fx,
                                const std::vector<T>& Fy, const std::vector<T>& Tq) {
  const int nb = M.nb, nj = M.nj, nq = 3 * nb, n = nq + 2 * nj;
  std::vector<T> K((size_t)n * n, T(0.0)), r(n, T(0.0));
  for (int b = 0; b < nb; ++b) {
    K[(size_t)(3 * b) * n + 3 * b] = T(M.mass[b]);
    K[(size_t)(3 * b + 1) * n + 3 * b + 1] = T(M.mass[b]);
    K[(size_t)(3 * b + 2) * n + 3 * b + 2] = T(M.inertia[b]);
    r[3 * b] = Fx[b];
    r[3 * b + 1] = Fy[b];
    r[3 * b + 2] = Tq[b];
  }
  for (int j = 0; j < nj; ++j) {
    const int c = M.jchild[j], p = M.jparent[j];
    T rcx, rcy, rpx, rpy;
    lever_arm(xt[3 * c + 2], M.jrho_c + 2 * j, rcx, rcy);
    lever_arm(xt[3 * p + 2], M.jrho_p + 2 * j, rpx, rpy);
    // grad C_j: +[I, d(R rho_c)/d theta] on the child, -[I, d(R rho_p)/d theta]
    // on the parent, with d(R rho)/d theta = (-r_y, r_x)
    const int row = nq + 2 * j;
    struct E { int r, c; T v; };
    const E ent[8] = {{row, 3 * c, T(1.0)},         {row, 3 * c + 2, -rcy},
                      {row + 1, 3 * c + 1, T(1.0)}, {row + 1, 3 * c + 2, rcx},
                      {row, 3 * p, T(-1.0)},        {row, 3 * p + 2, rpy},
                      {row + 1, 3 * p + 1, T(-1.0)}, {row + 1, 3 * p + 2, -rpx}};
    for (const E& e : ent) {
      K[(size_t)e.r * n + e.c] = K[(size_t)e.r * n + e.c] + e.v;  // grad C
      K[(size_t)e.c * n + e.r] = K[(size_t)e.c * n + e.r] - e.v;  // -grad C^T
    }
    const T& wc = xt[3 * nb + 3 * c + 2];
    const T& wp = xt[3 * nb + 3 * p + 2];
    r[row] = wc * wc * rcx - wp * wp * rpx;
    r[row + 1] = wc * wc * rcy - wp * wp * rpy;
  }
  dense_solve(n, K, r);
  r.resize(nq);
  return r;
}

// Augmented right-hand side (f(x,u), Omega(x,u)) — NOT yet multiplied by s.
// State x~ = (q_1..q_nb, v_1..v_nb, y) with q_b = (p_x, p_y, theta),
// v_b = (v_x, v_y, omega).  Input u = (tau_1..tau_nj, then, unless the joint
// reaction forces are eliminated, lambda_1x, lambda_1y, ..., lambda_njx,
// lambda_njy, then three contact inputs per contact).
//
// Eq. (1): q' = v; M v' = W + J_c^T R_c phi_c + grad C^T lambda.  Here M is
// diag(m, m, I) per link, W holds gravity and the joint torques, the joint
// reaction force lambda_j acts +lambda_j on the child at its anchor and
// -lambda_j on the parent at its anchor (grad C^T lambda for the revolute
// constraint C = p_c + R_c rho_c - p_p - R_p rho_p), the joint torque tau_j
// acts +tau_j on the child and -tau_j on the parent, and the contact force
// with contact-frame components (tangential, normal) acts at the contact
// point as t tangential + n normal (R_c phi_c; on flat ground t = (1, 0),
// n = (0, 1)).  With jelim the reaction forces come from Eq. (3) instead
// (eliminated_accel).
// Eq. (12): Omega_i = sum over the contact's path constraints g <= 0 of
// h(g), with g = (-lambda_n, -lambda_t+, -lambda_t-, -phi_i(q),
// lambda_t+ + lambda_t- - mu lambda_n), phi_i the signed distance of the
// contact point to the contact surface.
template <class T>
void rhs(const OracleModel& M, const T* xt, const T* u, T* out) {
  const int nb = M.nb, nj = M.nj, nc = M.nc;
  const int ci = (M.jelim ? 1 : 3) * nj;  // first contact input
  std::vector<T> Fx(nb, T(0.0)), Fy(nb, T(0.0)), Tq(nb, T(0.0));
  for (int b = 0; b < nb; ++b) Fy[b] = T(-M.mass[b] * M.g);
  for (int j = 0; j < nj; ++j) {
    const int p = M.jparent[j], c = M.jchild[j];
    const T& tau = u[j];
    if (M.jelim) {
      Tq[c] = Tq[c] + tau;
      Tq[p] = Tq[p] - tau;
      continue;
    }
    const T& lx = u[nj + 2 * j];
    const T& ly = u[nj + 2 * j + 1];
    T rcx, rcy, rpx, rpy;
    lever_arm(xt[3 * c + 2], M.jrho_c + 2 * j, rcx, rcy);
    lever_arm(xt[3 * p + 2], M.jrho_p + 2 * j, rpx, rpy);
    Fx[c] = Fx[c] + lx;
    Fy[c] = Fy[c] + ly;
    Tq[c] = Tq[c] + cross2(rcx, rcy, lx, ly) + tau;
    Fx[p] = Fx[p] - lx;
    Fy[p] = Fy[p] - ly;
    Tq[p] = Tq[p] - cross2(rpx, rpy, lx, ly) - tau;
  }
  for (int i = 0; i < nc; ++i) {
    const int b = M.cbody[i];
    T rx, ry;
    lever_arm(xt[3 * b + 2], M.crho + 2 * i, rx, ry);
    // signed distance and contact frame at the contact point p + r
    const Frame<T> fr = contact_frame(M, xt[3 * b] + rx, xt[3 * b + 1] + ry);
    const T& phi = fr.phi;
    T fx, fy;
    if (M.aux == 0) {
      const T& ln = u[ci + 3 * i];
      const T& ltp = u[ci + 3 * i + 1];
      const T& ltm = u[ci + 3 * i + 2];
      const T ft = ltp - ltm;  // tangential component
      fx = fr.tx * ft + fr.nx * ln;
      fy = fr.ty * ft + fr.ny * ln;
      out[6 * nb + i] = sabs_plus(-ln) + sabs_plus(-ltp) + sabs_plus(-ltm) + sabs_plus(-phi) +
                        sabs_plus(ltp + ltm - M.cmu[i] * ln);
    } else {
      // Eq. (12): contact-frame force (phi_t, phi_n) and multiplier gamma; the
      // auxiliary states integrate phi_n, lambda^c = t^T J_c v + gamma
      // d||phi_t||~/dphi_t (Sec. II-A), gamma and rho^c = |mu phi_n|~ -
      // ||phi_t||~, then the path penalty of the contact's nonnegativity
      // constraints (phi_n, phi, gamma, rho^c >= 0).
      const T& ft = u[ci + 3 * i];
      const T& fn = u[ci + 3 * i + 1];
      const T& gam = u[ci + 3 * i + 2];
      fx = fr.tx * ft + fr.nx * fn;
      fy = fr.ty * ft + fr.ny * fn;
      // contact-point velocity p' + omega x r = (v_x - omega r_y, v_y + omega r_x)
      const T vcx = xt[3 * nb + 3 * b] - xt[3 * nb + 3 * b + 2] * ry;
      const T vcy = xt[3 * nb + 3 * b + 1] + xt[3 * nb + 3 * b + 2] * rx;
      const T vt = fr.tx * vcx + fr.ty * vcy;  // tangential velocity t^T J_c v
      const T lam_c = vt + gam * (ft / sqrt(1.0 + ft * ft));
      const T rho_c = smooth_abs(M.cmu[i] * fn) - smooth_abs(ft);
      out[6 * nb + 4 * i] = fn;
      out[6 * nb + 4 * i + 1] = lam_c;
      out[6 * nb + 4 * i + 2] = gam;
      out[6 * nb + 4 * i + 3] = rho_c;
      out[6 * nb + 4 * nc + i] = sabs_plus(-fn) + sabs_plus(-phi) + sabs_plus(-gam) +
                                 sabs_plus(-rho_c);
    }
    Fx[b] = Fx[b] + fx;
    Fy[b] = Fy[b] + fy;
    Tq[b] = Tq[b] + cross2(rx, ry, fx, fy);
  }
  std::vector<T> vd;
  if (M.jelim) vd = eliminated_accel(M, xt, Fx, Fy, Tq);
  for (int b = 0; b < nb; ++b) {
    for (int k = 0; k < 3; ++k) out[3 * b + k] = xt[3 * nb + 3 * b + k];
    if (M.jelim) {
      for (int k = 0; k < 3; ++k) out[3 * nb + 3 * b + k] = vd[3 * b + k];
      continue;
    }
    out[3 * nb + 3 * b + 0] = Fx[b] / M.mass[b];
    out[3 * nb + 3 * b + 1] = Fy[b] / M.mass[b];
    out[3 * nb + 3 * b + 2] = Tq[b] / M.inertia[b];
  }
}

// Butcher tableaux of the explicit fixed-step schemes.  Classical RK4 is the
// default; the paper integrates with a Runge-Kutta-Fehlberg method (Sec. VI):
// Fehlberg's six-stage 4(5) pair, advanced with its fifth-order weights (a
// fixed step has no use for the embedded fourth-order error estimate).
struct Tableau {
  int s;           // stages
  double c[6];     // stage times
  double a[6][6];  // stage coupling (strictly lower triangular)
  double b[6];     // weights
};

const Tableau kRK4 = {4,
                      {0.0, 0.5, 0.5, 1.0},
                      {{0.0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}},
                      {1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0}};

const Tableau kRKF45 = {6,
                        {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0},
                        {{0.0},
                         {1.0 / 4.0},
                         {3.0 / 32.0, 9.0 / 32.0},
                         {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0},
                         {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0},
                         {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}},
                        {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0,
                         2.0 / 55.0}};

const Tableau& tableau_of(int scheme) { return scheme == 1 ? kRKF45 : kRK4; }

// n_sub fixed steps of the explicit Runge-Kutta scheme `tb` applied to
// d x/d tau = s F(x, u(tau)) on tau in [0,1], u(tau) = (1 - tau) u_L + tau u_R
// (first-order hold), Eqs. (14)-(15):
//   k_j = s F(x + h sum_{l<j} a_jl k_l, u((i + c_j) h)),  x <- x + h sum_j b_j k_j.
template <class T, class RHS>
void rk_foh(const RHS& F, const Tableau& tb, int nxt, int nu, const T* x0, const T* uL,
            const T* uR, const T& s, int nsub, T* x1) {
  const double h = 1.0 / nsub;
  std::vector<T> x(x0, x0 + nxt), xs(nxt), acc(nxt), u(nu), fv(nxt);
  std::vector<std::vector<T>> k(tb.s, std::vector<T>(nxt));
  for (int i = 0; i < nsub; ++i) {
    for (int j = 0; j < tb.s; ++j) {
      const double tau = (i + tb.c[j]) * h;
      for (int r = 0; r < nxt; ++r) {
        T v = x[r];
        for (int l = 0; l < j; ++l)
          if (tb.a[j][l] != 0.0) v = v + (tb.a[j][l] * h) * k[l][r];
        xs[r] = v;
      }
      for (int q = 0; q < nu; ++q) u[q] = (1.0 - tau) * uL[q] + tau * uR[q];
      F(xs.data(), u.data(), fv.data());
      for (int r = 0; r < nxt; ++r) k[j][r] = s * fv[r];
    }
    for (int r = 0; r < nxt; ++r) {
      acc[r] = T(0.0);
      for (int j = 0; j < tb.s; ++j) acc[r] = acc[r] + tb.b[j] * k[j][r];
      x[r] = x[r] + h * acc[r];
    }
  }
  for (int r = 0; r < nxt; ++r) x1[r] = x[r];
}

// IND on one interval: seed duals in (x~_k, u_L, u_R, s), run rk_foh, read
// the tangents.  Direction order: x~ (nxt), u_L (nu), u_R (nu), s (1).
template <class RHSD>
int ind_interval(const RHSD& F, const Tableau& tb, int nxt, int nu, int nsub, const double* x0,
                 const double* uL, const double* uR, double s, double* x1, double* A, double* Bm,
                 double* Bp, double* S) {
  const int C = nxt + 2 * nu + 1;
  if (C > MAXC) return 1;
  g_nd = C;
  std::vector<Dual> X0(nxt), UL(nu), UR(nu), X1(nxt);
  for (int r = 0; r < nxt; ++r) { X0[r] = Dual(x0[r]); X0[r].d[r] = 1.0; }
  for (int q = 0; q < nu; ++q) {
    UL[q] = Dual(uL[q]); UL[q].d[nxt + q] = 1.0;
    UR[q] = Dual(uR[q]); UR[q].d[nxt + nu + q] = 1.0;
  }
  Dual Sd(s); Sd.d[C - 1] = 1.0;
  rk_foh<Dual>(F, tb, nxt, nu, X0.data(), UL.data(), UR.data(), Sd, nsub, X1.data());
  for (int r = 0; r < nxt; ++r) {
    if (x1) x1[r] = X1[r].v;
    if (A) for (int c = 0; c < nxt; ++c) A[r * nxt + c] = X1[r].d[c];
    if (Bm) for (int q = 0; q < nu; ++q) Bm[r * nu + q] = X1[r].d[nxt + q];
    if (Bp) for (int q = 0; q < nu; ++q) Bp[r * nu + q] = X1[r].d[nxt + nu + q];
    if (S) S[r] = X1[r].d[C - 1];
  }
  return 0;
}

int model_ok(const OracleModel* M) {
  if (!M || M->nb < 1 || M->nj < 0 || M->nc < 0 || (M->aux != 0 && M->aux != 1)) return 0;
  if ((M->jelim != 0 && M->jelim != 1) || (M->scheme != 0 && M->scheme != 1)) return 0;
  if (!std::isfinite(M->terrain_amp) || !std::isfinite(M->terrain_k)) return 0;
  for (int j = 0; j < M->nj; ++j)
    if (M->jparent[j] < 0 || M->jparent[j] >= M->nb || M->jchild[j] < 0 || M->jchild[j] >= M->nb)
      return 0;
  for (int i = 0; i < M->nc; ++i)
    if (M->cbody[i] < 0 || M->cbody[i] >= M->nb) return 0;
  return 1;
}

// Controls of interval k: node layout U[N+1][nu] (u_L = U_k, u_R = U_{k+1});
// interval layout U[N][2][nu] (u_L, u_R per interval; FOH may jump at nodes,
// Sec. VI).
void controls_of(int layout, int nu, const double* U, long k, const double** uL,
                 const double** uR) {
  if (layout == 0) { *uL = U + k * nu; *uR = U + (k + 1) * nu; }
  else { *uL = U + 2 * k * nu; *uR = U + (2 * k + 1) * nu; }
}

template <class Fn>
void parallel_for(long n, int nthreads, const Fn& fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  nthreads = (int)std::min<long>(nthreads, std::max<long>(n, 1));
  if (nthreads <= 1) { for (long k = 0; k < n; ++k) fn(k); return; }
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&, t]() { for (long k = t; k < n; k += nthreads) fn(k); });
  for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// Dimensions n_x~ = 6 n_b + n_c, n_u = 3 n_j + 3 n_c.
int oracle_dims(const OracleModel* M, int* nxt, int* nu) {
  if (!model_ok(M)) return 1;
  *nxt = nxt_of(*M);
  *nu = nu_of(*M);
  return 0;
}

// Unscaled augmented right-hand side (f, Omega) at one point.
int oracle_rhs(const OracleModel* M, const double* xt, const double* u, double* out) {
  if (!model_ok(M)) return 1;
  rhs<double>(*M, xt, u, out);
  return 0;
}

// The nonlinear flow map F~(x~_0, u_L, u_R, s) of one interval, plain FP64.
int oracle_flow(const OracleModel* M, int nsub, const double* x0, const double* uL,
                const double* uR, double s, double* x1) {
  if (!model_ok(M) || nsub < 1) return 1;
  auto F = [M](const double* x, const double* u, double* o) { rhs<double>(*M, x, u, o); };
  rk_foh<double>(F, tableau_of(M->scheme), nxt_of(*M), nu_of(*M), x0, uL, uR, s, nsub, x1);
  return 0;
}

// One interval: x~(1) and its IND Jacobian blocks A [nxt][nxt], B-/B+ [nxt][nu], S [nxt].
int oracle_interval(const OracleModel* M, int nsub, const double* x0, const double* uL,
                    const double* uR, double s, double* x1, double* A, double* Bm, double* Bp,
                    double* S) {
  if (!model_ok(M) || nsub < 1) return 1;
  auto F = [M](const Dual* x, const Dual* u, Dual* o) { rhs<Dual>(*M, x, u, o); };
  return ind_interval(F, tableau_of(M->scheme), nxt_of(*M), nu_of(*M), nsub, x0, uL, uR, s, x1,
                      A, Bm, Bp, S);
}

// All N intervals of a multiple-shooting grid (independently, Eq. (17b)).
// X [N+1][nxt]; U per layout; s [N].  Outputs: A [N][nxt][nxt], Bm/Bp
// [N][nxt][nu], S [N][nxt], defect [N][nxt], penalty [N][nc].  Any output
// pointer may be NULL.
int oracle_discretize(const OracleModel* M, int N, int nsub, int layout, const double* X,
                      const double* U, const double* s, double* A, double* Bm, double* Bp,
                      double* S, double* defect, double* penalty, int nthreads) {
  if (!model_ok(M) || N < 1 || nsub < 1 || (layout != 0 && layout != 1)) return 1;
  const int nxt = nxt_of(*M), nu = nu_of(*M), nx = pen_of(*M), nc = M->nc;
  if (nxt + 2 * nu + 1 > MAXC) return 1;
  int err = 0;
  parallel_for(N, nthreads, [&](long k) {
    const double *uL, *uR;
    controls_of(layout, nu, U, k, &uL, &uR);
    std::vector<double> x1(nxt);
    const size_t a = (size_t)k * nxt * nxt, b = (size_t)k * nxt * nu, v = (size_t)k * nxt;
    if (oracle_interval(M, nsub, X + k * nxt, uL, uR, s[k], x1.data(), A ? A + a : nullptr,
                        Bm ? Bm + b : nullptr, Bp ? Bp + b : nullptr, S ? S + v : nullptr))
      err = 1;
    if (defect)
      for (int r = 0; r < nxt; ++r) defect[v + r] = x1[r] - X[(k + 1) * nxt + r];
    if (penalty)
      for (int i = 0; i < nc; ++i) penalty[(size_t)k * nc + i] = x1[nx + i] - X[k * nxt + nx + i];
  });
  return err;
}

// Gradient of L = sum_k w_k . defect_k + sum_k rho_k . penalty_k with respect
// to X, U and s, contracted from the IND blocks:
//   lambda_k = w_k + (rho_k placed on the y rows)          (cotangent of x~(1))
//   dL/dx~_k    += A_k^T lambda_k,  minus rho_k on the y rows (penalty_k subtracts y_k),
//   dL/dx~_{k+1} -= w_k                                       (defect_k subtracts x~_{k+1}),
//   dL/du_L,k = B-_k^T lambda_k,  dL/du_R,k = B+_k^T lambda_k,  dL/ds_k = S_k . lambda_k.
// Node layout sums the u_L part of interval k and the u_R part of interval
// k-1 into node k.  gX [N+1][nxt], gU like U, gs [N]; L (scalar) may be NULL.
int oracle_vjp(const OracleModel* M, int N, int nsub, int layout, const double* X,
               const double* U, const double* s, const double* w, const double* rho, double* gX,
               double* gU, double* gs, double* L, int nthreads) {
  if (!model_ok(M) || N < 1 || nsub < 1 || (layout != 0 && layout != 1)) return 1;
  const int nxt = nxt_of(*M), nu = nu_of(*M), nx = pen_of(*M), nc = M->nc;
  std::vector<double> A((size_t)N * nxt * nxt), Bm((size_t)N * nxt * nu), Bp((size_t)N * nxt * nu),
      S((size_t)N * nxt), D((size_t)N * nxt), P((size_t)N * (nc > 0 ? nc : 1));
  if (oracle_discretize(M, N, nsub, layout, X, U, s, A.data(), Bm.data(), Bp.data(), S.data(),
                        D.data(), P.data(), nthreads))
    return 1;
  const long nU = (layout == 0) ? (long)(N + 1) * nu : (long)2 * N * nu;
  std::fill(gX, gX + (size_t)(N + 1) * nxt, 0.0);
  std::fill(gU, gU + nU, 0.0);
  double Ltot = 0.0;
  std::vector<double> lam(nxt);
  for (long k = 0; k < N; ++k) {
    for (int r = 0; r < nxt; ++r) lam[r] = w[k * nxt + r];
    for (int i = 0; i < nc; ++i) lam[nx + i] += rho[k * nc + i];
    const double* Ak = A.data() + (size_t)k * nxt * nxt;
    const double* Bmk = Bm.data() + (size_t)k * nxt * nu;
    const double* Bpk = Bp.data() + (size_t)k * nxt * nu;
    for (int c = 0; c < nxt; ++c) {
      double acc = 0.0;
      for (int r = 0; r < nxt; ++r) acc += Ak[r * nxt + c] * lam[r];
      gX[k * nxt + c] += acc;
    }
    for (int i = 0; i < nc; ++i) gX[k * nxt + nx + i] -= rho[k * nc + i];
    for (int r = 0; r < nxt; ++r) gX[(k + 1) * nxt + r] -= w[k * nxt + r];
    double* gL = (layout == 0) ? gU + k * nu : gU + 2 * k * nu;
    double* gR = (layout == 0) ? gU + (k + 1) * nu : gU + (2 * k + 1) * nu;
    for (int q = 0; q < nu; ++q) {
      double aL = 0.0, aR = 0.0;
      for (int r = 0; r < nxt; ++r) { aL += Bmk[r * nu + q] * lam[r]; aR += Bpk[r * nu + q] * lam[r]; }
      gL[q] += aL;
      gR[q] += aR;
    }
    double as = 0.0;
    for (int r = 0; r < nxt; ++r) as += S[k * nxt + r] * lam[r];
    gs[k] = as;
    for (int r = 0; r < nxt; ++r) Ltot += w[k * nxt + r] * D[k * nxt + r];
    for (int i = 0; i < nc; ++i) Ltot += rho[k * nc + i] * P[k * nc + i];
  }
  if (L) *L = Ltot;
  return 0;
}

// The same integrator (scheme 0: RK4, 1: RKF45) and IND on a linear
// right-hand side F(x,u) = Ac x + Bc u (Ac [n][n], Bc [n][m], row-major).
// Used only to pin rk_foh/IND against closed forms.
int oracle_linear_interval(int n, int m, const double* Ac, const double* Bc, int nsub,
                           const double* x0, const double* uL, const double* uR, double s,
                           double* x1, double* A, double* Bm, double* Bp, double* S, int scheme) {
  if (n < 1 || m < 0 || nsub < 1 || n + 2 * m + 1 > MAXC || scheme < 0 || scheme > 1) return 1;
  auto F = [=](const Dual* x, const Dual* u, Dual* o) {
    for (int r = 0; r < n; ++r) {
      Dual acc(0.0);
      for (int c = 0; c < n; ++c) acc = acc + Ac[r * n + c] * x[c];
      for (int q = 0; q < m; ++q) acc = acc + Bc[r * m + q] * u[q];
      o[r] = acc;
    }
  };
  return ind_interval(F, tableau_of(scheme), n, m, nsub, x0, uL, uR, s, x1, A, Bm, Bp, S);
}

// The Butcher tableau of a scheme: stages, c [6], a [6][6] row-major, b [6].
int oracle_tableau(int scheme, int* stages, double* c, double* a, double* b) {
  if (scheme < 0 || scheme > 1) return 1;
  const Tableau& tb = tableau_of(scheme);
  *stages = tb.s;
  for (int i = 0; i < 6; ++i) {
    c[i] = tb.c[i];
    b[i] = tb.b[i];
    for (int j = 0; j < 6; ++j) a[6 * i + j] = tb.a[i][j];
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Node constraints: the impact map G~ and the relaxed impulse complementarity
// Theta^delta imposed at every grid node (Sec. IV-C, Eqs. (17e)-(17f)), with
// their Jacobians by the same forward-mode dual numbers.
// ---------------------------------------------------------------------------
namespace {

// Fischer-Burmeister relaxation, Eq. (16): FB^delta(a, b) = a + b - sqrt(a^2 + b^2 + delta).
template <class T> T fischer_burmeister(const T& a, const T& b, double delta) {
  return a + b - sqrt(a * a + b * b + delta);
}

// G~(x~+, x~-, Phi) and Theta^delta(x+, x-, Phi, Gamma) at one node.
//
// Impact dynamics Eq. (6a): M (v+ - v-) = J_c^T R_c Phi + grad C^T Lambda.
// The joint impulse Lambda is eliminated with the post-impact joint
// constraint at the velocity level, grad C v+ = 0 (Sec. II-B):
//   w = v- + M^-1 J_c^T R_c Phi,  K = grad C M^-1 grad C^T,  Lambda = -K^-1 grad C w,
// and G~ stacks q+ - q- (pose continuity), M (v+ - v-) - J_c^T R_c Phi -
// grad C^T Lambda, and y+ - y- (auxiliary-state continuity).  Every
// kinematic quantity is taken at the pre-impact pose q-.  M = diag(m, m, I)
// per link; on flat ground R_c maps (Phi_t, Phi_n) to the world impulse
// (Phi_t, Phi_n).
//
// Theta collects, per contact i, the Fischer-Burmeister relaxations
// (Eq. (16)) of the impulse conditions Eqs. (6b)-(6e) and the sign
// conditions that go with them:
//   FB(Phi_n, phi),  FB(Phi_n, |c|~),  FB(Phi_n, |lambda^c|~),  FB(Gamma, rho),
//   -Phi_n, -phi, -Gamma, -rho,
// with phi the signed distance of the contact point, c = n^T J_c (v+ + e v-)
// its normal velocity after impact plus e times before (Eq. (6c)),
// lambda^c = t^T J_c v+ + Gamma d||Phi_t||~/dPhi_t (Eq. (6d)),
// rho = |mu Phi_n|~ - ||Phi_t||~ (Eq. (6e)); |.|~ the pseudo-Huber absolute
// value, which turns each "Phi_n times a signed quantity = 0" into the
// complementarity 0 <= Phi_n perp |quantity|~ >= 0.
template <class T>
void node_eval(const OracleModel& M, const T* xp, const T* xm, const T* Phi, const T* Gam,
               double delta, const double* e, T* g, T* th) {
  const int nb = M.nb, nj = M.nj, nc = M.nc, nq = 3 * nb;
  const T* qm = xm;
  const T* vm = xm + nq;
  const T* vp = xp + nq;
  std::vector<double> minv(nq);
  for (int b = 0; b < nb; ++b) {
    minv[3 * b] = minv[3 * b + 1] = 1.0 / M.mass[b];
    minv[3 * b + 2] = 1.0 / M.inertia[b];
  }
  // grad C (2 nj x nq): C_j = p_c + R(theta_c) rho_c - p_p - R(theta_p) rho_p.
  std::vector<T> G((size_t)2 * nj * nq, T(0.0));
  for (int j = 0; j < nj; ++j) {
    const int c = M.jchild[j], p = M.jparent[j];
    T rcx, rcy, rpx, rpy;
    lever_arm(qm[3 * c + 2], M.jrho_c + 2 * j, rcx, rcy);
    lever_arm(qm[3 * p + 2], M.jrho_p + 2 * j, rpx, rpy);
    // d(R rho)/dtheta = (-r_y, r_x)
    G[(2 * j) * nq + 3 * c] = G[(2 * j) * nq + 3 * c] + 1.0;
    G[(2 * j + 1) * nq + 3 * c + 1] = G[(2 * j + 1) * nq + 3 * c + 1] + 1.0;
    G[(2 * j) * nq + 3 * c + 2] = G[(2 * j) * nq + 3 * c + 2] - rcy;
    G[(2 * j + 1) * nq + 3 * c + 2] = G[(2 * j + 1) * nq + 3 * c + 2] + rcx;
    G[(2 * j) * nq + 3 * p] = G[(2 * j) * nq + 3 * p] - 1.0;
    G[(2 * j + 1) * nq + 3 * p + 1] = G[(2 * j + 1) * nq + 3 * p + 1] - 1.0;
    G[(2 * j) * nq + 3 * p + 2] = G[(2 * j) * nq + 3 * p + 2] + rpy;
    G[(2 * j + 1) * nq + 3 * p + 2] = G[(2 * j + 1) * nq + 3 * p + 2] - rpx;
  }
  // J_c^T R_c Phi as a generalized impulse (nq), the contact lever arms and
  // the contact frames (at the pre-impact contact points).
  std::vector<T> Jphi(nq, T(0.0)), crx(nc), cry(nc);
  std::vector<Frame<T>> fr(nc);
  for (int i = 0; i < nc; ++i) {
    const int b = M.cbody[i];
    lever_arm(qm[3 * b + 2], M.crho + 2 * i, crx[i], cry[i]);
    fr[i] = contact_frame(M, qm[3 * b] + crx[i], qm[3 * b + 1] + cry[i]);
    const T& pt = Phi[2 * i];
    const T& pn = Phi[2 * i + 1];
    const T ix = fr[i].tx * pt + fr[i].nx * pn;  // world impulse R_c Phi
    const T iy = fr[i].ty * pt + fr[i].ny * pn;
    Jphi[3 * b] = Jphi[3 * b] + ix;
    Jphi[3 * b + 1] = Jphi[3 * b + 1] + iy;
    Jphi[3 * b + 2] = Jphi[3 * b + 2] + cross2(crx[i], cry[i], ix, iy);
  }
  // Lambda = -K^-1 grad C w.
  std::vector<T> w(nq);
  for (int a = 0; a < nq; ++a) w[a] = vm[a] + minv[a] * Jphi[a];
  std::vector<T> K((size_t)4 * nj * nj, T(0.0)), lam(2 * nj, T(0.0));
  for (int r = 0; r < 2 * nj; ++r) {
    for (int c2 = 0; c2 < 2 * nj; ++c2) {
      T acc(0.0);
      for (int a = 0; a < nq; ++a) acc = acc + G[r * nq + a] * minv[a] * G[c2 * nq + a];
      K[r * 2 * nj + c2] = acc;
    }
    T acc(0.0);
    for (int a = 0; a < nq; ++a) acc = acc + G[r * nq + a] * w[a];
    lam[r] = acc;
  }
  if (nj > 0) dense_solve(2 * nj, K, lam);
  for (int r = 0; r < 2 * nj; ++r) lam[r] = -lam[r];
  // G~
  for (int a = 0; a < nq; ++a) g[a] = xp[a] - xm[a];
  for (int a = 0; a < nq; ++a) {
    T acc = (1.0 / minv[a]) * (vp[a] - vm[a]) - Jphi[a];
    for (int r = 0; r < 2 * nj; ++r) acc = acc - G[r * nq + a] * lam[r];
    g[nq + a] = acc;
  }
  for (int a = 2 * nq; a < nxt_of(M); ++a) g[a] = xp[a] - xm[a];
  // Theta
  for (int i = 0; i < nc; ++i) {
    const int b = M.cbody[i];
    const T& pt = Phi[2 * i];
    const T& pn = Phi[2 * i + 1];
    const T& phi = fr[i].phi;
    // contact-point velocity p' + omega x r = (v_x - omega r_y, v_y + omega r_x)
    // after (p) and before (m) the impact, in the contact frame
    const T vxp = vp[3 * b] - vp[3 * b + 2] * cry[i];
    const T vyp = vp[3 * b + 1] + vp[3 * b + 2] * crx[i];
    const T vxm = vm[3 * b] - vm[3 * b + 2] * cry[i];
    const T vym = vm[3 * b + 1] + vm[3 * b + 2] * crx[i];
    const T vtp = fr[i].tx * vxp + fr[i].ty * vyp;
    const T vnp = fr[i].nx * vxp + fr[i].ny * vyp;
    const T vnm = fr[i].nx * vxm + fr[i].ny * vym;
    const T cn = vnp + e[i] * vnm;
    const T lc = vtp + Gam[i] * (pt / sqrt(1.0 + pt * pt));
    const T rho = smooth_abs(M.cmu[i] * pn) - smooth_abs(pt);
    T* o = th + 8 * i;
    o[0] = fischer_burmeister(pn, phi, delta);
    o[1] = fischer_burmeister(pn, smooth_abs(cn), delta);
    o[2] = fischer_burmeister(pn, smooth_abs(lc), delta);
    o[3] = fischer_burmeister(Gam[i], rho, delta);
    o[4] = -pn;
    o[5] = -phi;
    o[6] = -Gam[i];
    o[7] = -rho;
  }
}

}  // namespace

extern "C" {

// Node constraints at n nodes.  Xp, Xm [n][nxt] post-/pre-impact states,
// Phi [n][2 nc] contact impulses (Phi_t, Phi_n) per contact, Gam [n][nc]
// multipliers, delta > 0, e [nc] restitution coefficients.  Outputs (any may
// be NULL): g [n][nxt] = G~, theta [n][8 nc] = Theta^delta, and their full
// Jacobians with respect to z = (x~+, x~-, Phi, Gamma) (2 nxt + 3 nc
// columns): Jg [n][nxt][ncol], Jth [n][8 nc][ncol].
int oracle_node(const OracleModel* M, int n, const double* Xp, const double* Xm,
                const double* Phi, const double* Gam, double delta, const double* e, double* g,
                double* theta, double* Jg, double* Jth, int nthreads) {
  if (!model_ok(M) || n < 1 || !(delta > 0.0)) return 1;
  const int nxt = nxt_of(*M), nc = M->nc, ncol = 2 * nxt + 3 * nc;
  if (ncol > MAXC) return 1;
  parallel_for(n, nthreads, [&](long k) {
    g_nd = ncol;
    std::vector<Dual> xp(nxt), xm(nxt), ph(2 * nc), gm(nc), gv(nxt), tv(8 * nc);
    for (int r = 0; r < nxt; ++r) {
      xp[r] = Dual(Xp[k * nxt + r]); xp[r].d[r] = 1.0;
      xm[r] = Dual(Xm[k * nxt + r]); xm[r].d[nxt + r] = 1.0;
    }
    for (int i = 0; i < 2 * nc; ++i) { ph[i] = Dual(Phi[k * 2 * nc + i]); ph[i].d[2 * nxt + i] = 1.0; }
    for (int i = 0; i < nc; ++i) { gm[i] = Dual(Gam[k * nc + i]); gm[i].d[2 * nxt + 2 * nc + i] = 1.0; }
    node_eval<Dual>(*M, xp.data(), xm.data(), ph.data(), gm.data(), delta, e, gv.data(), tv.data());
    for (int r = 0; r < nxt; ++r) {
      if (g) g[k * nxt + r] = gv[r].v;
      if (Jg) for (int c = 0; c < ncol; ++c) Jg[((size_t)k * nxt + r) * ncol + c] = gv[r].d[c];
    }
    for (int r = 0; r < 8 * nc; ++r) {
      if (theta) theta[k * 8 * nc + r] = tv[r].v;
      if (Jth) for (int c = 0; c < ncol; ++c) Jth[((size_t)k * 8 * nc + r) * ncol + c] = tv[r].d[c];
    }
  });
  return 0;
}

// Psi^{delta,eps}(y-_{k+1}, y+_k) at N intervals, from the node states
// Xp, Xm [N+1][nxt] (post-/pre-impact).  With d = y-_{k+1} - y+_k the
// auxiliary-state increment over interval k:
//   aux model 1 (Eq. (12) states phi_n, lambda^c, gamma, rho^c at y index
//     4i..4i+3, path penalty at 4 nc + i): per contact i the integral
//     cross-complementarity pairs (phi_n, lambda^c) and (gamma, rho^c)
//     relaxed by Eq. (16), FB(d[4i], d[4i+1]) and FB(d[4i+2], d[4i+3]), at
//     rows 2i and 2i+1; then per contact the relaxed path-constraint row of
//     Eq. (13), d[4 nc + i] - eps, at row 2 nc + i (3 nc rows);
//   aux model 0 (one path-penalty state per contact): d[i] - eps (nc rows).
// Outputs (any may be NULL): psi [N][npsi], J [N][npsi][2 ny] with columns
// (y+_k, y-_{k+1}).
int oracle_psi(const OracleModel* M, int N, const double* Xp, const double* Xm, double delta,
               double eps, double* psi, double* J, int nthreads) {
  if (!model_ok(M) || N < 1 || !(delta > 0.0)) return 1;
  const int nxt = nxt_of(*M), nc = M->nc, ny = nxt - 6 * M->nb;
  const int npsi = M->aux ? 3 * nc : nc, ncol = 2 * ny;
  if (ncol > MAXC) return 1;
  parallel_for(N, nthreads, [&](long k) {
    g_nd = ncol;
    std::vector<Dual> d(ny), out(npsi);
    for (int j = 0; j < ny; ++j) {
      Dual yp(Xp[k * nxt + 6 * M->nb + j]), ym(Xm[(k + 1) * nxt + 6 * M->nb + j]);
      yp.d[j] = 1.0;
      ym.d[ny + j] = 1.0;
      d[j] = ym - yp;
    }
    if (M->aux) {
      for (int i = 0; i < nc; ++i) {
        out[2 * i] = fischer_burmeister(d[4 * i], d[4 * i + 1], delta);
        out[2 * i + 1] = fischer_burmeister(d[4 * i + 2], d[4 * i + 3], delta);
        out[2 * nc + i] = d[4 * nc + i] - eps;
      }
    } else {
      for (int i = 0; i < nc; ++i) out[i] = d[i] - eps;
    }
    for (int r = 0; r < npsi; ++r) {
      if (psi) psi[k * npsi + r] = out[r].v;
      if (J) for (int c = 0; c < ncol; ++c) J[((size_t)k * npsi + r) * ncol + c] = out[r].d[c];
    }
  });
  return 0;
}

// The same G~ and Theta in plain FP64 (no derivatives), for finite differences.
int oracle_node_value(const OracleModel* M, const double* xp, const double* xm, const double* Phi,
                      const double* Gam, double delta, const double* e, double* g, double* theta) {
  if (!model_ok(M) || !(delta > 0.0)) return 1;
  node_eval<double>(*M, xp, xm, Phi, Gam, delta, e, g, theta);
  return 0;
}

}  // extern "C"
