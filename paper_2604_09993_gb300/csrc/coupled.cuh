// coupled.cuh — tables of the coupled-dynamics path (coupled.cu): models
// whose links are coupled within an interval, which the per-link kernels
// cannot treat.  That is the case when
//  * the joint reaction forces are eliminated at the acceleration level
//    (Sec. II-A, Eq. (3)): every link's acceleration then depends on every
//    link's angle and rate through the solve of K lambda = ..., K = grad C
//    M^-1 grad C^T, so the Jacobian blocks are dense in those rows;
//  * the contact surface is the sinusoid of Sec. VI-B: the contact force's
//    direction and the signed distance depend on the foot's x position;
//  * the integrator is the Runge-Kutta-Fehlberg 4(5) tableau (Sec. VI).
//
// Rows of the state fall into two classes.  "Live" rows feed back into the
// right-hand side or into the stage values another row needs: theta and
// omega of every link and (p_x, p_y, v_x, v_y) of every link that carries a
// contact.  They are integrated with the full Runge-Kutta stage recursion.
// The other rows — (p_x, p_y, v_x, v_y) of links without a contact and the
// auxiliary states — never feed back, so their tangents are quadratures of
// the stage slopes: v += h sum_j b_j k_j, and, since p' = s v, p += h s v +
// h^2 s sum_l beta_l kv_l with beta_l = sum_j b_j a_jl (exact for any explicit
// tableau), which needs no stage storage.
#pragma once

#include "common.cuh"

namespace ciscvx {

constexpr int CPL_MAXJ = NODE_MAXJ;                 // joints (the KKT system has 2 n_j rows)
constexpr int CPL_MAXROW = 6 * MAXB + 5 * MAXB;     // state rows n_x~
constexpr int CPL_MAXSKY = NODE_MAXJ * (2 * NODE_MAXJ + 1);  // skyline entries of K (<= n_k (n_k+1) / 2)
constexpr int CPL_MAXSTAGE = 6;
// per-contact stage fields: aux model 0 / aux model 1 (see coupled.cu)
constexpr int CPL_CF0 = 14, CPL_CF1 = 21;

struct CplTab {
  int nb, nj, nc, nxt, nu, ny, aux, jelim, scheme;
  int C;       // tangent columns n_x~ + 2 n_u + 1
  int nk;      // KKT rows 2 n_j (0 without elimination)
  int nsky;    // skyline entries of K
  int nlive, nquad;
  int ci0;     // first contact input (n_j with elimination, 3 n_j without)
  int pen0;    // first path-penalty state row (the penalty output's rows)
  int stages;  // tableau stages
  int nks;     // stored stage slopes per row (1 for RK4: only the previous one is used)
  // stage data (per interval, per substep, per stage; in the tangent precision)
  int sd_arm, sd_qw, sd_F, sd_K, sd_con, sd_size, ncf;
  // per-lane scratch of the nominal kernel (doubles, element major): live
  // rows x, stage values, accumulator (RK4 only), stored slopes; quadrature
  // rows; generalized forces, lever arms, factor of K, reaction forces
  int n_xl, n_xs, n_acc, n_k, n_xq, n_f, n_arm, n_carm, n_K, n_lam, n_qw, n_size;
  // per-thread scratch of the tangent kernel (tangent precision, element major)
  int t_pl, t_acc, t_k, t_xs, t_pq, t_e, t_x, t_size;
  double g, ta, tk;  // gravity; contact surface y = ta sin(tk x)
  double c[CPL_MAXSTAGE], a[CPL_MAXSTAGE][CPL_MAXSTAGE], b[CPL_MAXSTAGE], beta[CPL_MAXSTAGE];
  double mass[MAXB], inertia[MAXB], minv[MAXB], iinv[MAXB];
  // FP32 copies for the FP32 tangent kernel (no conversions in its loops)
  float cf[CPL_MAXSTAGE], af[CPL_MAXSTAGE][CPL_MAXSTAGE], bf[CPL_MAXSTAGE], betaf[CPL_MAXSTAGE];
  float minvf[MAXB], iinvf[MAXB];
  int nadj[MAXB];
  unsigned char adj[MAXB][NODE_MAXADJ];  // (joint << 1) | (1 if the link is the joint's parent)
  int contact[MAXB];                     // contact on the link, or -1
  int jpar[MAXJ], jchi[MAXJ];
  double jrp[MAXJ][2], jrc[MAXJ][2];
  // K in skyline form, joints in children-first order (see node_symbolic)
  int npos[CPL_MAXJ], nord[CPL_MAXJ], nf[2 * CPL_MAXJ], noff[2 * CPL_MAXJ + 1];
  int cbody[MAXB];
  double crho[MAXB][2], mu[MAXB];
  short lrow[CPL_MAXROW], qrow[CPL_MAXROW];  // live / quadrature slot of each state row, or -1
  // Tangent columns the tangent kernel integrates.  The columns of A for the
  // positions and linear velocities of links without a contact and for the
  // auxiliary states are closed-form (those states never enter the
  // right-hand side: A e_p = e_p, A e_v = e_v + s e_p, A e_y = e_y); the
  // nominal kernel writes them.
  int cnt;                                   // columns integrated
  short cperm[CPL_MAXROW + 2 * (3 * MAXJ + 3 * MAXB) + 1];  // integrated column index -> column
  // Compact A (CISCVX_OUT_COMPACT): column-major, column c's structural
  // nonzeros at [colptr[c], colptr[c + 1]) in ascending rows (every row for an
  // integrated column; see cpl_col_kind); compact B- / B+ are every entry,
  // column-major (column q at q n_x~).
  int colptr[CPL_MAXROW + 1];
};

// Kind of column c (< n_x~) of A for a model with coupled links: 0 integrated
// (every row may be nonzero), 1 A e_c = e_c (position of a link without a
// contact, auxiliary state), 2 A e_c = e_c + s e_{c - 3 n_b} (linear velocity
// of a link without a contact; its position row comes first).
inline int cpl_col_kind(const DevModel& M, int c) {
  const int nb = M.nb, nq = 3 * nb;
  if (c >= 6 * nb) return 1;
  if (M.body[(c % nq) / 3].contact >= 0 || (c % 3) == 2) return 0;
  return c < nq ? 1 : 2;
}

// Structural nonzeros of A in the compact order (column-major): column c has
// n_x~ of them when integrated, 1 or 2 otherwise.
inline int cpl_col_nnz(const DevModel& M, int c) {
  const int k = cpl_col_kind(M, c);
  return k == 0 ? M.nxt : (k == 2 ? 2 : 1);
}

// True when the model needs the coupled path.
inline bool cpl_needed(const DevModel& M) { return M.jelim || M.scheme != 0 || M.ta != 0.0; }

// Builds the tables; returns an error text or nullptr.
const char* cpl_build(const DevModel& M, CplTab& T);

// Bytes of stage data per interval.
size_t cpl_interval_bytes(const CplTab& T, int nsub, int prec);

// Linearized discretization of intervals [0, N) in chunks of at most
// `chunk` intervals through the workspace (stage data of one chunk).  With
// `entries`, interval e is entry e = (instance, k) of the batch instance
// table `inst` (element offsets into the packed arrays); else interval e.
// compact: A, Bm, Bp in the compact layout (CplTab::colptr).
cudaError_t launch_coupled(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                           const double* U, const double* s, void* A, void* Bm, void* Bp, void* S,
                           double* defect, double* penalty, void* ws, long chunk,
                           unsigned* status, cudaStream_t st, const int2* entries = nullptr,
                           const DevInst* inst = nullptr, bool compact = false);
// Compiles the specialized kernels and sets the generic kernels' limits
// (before a launch is captured in a graph).
cudaError_t cpl_prepare(const CplTab& T, int prec);

// Run-time specialized tangent kernel (jit.cu): null when unavailable (no
// NVRTC, a failed compile, or CISCVX_COUPLED_JIT=0); then the generic kernel runs.
struct CplJit {
  void* fn = nullptr;  // CUfunction
  int bs = 0;
  size_t smem = 0;
  int blocks_per_sm = 0;  // resident blocks per SM at (bs, smem); 0 if unknown
};
const CplJit* cpl_jit_tangent(const CplTab& T, int prec);
const CplJit* cpl_jit_nominal(const CplTab& T, int prec);
cudaError_t cpl_jit_launch_nominal(const CplJit& J, const CplTab& T, long i0, long n, int nsub,
                                   int layout, const double* X, const double* U, const double* s,
                                   void* sd, void* A, double* defect, double* penalty,
                                   unsigned* status, cudaStream_t st, const int2* entries,
                                   const DevInst* inst, int cmp);
const CplJit* cpl_jit_adjoint(const CplTab& T, int prec);
cudaError_t cpl_jit_launch_adjoint(const CplJit& J, const CplTab& T, int prec, long i0, long n, long N, int nsub,
                                   const double* s, const void* sd, const double* w, const double* rho,
                                   double* gX, double* gs, double* ubar, unsigned* status, cudaStream_t st);
cudaError_t cpl_jit_launch(const CplJit& J, const CplTab& T, int prec, long i0, long n, int nsub,
                           const double* s, const void* sd, void* A, void* Bm, void* Bp, void* S,
                           unsigned* status, cudaStream_t st, int layout, const int2* entries,
                           const DevInst* inst, int cmp);

// The linearization (as launch_coupled, single instance) and the VJP (as
// launch_coupled_vjp) of the same intervals from one nominal pass per chunk;
// workspace as for launch_coupled_vjp.
cudaError_t launch_coupled_and_vjp(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                                   const double* U, const double* s, void* A, void* Bm, void* Bp, void* S,
                                   double* defect, double* penalty, const double* w, const double* rho,
                                   double* gX, double* gU, double* gs, double* L, void* ws, size_t ws_bytes,
                                   unsigned* status, cudaStream_t st, bool compact);

// Reverse-mode VJP of the coupled path (coupled.cu): the nominal kernel's
// forward pass into the stage data of a chunk, then the adjoint kernel (thread
// = interval) backward over the stages; no dense block is formed.  Workspace
// of a chunk of n intervals: stage data, defects, penalty increments and the
// per-interval input cotangents (dL/du_L, dL/du_R).
struct CplAdjLayout {
  size_t stage, defect, penalty, ubar, lpart, total;
};
CplAdjLayout cpl_adjoint_layout(const CplTab& T, long n, int nsub, int prec);
size_t cpl_adjoint_bytes(const CplTab& T, long n, int nsub, int prec);
cudaError_t launch_coupled_vjp(const CplTab& T, long N, int nsub, int prec, int layout, const double* X,
                               const double* U, const double* s, const double* w, const double* rho,
                               double* gX, double* gU, double* gs, double* L, void* ws, size_t ws_bytes,
                               unsigned* status, cudaStream_t st);

}  // namespace ciscvx
