/*
 * ciscvx.h — C ABI of the CI-SCvx discretization/linearization library (GB300, sm_103a).
 *
 * The library computes, for every interval k of a multiple-shooting grid and
 * independently of the other intervals, the integral form of the time-dilated
 * augmented system (Buckner & Elango, Sec. IV-B, Eqs. (14)-(15))
 *
 *     x~(1) = F~(x~_k, U_k, s_k),   d x~ / d tau = s_k (f(x,u), Omega(x,u)),  tau in [0,1],
 *
 * with a first-order-hold control u(tau) = (1 - tau) u_L + tau u_R (Sec. VI),
 * integrated by n_sub classical RK4 steps, and its Jacobian blocks (Internal
 * Numerical Differentiation, Sec. VI)
 *
 *     A_k = dF~/dx~_k,  B-_k = dF~/du_L,  B+_k = dF~/du_R,  S_k = dF~/ds_k,
 *
 * the defects of the dynamics constraint Eq. (17b), defect_k = x~(1) - x~_{k+1},
 * and the increments of the path-constraint penalty states that Eq. (13)
 * bounds, penalty_k = y(1) - y_k.  It also returns the vector-Jacobian product
 * of L = sum_k w_k . defect_k + sum_k rho_k . penalty_k with respect to all
 * node states, controls and dilation factors.
 *
 * Model (Sec. II-A, Eq. (1)): planar links in maximal coordinates, link b has
 * q_b = (p_x, p_y, theta), v_b = (v_x, v_y, omega), mass matrix diag(m, m, I).
 * Revolute joint j (parent p, child c) carries a joint torque tau_j (+tau on
 * the child, -tau on the parent) and a world-frame reaction force
 * lambda_j = (lambda_x, lambda_y) (+lambda on the child at its anchor,
 * -lambda on the parent at its anchor); both are FOH inputs.  Contact i on
 * flat ground y = 0 (normal (0,1), tangent (1,0)) at a body-frame point of one
 * link carries inputs (lambda_n, lambda_t+, lambda_t-): world force
 * (lambda_t+ - lambda_t-, lambda_n).  Gravity acts along -y.  A body-frame
 * point rho sits at p + R(theta) rho, R = [[cos, -sin], [sin, cos]].
 * Auxiliary state (Sec. IV-A, Eq. (12)): one state y_i per contact with
 * y_i' = Omega_i = sum over g in (-lambda_n, -lambda_t+, -lambda_t-, -phi_i(q),
 * lambda_t+ + lambda_t- - mu lambda_n) of h(g), h(z) = sqrt(1 + max(z,0)^2) - 1,
 * phi_i the signed distance of the contact point to the ground.
 *
 * Layouts (row-major, FP64 unless stated):
 *   state  x~ = (q_1..q_nb, v_1..v_nb, y_1..y_nc),  n_x~ = 6 n_b + n_c
 *   input  u  = (tau_1..tau_nj, lambda_1x, lambda_1y, .., lambda_njx, lambda_njy,
 *                [lambda_n, lambda_t+, lambda_t-] per contact),  n_u = 3 n_j + 3 n_c
 *   X [N+1][n_x~] node states;  s [N] dilation factors
 *   U  CISCVX_FOH_NODE: [N+1][n_u], u_L = U_k, u_R = U_{k+1}
 *      CISCVX_FOH_INTERVAL: [N][2][n_u], (u_L, u_R) per interval (may jump at nodes)
 *   A [N][n_x~][n_x~], Bm/Bp [N][n_x~][n_u], S [N][n_x~]: FP64 for CISCVX_FP64,
 *      FP32 for CISCVX_FP32_PHI
 *   defect [N][n_x~], penalty [N][n_c], z [N][n_x~]: always FP64
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller (unless stated),
 *     valid for the duration of the asynchronous work; the library keeps no
 *     reference to them after the call returns.
 *   - Compute calls are asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and allocate no memory; scratch memory, where an
 *     operation needs it, is a caller-provided workspace sized by
 *     ciscvx_workspace_size().
 *   - Argument errors are reported synchronously by the return value, with a
 *     message from ciscvx_last_error() (thread-local); nothing is launched.
 *   - Errors found on the device (non-finite results) set bits in the
 *     model's/plan's device status word; ciscvx_sync_status() reads and clears it.
 */
#ifndef CISCVX_H_
#define CISCVX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CISCVX_VERSION_MAJOR 0
#define CISCVX_VERSION_MINOR 9

typedef enum {
  CISCVX_OK = 0,
  CISCVX_EINVAL = 1,       /* invalid argument (null pointer, size, index, layout) */
  CISCVX_ENOMEM = 2,       /* host or device allocation failed (create calls only) */
  CISCVX_ECUDA = 3,        /* a CUDA runtime call failed */
  CISCVX_ENONFINITE = 4,   /* the device produced a non-finite state or block */
  CISCVX_ETIMEOUT = 5,     /* reserved: a bounded device wait gave up */
  CISCVX_EUNSUPPORTED = 6  /* valid request outside the library's limits */
} ciscvx_status;

typedef enum {
  CISCVX_FP64 = 0,      /* state, penalty and Phi blocks in FP64 */
  CISCVX_FP32_PHI = 1,  /* Phi blocks (A, B-, B+, S) propagated and stored in FP32;
                           state, defect and penalty stay FP64.  Accuracy is
                           block-normwise (error <= 1e-4 of max|block|, an
                           absolute error on the block's scale): entries far
                           below that scale carry no relative accuracy; use
                           CISCVX_FP64 where small entries matter one by one */
  CISCVX_TF32_TC = 2,   /* reserved: tensor-core Phi products; returns EUNSUPPORTED */
  CISCVX_BF16_TC = 3    /* reserved: tensor-core Phi products; returns EUNSUPPORTED */
} ciscvx_precision;

typedef enum {
  CISCVX_FOH_NODE = 0,     /* U [N+1][n_u]: controls shared by neighbouring intervals */
  CISCVX_FOH_INTERVAL = 1  /* U [N][2][n_u]: per-interval (u_L, u_R) */
} ciscvx_u_layout;

typedef enum {
  CISCVX_OUT_DENSE = 0,   /* A [N][n_x~][n_x~], Bm/Bp [N][n_x~][n_u] (structural zeros stored) */
  CISCVX_OUT_COMPACT = 1  /* A [N][nnz_A], Bm/Bp [N][nnz_B]: structural nonzeros only, in the
                             order of ciscvx_model_pattern; S, defect, penalty, z as for dense */
} ciscvx_out_format;

/* Limits of the library (ciscvx_model_create / ciscvx_discretize_vjp return
 * CISCVX_EUNSUPPORTED beyond them). */
#define CISCVX_MAX_BODIES 32          /* links per model */
#define CISCVX_MAX_INPUTS_PER_BODY 15 /* inputs acting on one link (<= 4 joints + 1 contact) */
#define CISCVX_MAX_VJP_SUBSTEPS 64    /* RK4 substeps per interval in the VJP */

/* ---------------------------------------------------------------- model --- */

typedef struct {
  double mass;     /* > 0 */
  double inertia;  /* rotational inertia about the centre of mass, > 0 */
} ciscvx_body_desc;

typedef struct {
  int parent, child;        /* link indices, distinct, in [0, n_bodies) */
  double rho_parent[2];     /* joint anchor in the parent's body frame */
  double rho_child[2];      /* joint anchor in the child's body frame */
} ciscvx_joint_desc;

typedef struct {
  int body;                 /* link carrying the contact point (at most one contact per link) */
  double rho[2];            /* contact point in the link's body frame */
  double mu;                /* friction coefficient, >= 0 */
} ciscvx_contact_desc;

/* Auxiliary state and contact model.
 *   CISCVX_AUX_PENALTY: contact inputs (lambda_n, lambda_t+, lambda_t-), world
 *     force (lambda_t+ - lambda_t-, lambda_n); one path-penalty state per
 *     contact (n_y = n_c), as described in the file header.
 *   CISCVX_AUX_CROSS: the full auxiliary state of Eq. (12).  Contact inputs
 *     (phi_t, phi_n, gamma): the contact-frame force (phi_t, phi_n) (the world
 *     force on flat ground) and the friction multiplier gamma.  Per contact i
 *     four cross-complementarity states integrating, in this order,
 *       phi_n,  lambda^c = t^T J_c v + gamma phi_t / sqrt(1 + phi_t^2),
 *       gamma,  rho^c = |mu phi_n|~ - |phi_t|~     (|x|~ = sqrt(1 + x^2) - 1),
 *     at y index 4 i .. 4 i + 3, then one path-penalty state per contact at y
 *     index 4 n_c + i integrating h(-phi_n) + h(-phi) + h(-gamma) + h(-rho^c)
 *     (n_y = 5 n_c).  The penalty output is the increment of the path-penalty
 *     states.  Provided for the dense and compact linearization (single
 *     and batch; z formed from the dense outputs, not provided with compact
 *     ones) and the VJP (the per-link discrete adjoint, also inside batch
 *     plans). */
typedef enum { CISCVX_AUX_PENALTY = 0, CISCVX_AUX_CROSS = 1 } ciscvx_aux_model;

/* Joint reaction forces (Sec. II-A).
 *   CISCVX_JOINT_FORCE_INPUT: lambda_j are FOH inputs (n_u = 3 n_j + 3 n_c,
 *     order tau, lambda, contact inputs); the links are then decoupled.
 *   CISCVX_JOINT_FORCE_ELIMINATED: the paper's model.  The joint constraints
 *     C_j = p_c + R_c rho_c - p_p - R_p rho_p are imposed at the acceleration
 *     level, Eq. (3): grad C v' + (v^T Hess C_j v)_j = 0, and with
 *     M v' = W + J_c^T R_c phi + grad C^T lambda this fixes lambda
 *     = K^-1 (kappa - grad C M^-1 (W + J_c^T R_c phi)), K = grad C M^-1 grad C^T,
 *     kappa_j = omega_c^2 r_c - omega_p^2 r_p.  Inputs: n_u = n_j + 3 n_c
 *     (tau, then contact inputs).  Needs a joint forest of at most
 *     CISCVX_NODE_MAX_JOINTS joints with at most CISCVX_NODE_MAX_JOINTS_PER_LINK
 *     on one link (EUNSUPPORTED otherwise). */
typedef enum { CISCVX_JOINT_FORCE_INPUT = 0, CISCVX_JOINT_FORCE_ELIMINATED = 1 } ciscvx_joint_force_model;

/* Integration scheme of the substeps (Sec. VI).  CISCVX_RK4: classical RK4.
 * CISCVX_RKF45: Fehlberg's six-stage 4(5) pair, advanced with its fifth-order
 * weights (fixed steps; the embedded estimate is not formed). */
typedef enum { CISCVX_RK4 = 0, CISCVX_RKF45 = 1 } ciscvx_scheme;

typedef struct {
  int n_bodies, n_joints, n_contacts;
  const ciscvx_body_desc* bodies;       /* [n_bodies] host memory */
  const ciscvx_joint_desc* joints;      /* [n_joints] host memory (may be NULL if 0) */
  const ciscvx_contact_desc* contacts;  /* [n_contacts] host memory (may be NULL if 0) */
  double gravity;                       /* magnitude, acting along -y, finite */
  int aux_model;                        /* CISCVX_AUX_PENALTY or CISCVX_AUX_CROSS */
  int joint_forces;                     /* ciscvx_joint_force_model (0: inputs) */
  int scheme;                           /* ciscvx_scheme (0: RK4) */
  /* Contact surface y = terrain_amp sin(terrain_wavenumber x) (Sec. VI-B);
   * terrain_amp = 0 is flat ground y = 0.  Signed distance phi = h^c /
   * ||grad h^c||, h^c = y - terrain_amp sin(terrain_wavenumber x); contact
   * frame: normal n = grad h^c / ||grad h^c||, tangent t = (n_y, -n_x); the
   * contact-frame force (tangential, normal) acts as t tangential + n normal. */
  double terrain_amp, terrain_wavenumber;
} ciscvx_model_desc;

typedef struct ciscvx_model ciscvx_model;

/* Model of Sec. II-A / Sec. IV-A (see the file header).  Copies the host
 * description, builds the per-link device tables on the current CUDA device
 * and allocates the model's device status word.  A model with eliminated
 * joint forces, a sinusoidal surface or the RKF45 scheme has coupled links:
 * it is linearized by ciscvx_discretize (dense outputs, z formed from them, a
 * workspace from ciscvx_discretize_workspace_size) or in a batch plan
 * (ciscvx_batch_discretize, dense outputs; the plan groups its instances by
 * n_sub and owns their stage-data workspace, and its host executor takes
 * them per instance), and its VJP by the coupled path's reverse-mode adjoint
 * (single instance, and in batch plans, where the fused pass runs the
 * linearization and the VJP as two calls).  Its compact outputs return
 * CISCVX_EUNSUPPORTED.  *out receives an opaque
 * handle owned by the caller (free with ciscvx_model_destroy).  Errors:
 * EINVAL (null, counts < 0, n_bodies < 1, bad indices, non-positive mass or
 * inertia, parent == child, non-finite values), EUNSUPPORTED (limits above,
 * two contacts on one link), ENOMEM / ECUDA (allocation). */
ciscvx_status ciscvx_model_create(const ciscvx_model_desc* desc, ciscvx_model** out);

/* Frees the model's device tables.  NULL is a no-op.  No work using the model
 * may be in flight. */
void ciscvx_model_destroy(ciscvx_model* model);

/* n_x = 6 n_b (x~ without the auxiliary states), n_y = n_c (CISCVX_AUX_CROSS:
 * 5 n_c), n_u = 3 n_j + 3 n_c (eliminated joint forces: n_j + 3 n_c).
 * Any output pointer may be NULL.  EINVAL on a null model. */
ciscvx_status ciscvx_model_dims(const ciscvx_model* model, int* n_x, int* n_y, int* n_u);

/* Structural nonzero pattern of A_k and of B-_k / B+_k (shared by both) for
 * the model `desc` describes.  Host computation only: needs no GPU and no
 * model handle.  The dynamics of Sec. II-A couple the links only through the
 * joint forces, which are inputs, so A_k is block diagonal per link (plus the
 * row of the contact's penalty state), and input q enters only the rows of
 * the links it acts on.  The pattern holds every entry that can be nonzero
 * for some (x~, U, s); entries outside it are exactly zero for all inputs.
 * (On a link that no input acts on, (om,th) is in the pattern but always 0.)
 * Compact outputs (CISCVX_OUT_COMPACT) store, per interval, the values of the
 * pattern's entries in this order:
 *   A: for each link b in order: (px,px) (px,vx) (py,py) (py,vy) (th,th)
 *      (th,om) (vx,vx) (vy,vy) (om,th) (om,om), then, if a contact sits on
 *      b, (y,py) (y,th) (y,vy) (y,om) (y,y); px/py/th = rows 3b, 3b+1, 3b+2,
 *      vx/vy/om = rows 3n_b + 3b + (0, 1, 2), y = the contact's path-penalty
 *      row (6n_b + contact index; CISCVX_AUX_CROSS: 6n_b + 4n_c + contact
 *      index); CISCVX_AUX_CROSS then adds, for the contact's rows
 *      c0..c3 = 6n_b + 4 (contact index) + (0..3) (phi_n, lambda^c, gamma,
 *      rho^c): (c0,c0) (c1,c1) (c2,c2) (c3,c3) (c1,vx) (c1,th) (c1,om);
 *   B: for each link b in order, for each input q acting on b (for each
 *      joint j in increasing index that has b as parent or child: tau_j,
 *      lambda_jx, lambda_jy; then, if a contact sits on b, its contact
 *      inputs in order): (px,q) if q has an x force component, (py,q) if a
 *      y component, (th,q) if q exerts a torque on b, (vx,q) if x, (vy,q) if
 *      y, (om,q) if a torque, then (y,q) if a contact sits on b;
 *      CISCVX_AUX_CROSS then adds, after the groups of a foot link, (c1,q)
 *      for each of its inputs in the same order that has an x component or
 *      a torque or is phi_t or gamma, then (c0,phi_n) (c2,gamma) (c3,phi_t)
 *      (c3,phi_n).  (gamma exerts no force: it has only the (y,gamma),
 *      (c1,gamma) and (c2,gamma) entries.)
 * A model with coupled links (joint forces eliminated, RKF45 or the
 * sinusoidal surface) has this pattern instead, column-major: for each
 * column c of A in order, every row r (ascending) when c is integrated by
 * the coupled path (theta and omega of every link, every state of a link
 * with a contact), else (c - 3n_b, c) (c) for the linear velocity of a link
 * without a contact and (c,c) for its position and for the auxiliary rows;
 * B: for each input q in order, every row.
 * Call with NULL arrays to get the counts; then a_row/a_col receive nnz_A
 * and b_row/b_col nnz_B int32 indices (host memory, caller-owned).  Any of
 * nnz_a, nnz_b may be NULL.  Errors: as ciscvx_model_create for the
 * description (EINVAL, EUNSUPPORTED). */
ciscvx_status ciscvx_model_pattern(const ciscvx_model_desc* desc, int* nnz_a, int* nnz_b,
                                   int32_t* a_row, int32_t* a_col, int32_t* b_row,
                                   int32_t* b_col);

/* Pattern sizes of a created model (as ciscvx_model_pattern).  EINVAL on a null model. */
ciscvx_status ciscvx_model_nnz(const ciscvx_model* model, int* nnz_a, int* nnz_b);

/* ------------------------------------------------------------ workspace --- */

typedef enum { CISCVX_OP_DISCRETIZE = 0, CISCVX_OP_VJP = 1 } ciscvx_op;

/* Bytes of device scratch memory that `op` needs for N intervals (0 if none).
 * EINVAL on null pointers, N < 1 or an unknown op/layout.  Where the scratch
 * depends on n_sub and the precision (CISCVX_OP_DISCRETIZE for a model with
 * coupled links; CISCVX_OP_VJP for one with coupled links) it returns
 * EUNSUPPORTED: use ciscvx_discretize_workspace_size. */
ciscvx_status ciscvx_workspace_size(const ciscvx_model* model, ciscvx_op op, int N,
                                    ciscvx_u_layout layout, size_t* bytes);

/* Scratch of `op` for N intervals of n_sub substeps in `precision` and
 * `layout`: *min_bytes (the least the call accepts) and *full_bytes (enough
 * to treat all N intervals at once); a workspace between the two is used in
 * chunks of as many intervals as fit.
 *   CISCVX_OP_DISCRETIZE: 0 and 0 for models without coupled links; for a
 *     model with coupled links the stage data of the nominal trajectory
 *     (n_sub x stages x (4 n_j + n_b + n_x~ + skyline(K) + contact fields)
 *     values per interval in the precision's dtype), minimum 32 intervals.
 *   CISCVX_OP_VJP: for a model without coupled links (either auxiliary
 *     model) min = full = ciscvx_workspace_size(CISCVX_OP_VJP); for a model
 *     with coupled links the coupled adjoint's stage data and cotangents per
 *     interval, minimum 32 intervals.
 * Either pointer may be NULL.  EINVAL on a null model, N < 1, n_sub < 1 or an
 * unknown op, precision or layout. */
ciscvx_status ciscvx_discretize_workspace_size(const ciscvx_model* model, ciscvx_op op, int N,
                                               int n_sub, ciscvx_precision precision,
                                               ciscvx_u_layout layout, size_t* min_bytes,
                                               size_t* full_bytes);

/* ----------------------------------------------------------- discretize --- */

/* Linearized discretization of Eqs. (14)-(15) and (17b) on every interval
 * k = 0..N-1 (see the file header for what is computed and all layouts).
 *   X [N+1][n_x~], U per `layout`, s [N]: inputs (FP64, device).
 *   A, Bm, Bp, S: outputs in the dtype of `precision` (device); A and S are
 *     required; Bm/Bp may be NULL only when n_u == 0.
 *   defect [N][n_x~], penalty [N][n_c]: FP64 outputs (device); penalty may be
 *     NULL when n_c == 0.
 *   z: optional FP64 affine term z_k = x~(1) - A x~_k - B- u_L - B+ u_R - S s_k
 *     (NULL to skip).
 *   workspace/ws_bytes: ignored (pass NULL, 0) unless the model has coupled
 *     links; then device scratch of at least the minimum of
 *     ciscvx_discretize_workspace_size, 16-byte aligned (contents overwritten).
 *     Such models run two kernels per chunk of intervals: the nominal
 *     trajectory in FP64 (one lane per interval, with the per-stage L D L^T
 *     solve of Eq. (3)), then one tangent column per thread in the
 *     precision's dtype.
 *   For a model with coupled links or the Eq. (12) auxiliary state, z is
 *   formed from the stored outputs by a post-pass.
 * Errors: EINVAL (nulls, N < 1, n_sub < 1, unknown layout/precision),
 * EUNSUPPORTED (tensor-core precisions), EINVAL also for a missing or short
 * workspace of a model with coupled links, ECUDA (launch failure). */
ciscvx_status ciscvx_discretize(const ciscvx_model* model, int N, int n_sub,
                                ciscvx_precision precision, ciscvx_u_layout layout,
                                const double* X, const double* U, const double* s, void* A,
                                void* Bm, void* Bp, void* S, double* defect, double* penalty,
                                double* z, void* workspace, size_t ws_bytes, void* stream);

/* ciscvx_discretize with compact A, Bm, Bp (CISCVX_OUT_COMPACT): A [N][nnz_A],
 * Bm/Bp [N][nnz_B] in the precision's dtype, values in ciscvx_model_pattern's
 * order; every other argument as for ciscvx_discretize (workspace: needed by a
 * model with coupled links only, as there; may be NULL otherwise).  The values
 * are those ciscvx_discretize stores at the pattern's positions (same
 * arithmetic), and no structural zero is written.  For a model with coupled
 * links the pattern is column-major: the columns the coupled path integrates
 * are full (every row), the closed-form ones keep their one or two entries
 * (A e_p = e_p, A e_v = e_v + s e_p for a link without a contact, A e_y =
 * e_y), and B-/B+ are full, column by column.  For the Eq. (12) model and
 * for coupled links z is formed by a post-pass over the compact values and
 * the pattern by rows.  Errors: as ciscvx_discretize. */
ciscvx_status ciscvx_discretize_compact(const ciscvx_model* model, int N, int n_sub,
                                        ciscvx_precision precision, ciscvx_u_layout layout,
                                        const double* X, const double* U, const double* s,
                                        void* A, void* Bm, void* Bp, void* S, double* defect,
                                        double* penalty, double* z, void* workspace,
                                        size_t ws_bytes, void* stream);

/* Vector-Jacobian product of L = sum_k w_k . defect_k + sum_k rho_k . penalty_k
 * (defect and penalty as above) with respect to X, U and s, by the discrete
 * adjoint of the RK4 substeps with the state checkpointed at every substep
 * start and the stages recomputed.  For a model with coupled links (Eq. (3)
 * elimination, RKF45, the sinusoidal surface; with either auxiliary model)
 * by the reverse-mode adjoint of the coupled path: per chunk of intervals the
 * FP64 nominal pass records its stage data in the workspace, then one thread
 * per interval runs the transposed stage maps backward; no block is formed.
 * For a per-link model with the Eq. (12) auxiliary state (CISCVX_AUX_CROSS)
 * the per-link adjoint covers each contact's four cross-complementarity rows
 * and its path penalty: lambda^c's integrand v_x - omega (R rho)_y puts
 * sources on the stage theta, omega and v_x of the backward sweep, and the
 * rows that integrate the inputs alone contribute their quadrature weights
 * times the slopes; scratch and substep limit as for the default model.
 *   w [N][n_x~], rho [N][n_c] (FP64, device; rho may be NULL when n_c == 0).
 *   gX [N+1][n_x~], gU like U, gs [N]: FP64 outputs (device), overwritten.
 *   L: optional FP64 scalar on the device (NULL to skip).
 *   precision: CISCVX_FP64 (adjoint in FP64) or CISCVX_FP32_PHI (adjoint
 *     cotangents in FP32; the checkpointed state stays FP64).
 *   workspace: device scratch of at least ciscvx_workspace_size(CISCVX_OP_VJP)
 *     bytes, 16-byte aligned; its contents are overwritten.
 * Errors: as ciscvx_discretize, plus EINVAL for a missing/short workspace and
 * EUNSUPPORTED for n_sub > CISCVX_MAX_VJP_SUBSTEPS. */
ciscvx_status ciscvx_discretize_vjp(const ciscvx_model* model, int N, int n_sub,
                                    ciscvx_precision precision, ciscvx_u_layout layout,
                                    const double* X, const double* U, const double* s,
                                    const double* w, const double* rho, double* gX, double* gU,
                                    double* gs, double* L, void* workspace, size_t ws_bytes,
                                    void* stream);

/* ---------------------------------------------------------------- batch --- */
/*
 * Many independent problem instances (different robots, horizons N and
 * substep counts, e.g. random restarts or homotopy sweeps) linearized by one
 * persistent launch.  A plan fixes the instances and packs their arrays back
 * to back in instance order: instance i's X starts at element offset
 * sum_{j<i} (N_j + 1) n_x~_j of the packed X buffer, and likewise for every
 * other array (ciscvx_batch_offsets gives each instance's offsets,
 * ciscvx_batch_sizes the buffer lengths).  Within an instance the layouts are
 * those of ciscvx_discretize / ciscvx_discretize_vjp.
 *
 * Work decomposition: intervals of instances that share (model, n_sub) are
 * grouped 32 at a time (a group may span instances), one group x one link is a
 * work item for one warp, and items are ordered by estimated cost, largest
 * first.  A persistent grid pulls items from a device counter.  The launch
 * sequence (counter reset + kernel) is captured once into a CUDA graph per
 * set of buffers and replayed.
 */

typedef struct ciscvx_batch_plan ciscvx_batch_plan;

/* Launch shape of the batched kernels (chosen by ciscvx_batch_autotune or given). */
typedef struct {
  int warps_per_cta;  /* 1, 2, 4 or 8 */
  int ctas_per_sm;    /* > 0: persistent grid of ctas_per_sm x SMs CTAs pulling items from a
                         queue; 0: one warp per work item */
  int lpt_order;      /* 1: items ordered by decreasing estimated cost; 0: instance order;
                         2 (persistent grids): two queues, the foot-link items and the others,
                         each in instance order, a share of the SMs (by estimated cost) taking
                         each, with the other queue taken over once the own one is empty */
  int use_graph;      /* 1: capture the launch sequence in a CUDA graph and replay it */
  int occupancy;      /* register cap of the kernels: 0 none (8 warps/SM), 1 <= 168 registers
                         (12 warps/SM), 2 <= 128 registers (16 warps/SM); 1 and 2 need
                         warps_per_cta <= 4 */
  int split;          /* fused linearization + VJP only (ciscvx_batch_discretize_and_vjp):
                         0 one warp per work item takes the linearization and the adjoint in
                         turn, sharing the integrated trajectory; 1 the linearization and the
                         adjoint of each item run on two warps of the same launch, each
                         integrating the trajectory itself (more work, but half the path per
                         warp: for batches too small to fill the GPU, where one warp's
                         instruction stream sets the time).  1 needs occupancy 0.  The other
                         entry points ignore it. */
} ciscvx_tune;

/* Element counts of the packed buffers (or, from ciscvx_batch_offsets, the
 * element offsets of one instance inside them).  A/Bm/Bp/S in the plan's Phi
 * dtype; everything else FP64.  L has one element per instance.  With compact
 * outputs an instance's A holds N nnz_A values and its Bm/Bp N nnz_B. */
typedef struct {
  size_t X, U, s, A, B, S, defect, penalty, L;
} ciscvx_batch_sizes;

typedef struct {
  const double* X;   /* packed inputs (device) */
  const double* U;
  const double* s;
  void* A;           /* packed outputs (device); Bm/Bp may be NULL only if every n_u == 0 */
  void* Bm;
  void* Bp;
  void* S;
  double* defect;
  double* penalty;   /* may be NULL only if every n_c == 0 */
} ciscvx_batch_io;

typedef struct {
  const double* X;   /* packed inputs (device) */
  const double* U;
  const double* s;
  const double* w;   /* cotangents, packed like defect */
  const double* rho; /* packed like penalty */
  double* gX;        /* packed like X */
  double* gU;        /* packed like U */
  double* gs;        /* packed like s */
  double* L;         /* [n_inst] per-instance L, or NULL */
} ciscvx_batch_vjp_io;

/* Builds the work decomposition for n_inst instances: instance i uses
 * models[model_idx[i]] with N[i] intervals and n_sub[i] substeps.  All arrays
 * are host memory, copied; the models must outlive the plan and live on the
 * current device.  format: dense or compact A/Bm/Bp for every instance.  tune may be NULL (defaults: 4 warps/CTA, persistent with
 * 2 CTAs/SM, cost order, graph, no register cap).  Allocates the plan's device tables (this
 * is the only allocating batch call besides autotuning's timing buffers).
 * Errors: EINVAL (nulls, n_inst < 1, bad indices, N < 1, n_sub < 1, layout,
 * precision, format), EUNSUPPORTED (tensor-core precisions), ENOMEM/ECUDA. */
ciscvx_status ciscvx_batch_plan_create(const ciscvx_model* const* models, int n_models,
                                       const int* model_idx, const int* N, const int* n_sub,
                                       int n_inst, ciscvx_precision precision,
                                       ciscvx_u_layout layout, ciscvx_out_format format,
                                       const ciscvx_tune* tune, ciscvx_batch_plan** out);

/* Frees the plan (no work using it may be in flight).  NULL is a no-op. */
void ciscvx_batch_plan_destroy(ciscvx_batch_plan* plan);

/* Lengths (elements) of the packed buffers. */
ciscvx_status ciscvx_batch_sizes_get(const ciscvx_batch_plan* plan, ciscvx_batch_sizes* out);

/* Element offsets of instance `inst` inside the packed buffers. */
ciscvx_status ciscvx_batch_offsets(const ciscvx_batch_plan* plan, int inst, ciscvx_batch_sizes* out);

/* Current launch shape of the plan. */
ciscvx_status ciscvx_batch_get_tune(const ciscvx_batch_plan* plan, ciscvx_tune* out);

/* Linearized discretization (as ciscvx_discretize) of every interval of every
 * instance, asynchronously on `stream`.  With use_graph the first call for a
 * given io captures the launch sequence into a graph (on a private stream of
 * the plan) and every call replays it on `stream`; make that first call
 * outside any capture of your own.  Errors: EINVAL (null io or required
 * pointer), ECUDA. */
ciscvx_status ciscvx_batch_discretize(ciscvx_batch_plan* plan, const ciscvx_batch_io* io,
                                      void* stream);

/* Bytes of device scratch ciscvx_batch_discretize_vjp needs (the minimum). */
ciscvx_status ciscvx_batch_vjp_workspace_size(const ciscvx_batch_plan* plan, size_t* bytes);

/* The minimum and the full size of that scratch; the two are equal (the
 * coupled instances' adjoint takes the minimum's chunked form). */
ciscvx_status ciscvx_batch_vjp_workspace_sizes(const ciscvx_batch_plan* plan, size_t* min_bytes,
                                               size_t* full_bytes);

/* VJP (as ciscvx_discretize_vjp) of every instance; L receives one value per
 * instance.  Per-link instances (either auxiliary model) take the batched
 * adjoint kernel; instances with coupled links then take the coupled path's
 * reverse-mode adjoint one after another in stream order (chunked in the last
 * part of the workspace).  workspace: device, >= ciscvx_batch_vjp_workspace_size
 * bytes, 16-byte aligned.  Errors: EINVAL, EUNSUPPORTED (n_sub >
 * CISCVX_MAX_VJP_SUBSTEPS in some per-link instance), ECUDA. */
ciscvx_status ciscvx_batch_discretize_vjp(ciscvx_batch_plan* plan, const ciscvx_batch_vjp_io* io,
                                          void* workspace, size_t ws_bytes, void* stream);

/* ciscvx_batch_discretize and ciscvx_batch_discretize_vjp of the same inputs
 * in one pass.  The adjoint's backward sweep needs the FP64 state at every
 * substep start, which the linearization computes anyway: here the
 * linearization records it and the backward sweep starts from it, so each
 * interval's trajectory is integrated once instead of twice.  Outputs are
 * those of the two calls (io's A..penalty; vjp's gX, gU, gs, L), equal to
 * them to rounding.  vjp->X, U, s are ignored (io's inputs are used).
 * workspace as for ciscvx_batch_discretize_vjp.  Launched directly (no graph).
 * With the fused tune's split = 1 (small batches) the two run on separate
 * warps of the same launch, each integrating the trajectory, as the two calls
 * would.  Coupled-link instances take one nominal pass per chunk for both
 * (its stage data feed the tangent kernel and the adjoint), in the coupled
 * part of the workspace.  Errors: as the two calls. */
ciscvx_status ciscvx_batch_discretize_and_vjp(ciscvx_batch_plan* plan, const ciscvx_batch_io* io,
                                              const ciscvx_batch_vjp_io* vjp, void* workspace,
                                              size_t ws_bytes, void* stream);

/* Times candidate launch shapes of ciscvx_batch_discretize on the given
 * buffers (their outputs are overwritten), keeps the fastest in the plan and
 * returns it in *chosen (may be NULL).  Results are cached per process by
 * (models' topology, substep counts, precision, device name); a cached choice
 * is reused without timing.  Synchronizes `stream`.  Errors: as
 * ciscvx_batch_discretize. */
ciscvx_status ciscvx_batch_autotune(ciscvx_batch_plan* plan, const ciscvx_batch_io* io,
                                    void* stream, ciscvx_tune* chosen);

/* End-to-end run on HOST buffers, pipelined: the instances are split into
 * n_chunks consecutive chunks of balanced cost; for each chunk the inputs are
 * copied host -> device, the chunk is linearized (with its VJP in the same
 * pass, as ciscvx_batch_discretize_and_vjp, if host_vjp is not NULL), and its
 * outputs are copied device -> host, on three
 * plan-owned streams so that one chunk's copies overlap its neighbours'
 * compute.  The call is asynchronous: `stream` waits for the last copy.
 *   host: packed host arrays in the layout of ciscvx_batch_io (inputs X, U, s;
 *     outputs A, Bm, Bp, S, defect, penalty); pinned memory lets the copies
 *     overlap (pageable memory still gives correct results).
 *   dev: device buffers of the full packed sizes, used as staging.
 *   host_vjp / dev_vjp: NULL, or the VJP cotangents (w, rho: host inputs) and
 *     gradients (gX, gU, gs, L: host outputs) with their device buffers; their
 *     X, U, s fields are ignored (host/dev are used).  workspace as for
 *     ciscvx_batch_discretize_vjp (with coupled-link instances at least the
 *     minimum of ciscvx_batch_vjp_workspace_sizes).
 * Coupled-link instances are linearized one after another within their
 * chunk (and their VJP taken by the coupled path's reverse-mode adjoint).

 * The first call with a new n_chunks builds the chunked work tables and
 * streams (device allocation); later calls with the same n_chunks allocate
 * nothing.  Errors: EINVAL (null buffers, n_chunks outside [1, n_inst], short
 * workspace), EUNSUPPORTED (VJP with n_sub > CISCVX_MAX_VJP_SUBSTEPS), ECUDA. */
ciscvx_status ciscvx_batch_run_host(ciscvx_batch_plan* plan, int n_chunks,
                                    const ciscvx_batch_io* host, const ciscvx_batch_io* dev,
                                    const ciscvx_batch_vjp_io* host_vjp,
                                    const ciscvx_batch_vjp_io* dev_vjp, void* workspace,
                                    size_t ws_bytes, void* stream);

/* As ciscvx_batch_autotune, for the fused pass of ciscvx_batch_discretize_and_vjp
 * (its launch shape is kept apart from the discretization's: the fused kernel
 * holds more state per thread).  When the fused pass would run at most one
 * warp per scheduler (work items <= 4 x SMs), the split form (tune.split = 1,
 * one warp per item, 1, 2 or 4 warps per CTA) is among the candidates.
 * Overwrites the outputs; workspace as for ciscvx_batch_discretize_vjp.
 * Errors: as ciscvx_batch_discretize_and_vjp. */
ciscvx_status ciscvx_batch_autotune_fused(ciscvx_batch_plan* plan, const ciscvx_batch_io* io,
                                          const ciscvx_batch_vjp_io* vjp, void* workspace,
                                          size_t ws_bytes, void* stream, ciscvx_tune* chosen);

/* Current launch shape of the plan's fused pass. */
ciscvx_status ciscvx_batch_get_tune_fused(const ciscvx_batch_plan* plan, ciscvx_tune* out);

/* As ciscvx_sync_status, for the plan's status word. */
ciscvx_status ciscvx_batch_sync_status(const ciscvx_batch_plan* plan, void* stream);

/* ----------------------------------------------------- node constraints --- */
/*
 * The constraints the transcription imposes at every grid node k = 0..n-1
 * (Sec. IV-C, Eqs. (17e)-(17f)), for pre-impact state x~-_k, post-impact
 * state x~+_k, contact impulses Phi_k and impulse multipliers Gamma_k:
 *
 *   G~(x~+, x~-, Phi) = 0: the impact map of Eq. (6a) with the joint impulse
 *     eliminated by the post-impact joint constraint grad C v+ = 0 (Sec. II-B):
 *       rows q:  q+ - q-                                       (3 n_b)
 *       rows v:  M (v+ - v-) - J_c^T Phi + grad C^T mu,         (3 n_b)
 *                mu = K^-1 grad C (v- + M^-1 J_c^T Phi),  K = grad C M^-1 grad C^T
 *       rows y:  y+ - y-                                       (n_c)
 *     with M = diag(m, m, I) per link, J_c the contact-point Jacobians, and
 *     every kinematic quantity at the pre-impact pose q-.  On flat ground the
 *     contact-frame impulse (Phi_t, Phi_n) is the world impulse.
 *   Theta^delta(x+, x-, Phi, Gamma) <= 0: per contact i, 8 rows, the
 *     Fischer-Burmeister relaxation FB(a,b) = a + b - sqrt(a^2 + b^2 + delta)
 *     (Eq. (16)) of the impulse conditions Eqs. (6b)-(6e), then the sign
 *     conditions that go with them:
 *       FB(Phi_n, phi), FB(Phi_n, |c|~), FB(Phi_n, |lambda^c|~), FB(Gamma, rho),
 *       -Phi_n, -phi, -Gamma, -rho,
 *     phi the signed distance of the contact point (at q-), c = its normal
 *     velocity under v+ plus e_i times that under v- (Eq. (6c)),
 *     lambda^c = its tangential velocity under v+ + Gamma Phi_t / sqrt(1 + Phi_t^2)
 *     (Eq. (6d)), rho = |mu Phi_n|~ - |Phi_t|~ (Eq. (6e)), and
 *     |x|~ = sqrt(1 + x^2) - 1 the pseudo-Huber absolute value (norm).
 *     "Phi_n times a signed quantity = 0" (Eqs. (6c), (6d)) is relaxed as the
 *     complementarity of Phi_n with the quantity's pseudo-Huber magnitude.
 *
 * The constraint between consecutive nodes, Psi (Eq. (17c)), is
 * ciscvx_psi_linearize below.
 */

/* Theta rows per contact, and the local variables its Jacobian is taken in. */
#define CISCVX_NODE_THETA_ROWS 8
#define CISCVX_NODE_THETA_COLS 12
/* Joints per model, and joints attached to one link, the node kernel supports. */
#define CISCVX_NODE_MAX_JOINTS 12
#define CISCVX_NODE_MAX_JOINTS_PER_LINK 8

typedef struct {
  double delta;               /* Fischer-Burmeister relaxation, finite, > 0 */
  const double* restitution;  /* [n_c] host memory: e_i >= 0 finite (NULL if n_c == 0) */
} ciscvx_node_params;

/* Node constraints and their Jacobians at n_nodes nodes (lane = node; FP64).
 *   Xp, Xm [n][n_x~]: post- and pre-impact states; Phi [n][2 n_c] impulses
 *     (Phi_t, Phi_n) per contact; Gam [n][n_c] multipliers (device; Phi and
 *     Gam may be NULL when n_c == 0).
 *   g [n][n_x~]: G~ (device, required).
 *   Jacobian blocks of G~ (device; each may be NULL to skip it):
 *     Gvm  [n][3 n_b][3 n_b]: d(v rows)/d v-   (symmetric: -M P)
 *     Gth  [n][3 n_b][n_b]  : d(v rows)/d theta-_b (the other pose
 *                             coordinates do not enter the v rows)
 *     Gphi [n][3 n_b][2 n_c]: d(v rows)/d Phi
 *     Gpx  [n][3 n_b][n_c]  : d(v rows)/d p_x- of the link carrying each
 *                             contact (the contact frame moves with the
 *                             contact point on a sinusoidal surface; 0 on
 *                             flat ground)
 *   On a sinusoidal surface the impulse acts as t Phi_t + n Phi_n with the
 *   contact frame at the pre-impact contact point, and phi, c and lambda^c
 *   below use that frame (phi = h^c / ||grad h^c||; velocities projected on
 *   n and t).
 *   The remaining blocks are constant and not stored: d(q rows)/dq+ = I,
 *   d(q rows)/dq- = -I, d(v rows)/dv+ = M, d(y rows)/dy+ = I,
 *   d(y rows)/dy- = -I, all others 0 (G~ does not depend on Gamma).
 *   theta [n][n_c][8]: Theta^delta (device; required when n_c > 0).
 *   dtheta [n][n_c][8][12] (device, may be NULL): each contact's rows
 *     differentiated in the local variables of the link carrying it, in the
 *     order (p_x-, p_y-, theta-, v_x+, v_y+, omega+, v_x-, v_y-, omega-,
 *     Phi_t, Phi_n, Gamma); Theta's derivatives in every other variable are 0
 *     (on flat ground the p_x- and v_x- columns are 0 too).
 * Errors: EINVAL (nulls, n_nodes < 1, delta or restitution invalid),
 * EUNSUPPORTED (more than CISCVX_NODE_MAX_JOINTS joints or more than
 * CISCVX_NODE_MAX_JOINTS_PER_LINK on one link, or a link that is the child of
 * two joints: the joint graph must be a forest), ECUDA. */
ciscvx_status ciscvx_node_linearize(const ciscvx_model* model, int n_nodes, const double* Xp,
                                    const double* Xm, const double* Phi, const double* Gam,
                                    const ciscvx_node_params* params, double* g, double* Gvm,
                                    double* Gth, double* Gphi, double* Gpx, double* theta,
                                    double* dtheta, void* stream);

/* ------------------------------------------ interval-node constraints --- */
/*
 * Psi^{delta,eps}(y-_{k+1}, y+_k) <= 0 (Sec. IV-C, Eq. (17c)) on the N grid
 * intervals between N+1 nodes, for the auxiliary-state increment
 * d_k = y-_{k+1} - y+_k (pre-impact state at the interval's end minus
 * post-impact state at its start; y = the last n_y entries of x~):
 *   CISCVX_AUX_CROSS (n_psi = 3 n_c): per contact i the integral
 *     cross-complementarity of Eq. (11) on the Eq. (12) pairs, relaxed by
 *     Eq. (16) with FB(a, b) = a + b - sqrt(a^2 + b^2 + delta):
 *       row 2i       FB(d[4i], d[4i+1])      (phi_n, lambda^c)
 *       row 2i+1     FB(d[4i+2], d[4i+3])    (gamma, rho^c)
 *     then the relaxed path constraints of Eq. (13):
 *       row 2 n_c + i   d[4 n_c + i] - epsilon;
 *     the nonnegativity of the increments comes from the path penalty (the
 *     integrands' sign constraints), as the paper prescribes, and the pair
 *     (phi_n, signed distance) has no state to pair (no auxiliary state
 *     integrates the signed distance).
 *   CISCVX_AUX_PENALTY (n_psi = n_c): row i = d[i] - epsilon.
 */

/* n_psi of the model: 3 n_c (CISCVX_AUX_CROSS) or n_c. */
ciscvx_status ciscvx_psi_rows(const ciscvx_model* model, int* n_psi);

/* Psi and its Jacobian at N intervals (one thread per interval and contact; FP64).
 *   Xp, Xm [N+1][n_x~]: post- and pre-impact node states (device; only their
 *     y entries are read: y+ of nodes 0..N-1, y- of nodes 1..N).
 *   psi [N][n_psi] (device, required when n_psi > 0).
 *   dpsi [N][n_psi][n_y] (device, may be NULL): d Psi_k / d y-_{k+1}; the
 *     Jacobian in y+_k is its negative, in every other variable 0.
 * Asynchronous on `stream`; a non-finite Psi sets the model's status word
 * (ciscvx_sync_status).  n_psi == 0 (no contacts) is a no-op.
 * Errors: EINVAL (null model, N < 1, delta not finite > 0, epsilon not
 * finite >= 0, null Xp/Xm/psi), ECUDA. */
ciscvx_status ciscvx_psi_linearize(const ciscvx_model* model, int N, const double* Xp,
                                   const double* Xm, double delta, double epsilon, double* psi,
                                   double* dpsi, void* stream);

/* ---------------------------------------------- SOCP canonicalization --- */
/*
 * The convex subproblem of one prox-linear SCP iteration (Sec. V: linearized
 * nonconvex constraints under an exact l1 penalty, convex constraints kept,
 * quadratic proximal term) assembled on the GPU in the canonical SOCP form
 * of a conic interior-point solver (Sec. VI: CSC matrices, row-wise
 * normalization, affine variable scaling):
 *
 *   minimize 1/2 z^T P z + c^T z   s.t.   A z = b,   h - G z in R+^l x Q^2 x ... x Q^2
 *
 * (Q^2 = {(s0, s1): s0 >= |s1|}), for the CITO problem of Eq. (17) at an
 * iterate zbar, on N intervals between N+1 nodes.
 *
 * Variables, period k = 0..N (node part, then, for k < N, interval part):
 *   x~-_k [n_x~], x~+_k [n_x~], Phi_k [2 n_c], Gamma_k [n_c],
 *   u_k [n_u] (CISCVX_FOH_NODE only), nuG+_k, nuG-_k [n_x~ each], tTheta_k [8 n_c];
 *   u_L,k, u_R,k [n_u each] (CISCVX_FOH_INTERVAL only), s_k [1],
 *   nuF+_k, nuF-_k [n_x~ each], tPsi_k [n_psi].
 * nu and t are the penalty slacks ("slack" columns); the rest are the
 * problem's variables.
 *
 * Equality rows, period k: G~ rows of node k [n_x~]
 *     J_G (z - zbar) + G~(zbar) - nuG+ + nuG- = 0;
 *   dynamics rows of interval k [n_x~] (k < N), Eq. (17b) linearized
 *     A_k x~+_k + B-_k u_L + B+_k u_R + S_k s_k - x~-_{k+1} - nuF+ + nuF- = b,
 *     b = A_k x~+bar_k + B-_k u_Lbar + B+_k u_Rbar + S_k sbar_k - F~bar_k,
 *     F~bar_k = defect_k + x~+bar_{k+1} (the linearization evaluated with
 *     X = the post-impact states x~+bar), u_L, u_R = u_k, u_{k+1} (node
 *     layout) or u_L,k, u_R,k;
 *   then x-_0 = x_init [n_x] and x+_N = x_final [n_x] (Eq. (17g)).
 * Inequality rows (G z <= h), nonnegative orthant first, period k:
 *   Theta rows of node k [8 n_c]: J_Theta (z - zbar) + Theta(zbar) - tTheta <= 0;
 *   -tTheta <= 0 [8 n_c]; -nuG+ <= 0, -nuG- <= 0 [2 n_x~];
 *   the input rows of u_k (node layout);
 *   for k < N: Psi rows [n_psi]: J_Psi (z - zbar) + Psi(zbar) - tPsi <= 0;
 *   -tPsi <= 0 [n_psi]; -nuF+ <= 0, -nuF- <= 0 [2 n_x~];
 *   s_k <= s_max, -s_k <= -s_min; the input rows of u_L,k then u_R,k
 *   (interval layout);
 *   input rows of one control vector (the set U of Eq. (17d)): per joint
 *   tau_j <= tau_max_j, -tau_j <= tau_max_j [2 n_j]; per contact,
 *   CISCVX_AUX_PENALTY: -lambda_n, -lambda_t+, -lambda_t- <= 0 and
 *   lambda_t+ + lambda_t- - mu lambda_n <= 0 [4]; CISCVX_AUX_CROSS:
 *   -gamma <= 0 [1].
 * Then, CISCVX_AUX_CROSS only, one Q^2 block per control vector (in the
 * order above) and contact: (mu phi_n, phi_t), i.e. G rows -mu e_phi_n and
 * -e_phi_t, h = 0: the friction cone |phi_t| <= mu phi_n.
 *
 * Objective: P = w_px on the diagonal of every problem variable plus the
 * torque cost w_torque * sum_k integral_0^1 |tau(t)|^2 dt of the FOH
 * torques ((|a|^2 + a.b + |b|^2) / 3 per interval, a, b its end values);
 * c = -w_px zbar on problem variables, w_ep on slack columns.
 *
 * Scaling: problem variables z = D zhat + o with per-component scale and
 * offset (x~ for x~- and x~+, u, s, Phi, Gamma; identity by default);
 * slacks unscaled.  A <- A D, b <- b - A o, G <- G D, h <- h - G o,
 * P <- D P D, c <- D (P o + c).  Then every equality and nonnegative row is
 * multiplied by rho = 1 / (max |entry| over its problem-variable columns)
 * (rho = 1 when there is none or it is 0), and each Q^2 block by the
 * smallest rho of its two rows; rho is returned per row.
 */

typedef struct ciscvx_socp ciscvx_socp;

typedef struct {
  double w_px;                 /* proximal weight, finite > 0 */
  double w_ep;                 /* exact-penalty weight, finite > 0 */
  double w_torque;             /* torque-cost weight, finite >= 0 */
  double s_min, s_max;         /* 0 <= s_min <= s_max, finite */
  const double* torque_max;    /* [n_j] host, finite > 0 (NULL if n_j == 0) */
  const double* x_init;        /* [n_x] host */
  const double* x_final;       /* [n_x] host */
  /* affine scaling z = D zhat + o; each pair may be NULL (scale 1, offset 0);
   * scales finite > 0, offsets finite */
  const double* scale_x; const double* offset_x;      /* [n_x~] */
  const double* scale_u; const double* offset_u;      /* [n_u] */
  double scale_s, offset_s;                           /* scale_s 0 means 1 */
  const double* scale_phi; const double* offset_phi;  /* [2 n_c] */
  const double* scale_gam; const double* offset_gam;  /* [n_c] */
  /* layout of the A, Bm, Bp inputs of ciscvx_socp_fill: CISCVX_OUT_DENSE, or
   * CISCVX_OUT_COMPACT (their structural nonzeros in ciscvx_model_pattern
   * order, as ciscvx_discretize_compact writes them) */
  int phi_format;
} ciscvx_socp_params;

typedef struct {
  int n_var, n_eq, n_ineq;     /* columns; rows of A; rows of G */
  int n_nonneg;                /* l: the first l rows of G */
  int n_soc;                   /* Q^2 blocks after them (each 2 rows) */
  long long nnz_A, nnz_G, nnz_P;
} ciscvx_socp_dims;

/* Builds the structure (host; the CSC patterns and the source map of every
 * entry, uploaded to the device) for model, N intervals and the control
 * layout.  The node blocks are taken dense (d(v rows)/dp_x- only on a
 * sinusoidal surface; Theta's p_x- and v_x- columns too), the interval blocks
 * at the model's structural pattern where the model has one (joint reaction
 * forces as inputs, one penalty state per contact: ciscvx_model_pattern),
 * dense otherwise.
 * Errors: EINVAL (nulls, N < 1, params invalid), EUNSUPPORTED (more than
 * 2^31 - 1 entries in a matrix; compact inputs for a model without a
 * pattern), ENOMEM, ECUDA. */
ciscvx_status ciscvx_socp_create(const ciscvx_model* model, int N, int layout,
                                 const ciscvx_socp_params* params, ciscvx_socp** out);
void ciscvx_socp_destroy(ciscvx_socp* socp);
ciscvx_status ciscvx_socp_get_dims(const ciscvx_socp* socp, ciscvx_socp_dims* dims);

/* The CSC index arrays and P's values (host buffers, any may be NULL):
 * *_colptr [n_var + 1], *_rowind [nnz]; rows sorted within a column; P holds
 * its upper triangle. */
ciscvx_status ciscvx_socp_structure(const ciscvx_socp* socp, int* A_colptr, int* A_rowind,
                                    int* G_colptr, int* G_rowind, int* P_colptr, int* P_rowind,
                                    double* P_values);

/* Device inputs of n_inst instances of the socp's shape, each array the
 * concatenation over instances of the per-instance layout (the outputs of
 * ciscvx_discretize at X = Xp, ciscvx_node_linearize at (Xp, Xm, Phi, Gam)
 * and ciscvx_psi_linearize at (Xp, Xm), in FP64 except the Phi blocks). */
typedef struct {
  const double* Xp;     /* [N+1][n_x~] iterate: post-impact node states */
  const double* Xm;     /* [N+1][n_x~] pre-impact node states */
  const double* U;      /* [N+1][n_u] or [N][2][n_u] per the layout */
  const double* s;      /* [N] */
  const double* Phi;    /* [N+1][2 n_c] (NULL if n_c == 0) */
  const double* Gam;    /* [N+1][n_c]   (NULL if n_c == 0) */
  int phi_precision;    /* CISCVX_FP64 or CISCVX_FP32_PHI: type of A, Bm, Bp, S */
  const void* A; const void* Bm; const void* Bp;  /* per the socp's phi_format */
  const void* S;                                  /* [N][n_x~] */
  const double* defect; /* [N][n_x~] */
  const double* g;      /* [N+1][n_x~] and the Jacobian blocks of ciscvx_node_linearize */
  const double* Gvm; const double* Gth; const double* Gphi;
  const double* Gpx;    /* read only on a sinusoidal surface */
  const double* theta; const double* dtheta;  /* NULL if n_c == 0 */
  const double* psi; const double* dpsi;      /* NULL if n_c == 0 */
} ciscvx_socp_inputs;

/* Device outputs, [n_inst][...] each, all required: A_values [nnz_A],
 * b [n_eq], G_values [nnz_G], h [n_ineq], c [n_var], and the row scales
 * rho_A [n_eq], rho_G [n_ineq] (to map the solver's duals back). */
typedef struct {
  double* A_values; double* b; double* G_values; double* h; double* c;
  double* rho_A; double* rho_G;
} ciscvx_socp_outputs;

/* Numeric phase for n_inst instances (asynchronous on stream): a row pass
 * (row scales, b and h), a CSC pass (the values of A and G) and a column
 * pass (c).  The inputs may not alias the outputs.  Errors: EINVAL (nulls,
 * n_inst < 1, phi_precision), ECUDA. */
ciscvx_status ciscvx_socp_fill(const ciscvx_socp* socp, int n_inst, const ciscvx_socp_inputs* in,
                               const ciscvx_socp_outputs* out, void* stream);

/* ------------------------------------------------ allocation-free VJP --- */

/* Bytes of device scratch the library keeps for ciscvx_discretize_vjp_static. */
#define CISCVX_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* The same VJP as ciscvx_discretize_vjp, for callers that cannot allocate
 * device memory when they call it.  The paper has no counterpart; this is a
 * deployment convenience.  Typical callers: a model-predictive-control loop
 * that re-linearizes every few milliseconds (cudaMalloc there can synchronize
 * the device and has unbounded latency), or a solver embedded in a framework
 * that owns all device memory through its own pool.
 *   Arguments are those of ciscvx_discretize_vjp without the workspace: the
 *   caller still passes all inputs and outputs (device pointers).
 *   Scratch: a static array of CISCVX_STATIC_SCRATCH_BYTES inside the library,
 *   held on every GPU that loads the library until the process exits.  The
 *   first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   Calls share the one array: calls whose work overlaps on the GPU (other
 *   streams or host threads) race; serialize them.  Nothing in the array
 *   needs clearing (every scratch element is written before it is read).
 *   The cached address is valid for the life of the device's primary
 *   context; after cudaDeviceReset do not call this entry point on that
 *   device again in the same process.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.  One
 *   exception at set-up: for a model with coupled links, the first call for
 *   a model shape and precision in the process compiles and loads the
 *   run-time specialized kernels (the runtime takes device memory for the
 *   loaded code); make that call, or any ciscvx_discretize /
 *   ciscvx_discretize_vjp call of that model and precision, at set-up.
 *   Models: all of them.  Per-link models (either auxiliary model) run the
 *   adjoint kernel, whose scratch is ciscvx_workspace_size(CISCVX_OP_VJP)
 *   for N intervals.  Models with coupled links run their adjoint in chunks
 *   of the intervals whose stage data fit the array; their minimum is the
 *   min_bytes of ciscvx_discretize_workspace_size(CISCVX_OP_VJP).
 * Errors: as ciscvx_discretize_vjp, and CISCVX_EUNSUPPORTED when the minimum
 * scratch of this request (min_bytes of ciscvx_discretize_workspace_size with
 * CISCVX_OP_VJP) exceeds CISCVX_STATIC_SCRATCH_BYTES. */
ciscvx_status ciscvx_discretize_vjp_static(const ciscvx_model* model, int N, int n_sub,
                                           ciscvx_precision precision, ciscvx_u_layout layout,
                                           const double* X, const double* U, const double* s,
                                           const double* w, const double* rho, double* gX,
                                           double* gU, double* gs, double* L, void* stream);

/* Waits for `stream`, then reads and clears the model's device status word.
 * Returns CISCVX_OK, or CISCVX_ENONFINITE if any call since the last read
 * produced a non-finite state or block; ECUDA if the stream reports an error. */
ciscvx_status ciscvx_sync_status(const ciscvx_model* model, void* stream);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char* ciscvx_last_error(void);

/* Library version as MAJOR * 1000 + MINOR. */
int ciscvx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CISCVX_H_ */
