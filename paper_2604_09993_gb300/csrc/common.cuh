// common.cuh — device-side model tables and helpers shared by the CI-SCvx kernels.
//
// Structure the kernels exploit (all exact consequences of the model in
// include/ciscvx.h, Sec. II-A Eq. (1) with joint reaction forces as inputs):
//
//  * Links are decoupled: link b's accelerations depend only on its own angle
//    and on the inputs acting on it, so every link is an independent ODE and
//    the Jacobian blocks are block-sparse by link.
//  * Translation: v' = s a(tau), p' = s v with a(tau) affine in tau under the
//    first-order hold.  RK4 integrates this polynomial trajectory exactly, so
//    p(1), v(1) and their derivatives have closed forms.
//  * Rotation: with r = R(theta) rho, r x F = cos(theta) (rho x F) - sin(theta)
//    (rho . F), so omega' = cos(theta) P(tau) - sin(theta) Q(tau) + T(tau) with
//    P, Q, T linear in u and hence affine in tau.  The sensitivity of (theta,
//    omega) to input k is p_k Psi_c + q_k Psi_s + t_k Psi_1, where Psi_c,
//    Psi_s, Psi_1 are the tangents driven by cos(theta) w(tau), -sin(theta)
//    w(tau), w(tau) with w = 1 - tau (u_L) or tau (u_R): the RK4 tangent
//    recursion is linear in its forcing, so superposition is exact.  Nine
//    tangent columns (theta_0, omega_0, s and six basis forcings) cover every
//    input of a link.
//  * The contact penalty state of a foot link depends on the foot's p_y and
//    theta and on its three contact inputs; its row is a quadrature of the
//    stage sensitivities with the RK4 weights.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/ciscvx.h"
#include "dev_math.cuh"

namespace ciscvx {

constexpr int MAXB = CISCVX_MAX_BODIES;
constexpr int MAXIN = CISCVX_MAX_INPUTS_PER_BODY;
constexpr int MAXJ = 2 * MAXB;          // joints per model (<= 4 per link)
constexpr int MAXU = 3 * MAXJ + 3 * MAXB;
constexpr int MAXSUB_VJP = CISCVX_MAX_VJP_SUBSTEPS;
constexpr int NODE_MAXJ = CISCVX_NODE_MAX_JOINTS;             // joints the node kernel supports
constexpr int NODE_MAXADJ = CISCVX_NODE_MAX_JOINTS_PER_LINK;  // joints on one link it supports

// device status bits
constexpr unsigned ST_NONFINITE = 1u;

// Per-link program: the inputs acting on the link with their coefficients
// (already divided by m or I), and the link's contact if it has one.
struct DevBody {
  int nin;           // inputs acting on this link
  int contact;       // contact index, or -1
  int cin;           // input index of the contact's lambda_n (lambda_t+ = cin+1, lambda_t- = cin+2)
  int slot0;         // first VJP partial slot of this link within an interval
  int a_off;         // first entry of this link in the compact A values of an interval
  int b_off;         // first entry of this link in the compact B-/B+ values of an interval
  double crho[2];    // contact point (body frame)
  double mu;         // friction coefficient
  double pad_;
  int idx[MAXIN + 1];  // input index per slot
  double ax[MAXIN + 1];  // dv_x/du   (sigma/m for an x force, else 0)
  double ay[MAXIN + 1];  // dv_y/du   (sigma/m for a y force, else 0)
  double p[MAXIN + 1];   // d(omega')/du coefficient of cos(theta): sigma (rho x e)/I
  double q[MAXIN + 1];   // coefficient of -sin(theta): sigma (rho . e)/I
  double t[MAXIN + 1];   // torque coefficient: sigma/I
};

// Compact outputs keep only the structural nonzeros of A and B-/B+, per
// interval, link by link (rows px, py, th, vx, vy, om of link b, y of its
// contact's path-penalty state).  Link b's A entries, at a_off: (px,px)
// (px,vx) (py,py) (py,vy) (th,th) (th,om) (vx,vx) (vy,vy) (om,th) (om,om),
// then for a foot link (y,py) (y,th) (y,vy) (y,om) (y,y).  Link b's B
// entries, at b_off, for each of its inputs q in slot order: (px,q) if the
// input has an x force component, (py,q) if it has a y component, (th,q) if
// it exerts a torque, (vx,q) if x, (vy,q) if y, (om,q) if a torque, then
// (y,q) for a foot link.  B- and B+ share the pattern.
// Eq. (12) model (cross-complementarity rows c0..c3 = phi_n, lambda^c, gamma,
// rho^c of the foot's contact): after the foot's A entries (c0,c0) (c1,c1)
// (c2,c2) (c3,c3) (c1,vx) (c1,th) (c1,om); after the link's B groups one
// (c1,q) per input in slot order that pushes along x, exerts a torque, or is
// phi_t or gamma, then (c0,phi_n) (c2,gamma) (c3,phi_t) (c3,phi_n).
constexpr int A_PER_LINK = 10, A_PER_FOOT = 5, A_PER_CROSS = 7, B_CROSS_FIXED = 4;

// One instance of a batch: model, horizon, substeps and its element offsets
// into the packed arrays.
struct DevInst {
  int model, N, nsub;
  int contract;                   // 1: the VJP runs outside the per-link adjoint kernel (coupled links: the coupled adjoint)
  long long x, u, s, a, b, v, p;  // element offsets: X/gX, U/gU, s/gs, A, Bm/Bp, S/defect/w, penalty/rho
  long long part, pb;             // VJP workspace offsets: per-input partials, per-(interval, link) partials
};
// the run-time compiled kernels read the same table as InstRec (dev_math.cuh)
static_assert(sizeof(DevInst) == sizeof(InstRec), "instance table layouts differ");

struct DevModel {
  int nb, nj, nc, nxt, nu, nslot;   // nslot = sum of nin over links
  int nnzA, nnzB;                    // structural nonzeros of A and of B-/B+ (compact outputs)
  int tree;                          // every link is the child of at most one joint
  int aux;                           // 0: one path-penalty state per contact; 1: Eq. (12) (4 + 1)
  int ny;                            // auxiliary states: nc or 5 nc
  int jelim;                         // joint reaction forces eliminated (Eq. (3)); coupled path only
  int scheme;                        // 0: RK4; 1: Runge-Kutta-Fehlberg 4(5) (coupled path only)
  double ta, tk;                     // contact surface y = ta sin(tk x) (ta = 0: flat; coupled path if not)
  double g;
  // joints and link inertia (node constraints: impact map)
  int jpar[MAXJ], jchi[MAXJ];
  double jrp[MAXJ][2], jrc[MAXJ][2];  // anchors in the parent / child body frame
  double mass[MAXB], inertia[MAXB];
  double minv[MAXB], iinv[MAXB];      // 1 / mass, 1 / inertia
  int nadj[MAXB];                     // joints attached to each link (node kernel)
  int adj[MAXB][NODE_MAXADJ];         // (joint << 1) | (1 if the link is the joint's parent)
  // Node kernel: K = C' M^-1 C'^T in skyline form.  Joints are ordered
  // children first (post-order of the joint tree), so K's Cholesky factor has
  // no fill outside each row's envelope [nf[i], i] (a forest's joint graph is
  // chordal with that elimination order).  Row i = 2 * position + component.
  int npos[MAXJ];                     // position of joint j in the order
  int nord[MAXJ];                     // joint at each position
  int nf[2 * NODE_MAXJ];              // first stored column of each row of K
  int noff[2 * NODE_MAXJ + 1];        // offset of each row in the skyline storage
  int lmin[MAXB];                     // first row of K touched by a joint on link b
  int in_n[MAXU];        // per input: number of (link, slot) contributions (1 or 2)
  int in_slot[MAXU][2];  // per input: partial slots that contribute
  DevBody body[MAXB];
};

// Zero `count` elements starting at each active lane's own pointer `base`,
// with the lanes of `active` writing every chunk together (consecutive lanes
// write consecutive 16-byte vectors when the chunk is 16-byte aligned and a
// whole number of vectors long, else consecutive elements).  A __syncwarp
// after it orders these writes before the lanes' own writes to the same rows.
template <typename T>
__device__ __forceinline__ void warp_zero_chunks(T* base, int count, unsigned active) {
  const int lane = threadIdx.x & 31;
  const int rank = __popc(active & ((1u << lane) - 1u));  // position among active lanes
  const int nact = __popc(active);
  unsigned m = active;
  while (m) {
    const int t = __ffs(m) - 1;
    m &= m - 1;
    T* p = (T*)__shfl_sync(active, (unsigned long long)base, t);
    const size_t bytes = (size_t)count * sizeof(T);
    if ((((size_t)p) & 15) == 0 && (bytes & 15) == 0) {
      float4* v = (float4*)p;
      const int nv = (int)(bytes >> 4);
      for (int i = rank; i < nv; i += nact) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int i = rank; i < count; i += nact) p[i] = T(0);
    }
  }
}

// State at every substep start of one link of one interval (what the
// adjoint's backward sweep needs: the FP64 values for the FP64 adjoint, the
// FP32 anchors for the FP32 adjoint), plus the end state and the penalty
// integrand's quadrature.  Filled by the discretization when the two are fused.
struct Checkpoints {
  // FP64 adjoint: the FP64 state (and sin/cos of theta) at each substep start
  double th[MAXSUB_VJP], om[MAXSUB_VJP], s[MAXSUB_VJP], c[MAXSUB_VJP];
  double py[MAXSUB_VJP], vy[MAXSUB_VJP];
  // FP32 adjoint: the FP32 anchors of the stage recursion at each substep start
  float thf[MAXSUB_VJP], omf[MAXSUB_VJP], pyf[MAXSUB_VJP], vyf[MAXSUB_VJP];
  double th_end, om_end, Yom;
  double Il, Ir, Ig;  // Eq. (12) model: lambda^c's state and input parts, rho^c's integral
  // the link's FOH input sums (AxL, AxR, AyL, AyR, PL, PR, QL, QR, TL, TR) and h = 1/n_sub
  double ins[10], h;
  // When sm is set, the FP32 anchors live in shared memory instead of
  // thf..vyf: anchor f (0 theta, 1 omega, 2 p_y, 3 v_y) of substep i at
  // sm[(4 i + f) sst] (element-major over the block's threads, so a warp's
  // accesses are conflict-free).  The fused pass sets it when the block's
  // anchors fit; local memory otherwise.
  float* sm;
  int sst;
  __device__ __forceinline__ void put_f(int i, int f, float v) {
    if (sm) sm[(4 * i + f) * sst] = v;
    else (f == 0 ? thf : f == 1 ? omf : f == 2 ? pyf : vyf)[i] = v;
  }
  __device__ __forceinline__ float get_f(int i, int f) const {
    return sm ? sm[(4 * i + f) * sst] : (f == 0 ? thf : f == 1 ? omf : f == 2 ? pyf : vyf)[i];
  }
};

__device__ __forceinline__ double rk_c(int j) { return j == 0 ? 0.0 : (j == 3 ? 1.0 : 0.5); }
__device__ __forceinline__ double rk_w(int j) {
  return (j == 0 || j == 3) ? (1.0 / 6.0) : (2.0 / 6.0);
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// FP32 anchor of an FP64 state value (TP = float), or the value itself (TP = double).
template <typename TP>
__device__ __forceinline__ TP anchor(double x) {
  if constexpr (std::is_same<TP, float>::value) return to_f32_rz(x);
  else return x;
}

// Threads per CTA for the single-instance kernels: with few warps (small N)
// one warp per CTA spreads them over separate SMs, each with its own FP64
// units, which shortens the latency-bound critical path; otherwise 4 warps.
inline int single_cta_threads(long warps) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms = n > 0 ? n : 1;
  }
  return warps < 4L * sms ? 32 : 128;
}

}  // namespace ciscvx

namespace ciscvx {
struct CplTab;
}

// The opaque model handle of the C ABI.
struct ciscvx_model {
  ciscvx::DevModel host;  // host copy of the device tables
  ciscvx::DevModel* dev;  // device copy
  ciscvx::CplTab* cpl;    // coupled-path tables (host), or null for per-link models
  unsigned* status;       // device status word
  int device;             // CUDA device the tables live on
  // Eq. (12) model: the compact pattern by rows (device), for z with compact
  // outputs: A rows [nxt + 1] offsets, then (entry, column) pairs; the same for B
  int32_t* zpat;
};

// Launchers (defined in disc.cu / vjp.cu), called by the host API in api.cu.
namespace ciscvx {
cudaError_t launch_discretize(const DevModel* dM, int nb, int N, int nsub, int prec, int layout,
                              bool compact, bool aux, const double* X, const double* U, const double* s, void* A,
                              void* Bm, void* Bp, void* S, double* defect, double* penalty,
                              double* z, unsigned* status, cudaStream_t st);
cudaError_t launch_vjp(const DevModel* dM, int nb, int nxt, int nu, int nslot, int N, int nsub,
                       int prec, int layout, const double* X, const double* U, const double* s,
                       const double* w, const double* rho, double* gX, double* gU, double* gs,
                       double* L, void* ws, unsigned* status, bool aux, cudaStream_t st);
size_t vjp_workspace_bytes(int nb, int nu, int nslot, int N, int layout);
// Node constraints (node.cu).
struct NodeParams {
  double delta;     // Fischer-Burmeister relaxation
  double e[MAXB];   // restitution per contact
};
size_t node_smem_per_warp(const DevModel& M);
cudaError_t launch_node(const DevModel& Mh, const DevModel* dM, int n, const double* Xp,
                        const double* Xm, const double* Phi, const double* Gam,
                        const NodeParams& P, double* g, double* Gvm, double* Gth, double* Gphi,
                        double* Gpx, double* theta, double* dtheta, unsigned* status,
                        cudaStream_t st);
// Structural nonzeros of A and B-/B+ in compact order (api.cu); for models
// without coupled links and without the Eq. (12) state.
void model_pattern(const DevModel& M, int32_t* ar, int32_t* ac, int32_t* br, int32_t* bc);
// The affine term z_k = x~(1) - A x~_k - B- u_L - B+ u_R - S s_k from the
// dense outputs (affine_z.cu), for the models whose kernels do not form it.
cudaError_t launch_affine_z(const DevModel& M, int N, int prec, int layout, const double* X, const double* U,
                            const double* s, const void* A, const void* Bm, const void* Bp, const void* S,
                            const double* defect, double* z, cudaStream_t st);
// The same from compact outputs, with the pattern by rows (ciscvx_model::zpat).
cudaError_t launch_affine_z_compact(const DevModel& M, int N, int prec, int layout, const double* X,
                                    const double* U, const double* s, const void* A, const void* Bm,
                                    const void* Bp, const void* S, const double* defect, const int32_t* zpat,
                                    double* z, cudaStream_t st);
// Psi^{delta,eps} rows per interval, and its launcher (psi.cu).
int psi_rows(const DevModel& M);
cudaError_t launch_psi(const DevModel& M, int N, const double* Xp, const double* Xm, double delta,
                       double eps, double* psi, double* dpsi, unsigned* status, cudaStream_t st);
// Records a formatted last-error message (thread-local) and returns st.
ciscvx_status set_error(ciscvx_status st, const char* fmt, ...);
}  // namespace ciscvx
