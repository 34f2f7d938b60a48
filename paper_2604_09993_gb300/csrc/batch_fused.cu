// batch_fused.cu — linearized discretization and its adjoint VJP of every
// work item in one pass.  The two share the FP64 state trajectory of the
// interval: the discretization's forward sweep records the state at every
// substep start (disc_link with CK), and the adjoint's backward sweep starts
// from those checkpoints (vjp_link with FUSED), so the trajectory is
// integrated once instead of twice.  Outputs are those of
// ciscvx_batch_discretize and ciscvx_batch_discretize_vjp.
#include "batch_common.cuh"

namespace ciscvx {

namespace {

// AUX: the batch holds an Eq. (12) model (its foot links take the CROSS
// forms; a separate instantiation, no register cap).
template <typename TP, int OCC, bool CMP, bool AUX = false>
__global__ void __launch_bounds__(Occ<OCC>::T, Occ<OCC>::B)
    k_batch_disc_vjp(BatchCommon c, const double* __restrict__ X, const double* __restrict__ U,
                     const double* __restrict__ s, TP* A, TP* Bm, TP* Bp, TP* S, double* defect,
                     double* penalty, const double* __restrict__ w,
                     const double* __restrict__ rho, double* gX, double* part, double* ps,
                     double* pL) {
  extern __shared__ float ck_smem[];
  const int lane = threadIdx.x & 31;
  int iter = 0;
  for (;;) {
    const int item = next_item(c, iter);
    if (item >= c.n_items) break;
    const int2 it = c.items[item];
    const int4 g = c.groups[it.x];
    if (lane < g.w) {
      const DevModel& M = *c.models[g.x];
      const int b = it.y;
      const int2 e = c.entries[g.z + lane];
      const DevInst& I = c.inst[e.x];
      const long k = e.y;
      const int N = I.N, nxt = M.nxt, nu = M.nu, nc = M.nc, nb = M.nb;
      const double* Xi = X + I.x;
      const double* uL = (c.layout == CISCVX_FOH_NODE) ? U + I.u + k * nu : U + I.u + 2 * k * nu;
      const double* uR = uL + nu;
      // compact values staged in dense blocks (c.stage_dense) take the dense strides
      const size_t sa = (CMP && !c.stage_dense) ? (size_t)M.nnzA : (size_t)nxt * nxt;
      const size_t sb = (CMP && !c.stage_dense) ? (size_t)M.nnzB : (size_t)nxt * nu;
      TP* Ak = A + I.a + k * sa;
      TP* Bmk = Bm ? Bm + I.b + k * sb : nullptr;
      TP* Bpk = Bp ? Bp + I.b + k * sb : nullptr;
      TP* Sk = S + I.v + (size_t)k * nxt;
      double* dk = defect + I.v + (size_t)k * nxt;
      double* pk = penalty ? penalty + I.p + (size_t)k * nc : nullptr;
      const double* wi = w + I.v;
      const DevBody& B = M.body[b];
      const double rc = (B.contact >= 0) ? rho[I.p + k * nc + B.contact] : 0.0;
      const double* wkm1 = (k > 0) ? wi + (k - 1) * nxt : nullptr;
      double* gXi = gX + I.x;
      double* gXN = (k == N - 1) ? gXi + (size_t)N * nxt : nullptr;
      double* pp = part + I.part + (size_t)k * M.nslot * 2;
      double* psk = ps + I.pb + k * nb;
      double* pLk = pL + I.pb + k * nb;
      const double sk = s[I.s + k];
      const double* xk = Xi + k * nxt;
      const double* xk1 = Xi + (k + 1) * nxt;
      Checkpoints ck;
      ck.sm = c.ck_smem ? ck_smem + threadIdx.x : nullptr;
      ck.sst = blockDim.x;
      if (AUX && M.aux && B.contact >= 0) {  // Eq. (12) model
        disc_link<TP, true, CMP, true, true>(M, b, g.y, sk, xk, xk1, uL, uR, Ak, Bmk, Bpk, Sk, dk, pk,
                                             nullptr, c.status, &ck);
        vjp_link<TP, true, true, true>(M, b, g.y, sk, xk, xk1, uL, uR, wi + k * nxt, wkm1, rc,
                                       gXi + (size_t)k * nxt, gXN, pp, psk, pLk, c.status, &ck);
      } else if (B.contact >= 0) {
        disc_link<TP, true, CMP, true>(M, b, g.y, sk, xk, xk1, uL, uR, Ak, Bmk, Bpk, Sk, dk, pk,
                                       nullptr, c.status, &ck);
        vjp_link<TP, true, true>(M, b, g.y, sk, xk, xk1, uL, uR, wi + k * nxt, wkm1, rc,
                                 gXi + (size_t)k * nxt, gXN, pp, psk, pLk, c.status, &ck);
      } else {
        disc_link<TP, false, CMP, true>(M, b, g.y, sk, xk, xk1, uL, uR, Ak, Bmk, Bpk, Sk, dk, pk,
                                        nullptr, c.status, &ck);
        vjp_link<TP, false, true>(M, b, g.y, sk, xk, xk1, uL, uR, wi + k * nxt, wkm1, rc,
                                  gXi + (size_t)k * nxt, gXN, pp, psk, pLk, c.status, &ck);
      }
    }
  }
}

}  // namespace

cudaError_t launch_disc_vjp_fused(const BatchCommon& c, int prec, int occ, bool compact, bool aux,
                                  unsigned blocks, unsigned threads, const double* X,
                                  const double* U, const double* s, void* A, void* Bm, void* Bp,
                                  void* S, double* defect, double* penalty, const double* w,
                                  const double* rho, double* gX, double* part, double* ps,
                                  double* pL, size_t smem, cudaStream_t st) {
#define CISCVX_FUSED1(TP, OCC, CMP)                                                            \
  k_batch_disc_vjp<TP, OCC, CMP><<<blocks, threads, smem, st>>>(c, X, U, s, (TP*)A, (TP*)Bm,     \
                                                             (TP*)Bp, (TP*)S, defect, penalty, w, \
                                                             rho, gX, part, ps, pL)
#define CISCVX_FUSED(TP, OCC)                   \
  do {                                          \
    if (compact) CISCVX_FUSED1(TP, OCC, true);  \
    else CISCVX_FUSED1(TP, OCC, false);         \
  } while (0)
  if (aux) {  // no register cap
#define CISCVX_FUSED_AUX(TP, CMP)                                                                    \
  k_batch_disc_vjp<TP, 0, CMP, true><<<blocks, threads, smem, st>>>(c, X, U, s, (TP*)A, (TP*)Bm, (TP*)Bp, \
                                                                    (TP*)S, defect, penalty, w, rho, gX,  \
                                                                    part, ps, pL)
    if (prec == CISCVX_FP64) {
      if (compact) CISCVX_FUSED_AUX(double, true); else CISCVX_FUSED_AUX(double, false);
    } else {
      if (compact) CISCVX_FUSED_AUX(float, true); else CISCVX_FUSED_AUX(float, false);
    }
#undef CISCVX_FUSED_AUX
  } else if (prec == CISCVX_FP64) {
    if (occ == 1) CISCVX_FUSED(double, 1);
    else if (occ == 2) CISCVX_FUSED(double, 2);
    else CISCVX_FUSED(double, 0);
  } else {
    if (occ == 1) CISCVX_FUSED(float, 1);
    else if (occ == 2) CISCVX_FUSED(float, 2);
    else CISCVX_FUSED(float, 0);
  }
#undef CISCVX_FUSED
#undef CISCVX_FUSED1
  return cudaGetLastError();
}

}  // namespace ciscvx
