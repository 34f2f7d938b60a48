// socp.cu — the convex subproblem of one prox-linear SCP iteration (Sec. V)
// in the canonical SOCP form of a conic solver, assembled on the GPU from the
// linearization outputs (Sec. VI: CSC matrices, row normalization, affine
// variable scaling).  The variables, rows, convex set, objective and scaling
// are the ones include/ciscvx.h states for ciscvx_socp_*.
//
// Two phases.  The symbolic phase (host, once per (model, N, layout)) lays out
// the columns and rows and lists every structural entry with a 64-bit source
// descriptor: which output block of which interval or node holds its value,
// or a constant.  It keeps the entries both row by row (for the row pass) and
// sorted into CSC order (for the value pass), and precomputes everything that
// does not depend on the iterate: the column scales and offsets, P and P o.
// The numeric phase (device, per call, any number of instances of that shape):
//   rows:   thread per (instance, row): the row's scaled max-norm over the
//           problem columns -> rho, and b (or h) = rho (J zbar - residual - J o)
//   values: thread per (instance, CSC entry): source * D[col] * rho[row]
//   c:      thread per (instance, column): D (P o - w_px zbar), or w_ep
// The descriptors are shared by all instances and stay in L2; every output is
// written once, coalesced.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"

using namespace ciscvx;

namespace {

// ---------------------------------------------------------------- sources ---
// bits 58..63 kind, bit 57 negate, bits 32..56 interval/node index, 0..31 offset
enum : unsigned {
  SRC_CONST = 1, SRC_A, SRC_BM, SRC_BP, SRC_S, SRC_GVM, SRC_GTH, SRC_GPHI, SRC_GPX, SRC_DTH, SRC_DPSI
};
// column iterate sources (kind bits as above, offset = component)
enum : unsigned { Z_SLACK = 0, Z_XP, Z_XM, Z_PHI, Z_GAM, Z_U, Z_UL, Z_UR, Z_S };
// row residual sources
enum : unsigned { R_CONST = 1, R_G, R_DYN, R_TH, R_PSI };

constexpr int SOCP_MAXK = (1 << 25) - 1;

inline uint64_t desc(unsigned kind, long k, unsigned off, bool neg = false) {
  return ((uint64_t)kind << 58) | ((uint64_t)(neg ? 1 : 0) << 57) | ((uint64_t)k << 32) | off;
}
__host__ __device__ inline unsigned d_kind(uint64_t d) { return (unsigned)(d >> 58); }
__host__ __device__ inline bool d_neg(uint64_t d) { return (d >> 57) & 1u; }
__host__ __device__ inline long d_k(uint64_t d) { return (long)((d >> 32) & 0x1FFFFFFull); }
__host__ __device__ inline unsigned d_off(uint64_t d) { return (unsigned)(d & 0xFFFFFFFFull); }

// Device copy of one matrix's tables.
struct MatDev {
  int nrow;
  long long nnz;
  const int* rowptr;         // [nrow + 1] row view
  const int* rcol;           // [nnz] column of each row-view entry
  const uint64_t* rsrc;      // [nnz] source of each row-view entry
  const uint64_t* res;       // [nrow] residual source (R_*)
  const int* crow;           // [nnz] row of each CSC entry
  const int* ccol;           // [nnz] column of each CSC entry
  const uint64_t* csrc;      // [nnz] source of each CSC entry
  int soc0;                  // first row of the Q^2 blocks (rows pair up from here), or nrow
};

// Per-call pointers and per-instance strides (elements).
struct SocpIO {
  int N, nxt, nu, nb, nc, npsi, ny, nq, n_var, node_layout, phi64;
  long long sX, sU, sS, sPhi, sGam, sA, sB, sSv, sDef, sG, sGvm, sGth, sGphi, sGpx, sTh, sDth, sPsi, sDpsi;
  const double *Xp, *Xm, *U, *s, *Phi, *Gam, *defect, *g, *Gvm, *Gth, *Gphi, *Gpx, *theta, *dtheta,
      *psi, *dpsi;
  const void *A, *Bm, *Bp, *S;
  const double* consts;
  const uint64_t* colz;  // [n_var] iterate source of each column
  const double* D;       // [n_var]
  const double* o;       // [n_var]
  const double* Po;      // [n_var] P o
  double w_px, w_ep;
};

__device__ __forceinline__ double phi_at(const SocpIO& I, const void* p, long long idx) {
  return I.phi64 ? ((const double*)p)[idx] : (double)((const float*)p)[idx];
}

__device__ double fetch(const SocpIO& I, long inst, uint64_t d) {
  const unsigned kind = d_kind(d), off = d_off(d);
  const long k = d_k(d);
  double v;
  switch (kind) {
    case SRC_CONST: v = I.consts[off]; break;
    case SRC_A: v = phi_at(I, I.A, inst * I.sA + k * (long long)I.nxt * I.nxt + off); break;
    case SRC_BM: v = phi_at(I, I.Bm, inst * I.sB + k * (long long)I.nxt * I.nu + off); break;
    case SRC_BP: v = phi_at(I, I.Bp, inst * I.sB + k * (long long)I.nxt * I.nu + off); break;
    case SRC_S: v = phi_at(I, I.S, inst * I.sSv + k * (long long)I.nxt + off); break;
    case SRC_GVM: v = I.Gvm[inst * I.sGvm + k * (long long)I.nq * I.nq + off]; break;
    case SRC_GTH: v = I.Gth[inst * I.sGth + k * (long long)I.nq * I.nb + off]; break;
    case SRC_GPHI: v = I.Gphi[inst * I.sGphi + k * (long long)I.nq * 2 * I.nc + off]; break;
    case SRC_GPX: v = I.Gpx[inst * I.sGpx + k * (long long)I.nq * I.nc + off]; break;
    case SRC_DTH: v = I.dtheta[inst * I.sDth + k * (long long)I.nc * 8 * CISCVX_NODE_THETA_COLS + off]; break;
    case SRC_DPSI: v = I.dpsi[inst * I.sDpsi + k * (long long)I.npsi * I.ny + off]; break;
    default: v = 0.0;
  }
  return d_neg(d) ? -v : v;
}

__device__ double zbar_at(const SocpIO& I, long inst, uint64_t d) {
  const unsigned off = d_off(d);
  const long k = d_k(d);
  switch (d_kind(d)) {
    case Z_XP: return I.Xp[inst * I.sX + k * I.nxt + off];
    case Z_XM: return I.Xm[inst * I.sX + k * I.nxt + off];
    case Z_PHI: return I.Phi[inst * I.sPhi + k * 2 * I.nc + off];
    case Z_GAM: return I.Gam[inst * I.sGam + k * I.nc + off];
    case Z_U: return I.U[inst * I.sU + k * I.nu + off];
    case Z_UL: return I.U[inst * I.sU + (2 * k) * I.nu + off];
    case Z_UR: return I.U[inst * I.sU + (2 * k + 1) * I.nu + off];
    case Z_S: return I.s[inst * I.sS + k];
    default: return 0.0;
  }
}

__device__ double residual_at(const SocpIO& I, long inst, uint64_t d) {
  const unsigned off = d_off(d);
  const long k = d_k(d);
  switch (d_kind(d)) {
    case R_G: return I.g[inst * I.sG + k * I.nxt + off];
    case R_DYN:  // F~(x~+_k, U_k, s_k) - x~-_{k+1}, with F~ = defect + x~+_{k+1}
      return I.defect[inst * I.sDef + k * I.nxt + off] + I.Xp[inst * I.sX + (k + 1) * I.nxt + off] -
             I.Xm[inst * I.sX + (k + 1) * I.nxt + off];
    case R_TH: return I.theta[inst * I.sTh + k * 8 * I.nc + off];
    case R_PSI: return I.psi[inst * I.sPsi + k * I.npsi + off];
    default: return 0.0;
  }
}

// Scaled max-norm of row r over the problem columns.
__device__ double row_norm(const SocpIO& I, const MatDev& T, long inst, int r) {
  double nrm = 0.0;
  for (int e = T.rowptr[r]; e < T.rowptr[r + 1]; ++e) {
    const int c = T.rcol[e];
    if (d_kind(I.colz[c]) == Z_SLACK) continue;
    nrm = fmax(nrm, fabs(fetch(I, inst, T.rsrc[e]) * I.D[c]));
  }
  return nrm;
}

__global__ void __launch_bounds__(256) k_socp_rows(SocpIO I, MatDev T, int n_inst, double* rho_out,
                                                    double* rhs_out) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long)n_inst * T.nrow) return;
  const long inst = g / T.nrow;
  const int r = (int)(g - inst * T.nrow);
  double nrm = 0.0, jz = 0.0, jo = 0.0;
  for (int e = T.rowptr[r]; e < T.rowptr[r + 1]; ++e) {
    const int c = T.rcol[e];
    const uint64_t zc = I.colz[c];
    const double v = fetch(I, inst, T.rsrc[e]);
    if (d_kind(zc) != Z_SLACK) {
      nrm = fmax(nrm, fabs(v * I.D[c]));
      jz = fma(v, zbar_at(I, inst, zc), jz);
      jo = fma(v, I.o[c], jo);
    }
  }
  if (r >= T.soc0) {  // a Q^2 block takes the larger norm of its two rows
    const int partner = T.soc0 + ((r - T.soc0) ^ 1);
    nrm = fmax(nrm, row_norm(I, T, inst, partner));
  }
  const uint64_t rd = T.res[r];
  const double rhs = (d_kind(rd) == R_CONST ? I.consts[d_off(rd)] : jz - residual_at(I, inst, rd)) - jo;
  const double rho = nrm > 0.0 ? 1.0 / nrm : 1.0;
  rho_out[inst * T.nrow + r] = rho;
  rhs_out[inst * T.nrow + r] = rho * rhs;
}

__global__ void __launch_bounds__(256) k_socp_values(SocpIO I, MatDev T, int n_inst, const double* rho,
                                                      double* val) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)n_inst * T.nnz) return;
  const long inst = (long)(g / T.nnz);
  const long long e = g - (long long)inst * T.nnz;
  val[g] = fetch(I, inst, T.csrc[e]) * I.D[T.ccol[e]] * rho[inst * T.nrow + T.crow[e]];
}

__global__ void __launch_bounds__(256) k_socp_c(SocpIO I, int n_inst, double* c) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long)n_inst * I.n_var) return;
  const long inst = g / I.n_var;
  const int j = (int)(g - inst * I.n_var);
  const uint64_t zc = I.colz[j];
  c[g] = d_kind(zc) == Z_SLACK ? I.w_ep : I.D[j] * (I.Po[j] - I.w_px * zbar_at(I, inst, zc));
}

// ---------------------------------------------------------- host builder ---
struct Entry {
  int row, col;
  uint64_t src;
};

struct HostMat {
  std::vector<Entry> e;       // row by row, in the order rows are made
  std::vector<uint64_t> res;  // per row
  int nrow = 0;
  int begin_row(uint64_t residual) {
    res.push_back(residual);
    return nrow++;
  }
  void add(int row, int col, uint64_t src) { e.push_back({row, col, src}); }
};

struct Builder {
  const DevModel& M;
  int N, nxt, nu, nb, nj, nc, nq, nx, ny, npsi;
  bool node, aux, terrain, jelim, has_pattern;
  std::vector<int> c_xm, c_xp, c_phi, c_gam, c_u, c_nuGp, c_nuGm, c_tth, c_uL, c_uR, c_s, c_nuFp, c_nuFm,
      c_tpsi;
  std::vector<uint64_t> colz;
  std::vector<double> D, o, consts;
  std::map<double, unsigned> const_idx;
  HostMat A, G;
  int n_nonneg = 0, n_soc = 0;
  std::vector<int32_t> par, pac, pbr, pbc;
  std::vector<int> contact_body;

  Builder(const DevModel& m, int N_, int layout) : M(m), N(N_) {
    nxt = M.nxt; nu = M.nu; nb = M.nb; nj = M.nj; nc = M.nc;
    nq = 3 * nb; nx = 6 * nb; ny = nxt - nx;
    aux = M.aux != 0; jelim = M.jelim != 0; terrain = M.ta != 0.0;
    npsi = aux ? 3 * nc : nc;
    node = layout == CISCVX_FOH_NODE;
    has_pattern = !aux && !jelim && M.scheme == 0 && !terrain;
    if (has_pattern) {
      par.resize(M.nnzA); pac.resize(M.nnzA); pbr.resize(M.nnzB); pbc.resize(M.nnzB);
      model_pattern(M, par.data(), pac.data(), pbr.data(), pbc.data());
    }
    contact_body.assign(nc, -1);
    for (int b = 0; b < nb; ++b)
      if (M.body[b].contact >= 0) contact_body[M.body[b].contact] = b;
  }

  unsigned cst(double v) {
    auto it = const_idx.find(v);
    if (it != const_idx.end()) return it->second;
    const unsigned i = (unsigned)consts.size();
    consts.push_back(v);
    const_idx[v] = i;
    return i;
  }
  uint64_t one(bool neg = false) { return desc(SRC_CONST, 0, cst(1.0), neg); }
  uint64_t value(double v) { return desc(SRC_CONST, 0, cst(v)); }
  uint64_t rconst(double v) { return desc(R_CONST, 0, cst(v)); }

  // columns: n of them, iterate source kind zk at index k (components 0..n-1),
  // scale/offset vectors sc/of of length n (null = identity) or slack
  int take(std::vector<int>& v, int n, unsigned zk, long k, const double* sc, const double* of) {
    const int c0 = (int)colz.size();
    v.push_back(c0);
    for (int i = 0; i < n; ++i) {
      colz.push_back(zk == Z_SLACK ? 0 : desc(zk, k, (unsigned)i));
      D.push_back(zk != Z_SLACK && sc ? sc[i] : 1.0);
      o.push_back(zk != Z_SLACK && of ? of[i] : 0.0);
    }
    return c0;
  }

  void columns(const ciscvx_socp_params& P) {
    const double ss[1] = {P.scale_s != 0.0 ? P.scale_s : 1.0}, os[1] = {P.offset_s};
    for (int k = 0; k <= N; ++k) {
      take(c_xm, nxt, Z_XM, k, P.scale_x, P.offset_x);
      take(c_xp, nxt, Z_XP, k, P.scale_x, P.offset_x);
      take(c_phi, 2 * nc, Z_PHI, k, P.scale_phi, P.offset_phi);
      take(c_gam, nc, Z_GAM, k, P.scale_gam, P.offset_gam);
      if (node) take(c_u, nu, Z_U, k, P.scale_u, P.offset_u);
      take(c_nuGp, nxt, Z_SLACK, 0, nullptr, nullptr);
      take(c_nuGm, nxt, Z_SLACK, 0, nullptr, nullptr);
      take(c_tth, 8 * nc, Z_SLACK, 0, nullptr, nullptr);
      if (k < N) {
        if (!node) {
          take(c_uL, nu, Z_UL, k, P.scale_u, P.offset_u);
          take(c_uR, nu, Z_UR, k, P.scale_u, P.offset_u);
        }
        take(c_s, 1, Z_S, k, ss, os);
        take(c_nuFp, nxt, Z_SLACK, 0, nullptr, nullptr);
        take(c_nuFm, nxt, Z_SLACK, 0, nullptr, nullptr);
        take(c_tpsi, npsi, Z_SLACK, 0, nullptr, nullptr);
      }
    }
  }
  int uL(int k) const { return node ? c_u[k] : c_uL[k]; }
  int uR(int k) const { return node ? c_u[k + 1] : c_uR[k]; }
  int contact_in(int ub, int i) const { return ub + (jelim ? 1 : 3) * nj + 3 * i; }

  void input_rows(int ub, const ciscvx_socp_params& P) {
    for (int j = 0; j < nj; ++j) {
      G.add(G.begin_row(rconst(P.torque_max[j])), ub + j, one());
      G.add(G.begin_row(rconst(P.torque_max[j])), ub + j, one(true));
    }
    for (int i = 0; i < nc; ++i) {
      const int c0 = contact_in(ub, i);
      if (aux) {
        G.add(G.begin_row(rconst(0.0)), c0 + 2, one(true));  // -gamma <= 0
      } else {
        for (int t = 0; t < 3; ++t) G.add(G.begin_row(rconst(0.0)), c0 + t, one(true));
        const int r = G.begin_row(rconst(0.0));  // lambda_t+ + lambda_t- - mu lambda_n <= 0
        G.add(r, c0, value(-M.body[contact_body[i]].mu));
        G.add(r, c0 + 1, one());
        G.add(r, c0 + 2, one());
      }
    }
  }

  void rows(const ciscvx_socp_params& P) {
    for (int k = 0; k <= N; ++k) {
      // G~ rows of node k
      for (int r = 0; r < nxt; ++r) {
        const int row = A.begin_row(desc(R_G, k, (unsigned)r));
        if (r < nq) {
          A.add(row, c_xm[k] + r, one(true));
          A.add(row, c_xp[k] + r, one());
        } else if (r < 2 * nq) {
          const int a = r - nq, b = a / 3;
          for (int c = 0; c < nq; ++c) {
            if (c % 3 == 2) A.add(row, c_xm[k] + c, desc(SRC_GTH, k, (unsigned)(a * nb + c / 3)));
            else if (terrain && c % 3 == 0 && M.body[c / 3].contact >= 0)
              A.add(row, c_xm[k] + c, desc(SRC_GPX, k, (unsigned)(a * nc + M.body[c / 3].contact)));
          }
          for (int c = 0; c < nq; ++c) A.add(row, c_xm[k] + nq + c, desc(SRC_GVM, k, (unsigned)(a * nq + c)));
          A.add(row, c_xp[k] + r, value(a % 3 == 2 ? M.inertia[b] : M.mass[b]));
          for (int j = 0; j < 2 * nc; ++j) A.add(row, c_phi[k] + j, desc(SRC_GPHI, k, (unsigned)(a * 2 * nc + j)));
        } else {
          A.add(row, c_xm[k] + r, one(true));
          A.add(row, c_xp[k] + r, one());
        }
        A.add(row, c_nuGp[k] + r, one(true));
        A.add(row, c_nuGm[k] + r, one());
      }
      // dynamics rows of interval k
      if (k < N) {
        for (int r = 0; r < nxt; ++r) {
          const int row = A.begin_row(desc(R_DYN, k, (unsigned)r));
          if (has_pattern) {
            for (size_t e = 0; e < par.size(); ++e)
              if (par[e] == r) A.add(row, c_xp[k] + pac[e], desc(SRC_A, k, (unsigned)(r * nxt + pac[e])));
          } else {
            for (int c = 0; c < nxt; ++c) A.add(row, c_xp[k] + c, desc(SRC_A, k, (unsigned)(r * nxt + c)));
          }
          A.add(row, c_xm[k + 1] + r, one(true));
          auto badd = [&](int q) {
            A.add(row, uL(k) + q, desc(SRC_BM, k, (unsigned)(r * nu + q)));
            A.add(row, uR(k) + q, desc(SRC_BP, k, (unsigned)(r * nu + q)));
          };
          if (has_pattern) {
            for (size_t e = 0; e < pbr.size(); ++e)
              if (pbr[e] == r) badd(pbc[e]);
          } else {
            for (int q = 0; q < nu; ++q) badd(q);
          }
          A.add(row, c_s[k], desc(SRC_S, k, (unsigned)r));
          A.add(row, c_nuFp[k] + r, one(true));
          A.add(row, c_nuFm[k] + r, one());
        }
      }
      // nonnegative rows of node k
      for (int i = 0; i < nc; ++i) {
        const int b = contact_body[i];
        // local variables (p_x-, p_y-, theta-, v+ (3), v- (3), Phi_t, Phi_n, Gamma)
        const int cols[CISCVX_NODE_THETA_COLS] = {
            c_xm[k] + 3 * b, c_xm[k] + 3 * b + 1, c_xm[k] + 3 * b + 2,
            c_xp[k] + nq + 3 * b, c_xp[k] + nq + 3 * b + 1, c_xp[k] + nq + 3 * b + 2,
            c_xm[k] + nq + 3 * b, c_xm[k] + nq + 3 * b + 1, c_xm[k] + nq + 3 * b + 2,
            c_phi[k] + 2 * i, c_phi[k] + 2 * i + 1, c_gam[k] + i};
        for (int j = 0; j < 8; ++j) {
          const int row = G.begin_row(desc(R_TH, k, (unsigned)(8 * i + j)));
          for (int v = 0; v < CISCVX_NODE_THETA_COLS; ++v) {
            if (!terrain && (v == 0 || v == 6)) continue;  // zero on flat ground
            G.add(row, cols[v], desc(SRC_DTH, k, (unsigned)((8 * i + j) * CISCVX_NODE_THETA_COLS + v)));
          }
          G.add(row, c_tth[k] + 8 * i + j, one(true));
        }
      }
      for (int r = 0; r < 8 * nc; ++r) G.add(G.begin_row(rconst(0.0)), c_tth[k] + r, one(true));
      for (int r = 0; r < nxt; ++r) G.add(G.begin_row(rconst(0.0)), c_nuGp[k] + r, one(true));
      for (int r = 0; r < nxt; ++r) G.add(G.begin_row(rconst(0.0)), c_nuGm[k] + r, one(true));
      if (node) input_rows(c_u[k], P);
      if (k < N) {
        for (int r = 0; r < npsi; ++r) {
          const int row = G.begin_row(desc(R_PSI, k, (unsigned)r));
          int ja, jb = -1;
          if (aux && r < 2 * nc) {
            ja = 4 * (r >> 1) + 2 * (r & 1);
            jb = ja + 1;
          } else {
            ja = aux ? 4 * nc + (r - 2 * nc) : r;
          }
          for (int j : {ja, jb}) {
            if (j < 0) continue;
            G.add(row, c_xp[k] + nx + j, desc(SRC_DPSI, k, (unsigned)(r * ny + j), true));
            G.add(row, c_xm[k + 1] + nx + j, desc(SRC_DPSI, k, (unsigned)(r * ny + j)));
          }
          G.add(row, c_tpsi[k] + r, one(true));
        }
        for (int r = 0; r < npsi; ++r) G.add(G.begin_row(rconst(0.0)), c_tpsi[k] + r, one(true));
        for (int r = 0; r < nxt; ++r) G.add(G.begin_row(rconst(0.0)), c_nuFp[k] + r, one(true));
        for (int r = 0; r < nxt; ++r) G.add(G.begin_row(rconst(0.0)), c_nuFm[k] + r, one(true));
        G.add(G.begin_row(rconst(P.s_max)), c_s[k], one());
        G.add(G.begin_row(rconst(-P.s_min)), c_s[k], one(true));
        if (!node) {
          input_rows(c_uL[k], P);
          input_rows(c_uR[k], P);
        }
      }
    }
    // boundary conditions (Eq. (17g))
    for (int r = 0; r < nx; ++r) A.add(A.begin_row(rconst(P.x_init[r])), c_xm[0] + r, one());
    for (int r = 0; r < nx; ++r) A.add(A.begin_row(rconst(P.x_final[r])), c_xp[N] + r, one());
    n_nonneg = G.nrow;
    if (aux) {  // friction cones (mu phi_n, phi_t) in Q^2, per control vector and contact
      auto cones = [&](int ub) {
        for (int i = 0; i < nc; ++i) {
          const int c0 = contact_in(ub, i);
          G.add(G.begin_row(rconst(0.0)), c0 + 1, value(-M.body[contact_body[i]].mu));
          G.add(G.begin_row(rconst(0.0)), c0, one(true));
          ++n_soc;
        }
      };
      for (int k = 0; k <= N; ++k) {
        if (node) cones(c_u[k]);
        else if (k < N) {
          cones(c_uL[k]);
          cones(c_uR[k]);
        }
      }
    }
  }
};

template <typename T>
T* upload(const std::vector<T>& v, cudaError_t& e) {
  T* d = nullptr;
  if (e != cudaSuccess || v.empty()) return nullptr;
  e = cudaMalloc(&d, v.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return d;
}

}  // namespace

struct ciscvx_socp {
  int N, layout, device;
  ciscvx_socp_dims dims;
  int nxt, nu, nb, nc, npsi, ny, nq;
  double w_px, w_ep;
  std::vector<int> A_colptr, A_rowind, G_colptr, G_rowind, P_colptr, P_rowind;
  std::vector<double> P_val;
  MatDev dA, dG;
  std::vector<void*> allocs;
  const double *consts, *D, *o, *Po;
  const uint64_t* colz;
};

namespace {

// Sorts a matrix's entries into CSC order and fills its host index arrays and
// device tables.
bool finish(const HostMat& H, int n_var, std::vector<int>& colptr, std::vector<int>& rowind,
            MatDev& T, ciscvx_socp* so, int soc0, cudaError_t& e) {
  const long long nnz = (long long)H.e.size();
  std::vector<int> rowptr(H.nrow + 1, 0), rcol(nnz), crow(nnz), ccol(nnz);
  std::vector<uint64_t> rsrc(nnz), csrc(nnz);
  for (long long i = 0; i < nnz; ++i) {
    ++rowptr[H.e[i].row + 1];
    rcol[i] = H.e[i].col;
    rsrc[i] = H.e[i].src;
  }
  for (int r = 0; r < H.nrow; ++r) rowptr[r + 1] += rowptr[r];
  std::vector<long long> perm(nnz);
  for (long long i = 0; i < nnz; ++i) perm[i] = i;
  std::sort(perm.begin(), perm.end(), [&](long long a, long long b) {
    return H.e[a].col != H.e[b].col ? H.e[a].col < H.e[b].col : H.e[a].row < H.e[b].row;
  });
  colptr.assign(n_var + 1, 0);
  rowind.resize(nnz);
  for (long long i = 0; i < nnz; ++i) {
    const Entry& x = H.e[perm[i]];
    if (i > 0 && x.col == H.e[perm[i - 1]].col && x.row == H.e[perm[i - 1]].row) return false;
    crow[i] = x.row;
    ccol[i] = x.col;
    csrc[i] = x.src;
    rowind[i] = x.row;
    ++colptr[x.col + 1];
  }
  for (int c = 0; c < n_var; ++c) colptr[c + 1] += colptr[c];
  T.nrow = H.nrow;
  T.nnz = nnz;
  T.soc0 = soc0;
  auto up = [&](auto& v) {
    auto* p = upload(v, e);
    if (p) so->allocs.push_back((void*)p);
    return p;
  };
  T.rowptr = up(rowptr);
  T.rcol = up(rcol);
  T.rsrc = up(rsrc);
  T.res = up(H.res);
  T.crow = up(crow);
  T.ccol = up(ccol);
  T.csrc = up(csrc);
  return true;
}

void free_socp(ciscvx_socp* so) {
  for (void* p : so->allocs) cudaFree(p);
  delete so;
}

bool finite_pos(const double* v, int n) {
  if (!v) return true;
  for (int i = 0; i < n; ++i)
    if (!(std::isfinite(v[i]) && v[i] > 0.0)) return false;
  return true;
}
bool finite_all(const double* v, int n) {
  if (!v) return true;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace

extern "C" {

ciscvx_status ciscvx_socp_create(const ciscvx_model* m, int N, int layout, const ciscvx_socp_params* P,
                                 ciscvx_socp** out) {
  if (!m || !P || !out) return set_error(CISCVX_EINVAL, "null model, params or output");
  *out = nullptr;
  if (N < 1 || N > SOCP_MAXK) return set_error(CISCVX_EINVAL, "N must be in [1, %d] (got %d)", SOCP_MAXK, N);
  if (layout != CISCVX_FOH_NODE && layout != CISCVX_FOH_INTERVAL)
    return set_error(CISCVX_EINVAL, "unknown control layout %d", layout);
  const DevModel& M = m->host;
  const int nx = 6 * M.nb;
  if (!(std::isfinite(P->w_px) && P->w_px > 0.0) || !(std::isfinite(P->w_ep) && P->w_ep > 0.0) ||
      !(std::isfinite(P->w_torque) && P->w_torque >= 0.0))
    return set_error(CISCVX_EINVAL, "weights must be finite, w_px and w_ep > 0, w_torque >= 0");
  if (!(std::isfinite(P->s_min) && std::isfinite(P->s_max) && P->s_min >= 0.0 && P->s_min <= P->s_max))
    return set_error(CISCVX_EINVAL, "need finite 0 <= s_min <= s_max");
  if ((M.nj > 0 && !P->torque_max) || !finite_pos(P->torque_max, M.nj))
    return set_error(CISCVX_EINVAL, "torque_max must hold n_j finite values > 0");
  if (!P->x_init || !P->x_final || !finite_all(P->x_init, nx) || !finite_all(P->x_final, nx))
    return set_error(CISCVX_EINVAL, "x_init and x_final must hold n_x finite values");
  if (!finite_pos(P->scale_x, M.nxt) || !finite_pos(P->scale_u, M.nu) || !finite_pos(P->scale_phi, 2 * M.nc) ||
      !finite_pos(P->scale_gam, M.nc) || !std::isfinite(P->scale_s) || P->scale_s < 0.0 ||
      !finite_all(P->offset_x, M.nxt) || !finite_all(P->offset_u, M.nu) || !finite_all(P->offset_phi, 2 * M.nc) ||
      !finite_all(P->offset_gam, M.nc) || !std::isfinite(P->offset_s))
    return set_error(CISCVX_EINVAL, "scales must be finite > 0 and offsets finite");

  Builder B(M, N, layout);
  B.columns(*P);
  B.rows(*P);
  const int n_var = (int)B.colz.size();
  if ((long long)B.A.e.size() > INT32_MAX || (long long)B.G.e.size() > INT32_MAX)
    return set_error(CISCVX_EUNSUPPORTED, "more than 2^31 - 1 entries in a matrix");

  ciscvx_socp* so = new ciscvx_socp();
  so->N = N; so->layout = layout; so->device = m->device;
  so->nxt = M.nxt; so->nu = M.nu; so->nb = M.nb; so->nc = M.nc; so->npsi = B.npsi; so->ny = B.ny;
  so->nq = B.nq; so->w_px = P->w_px; so->w_ep = P->w_ep;

  // objective: P = w_px on problem columns + the FOH torque cost, then D P D; P o
  std::map<std::pair<int, int>, double> Pm;  // (row, col), row <= col
  for (int j = 0; j < n_var; ++j)
    if (d_kind(B.colz[j]) != Z_SLACK) Pm[{j, j}] += P->w_px;
  const double w = P->w_torque;
  if (w > 0.0)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < M.nj; ++j) {
        const int a = B.uL(k) + j, b = B.uR(k) + j;
        Pm[{a, a}] += 2.0 * w / 3.0;
        Pm[{b, b}] += 2.0 * w / 3.0;
        Pm[{std::min(a, b), std::max(a, b)}] += w / 3.0;
      }
  std::vector<double> Po(n_var, 0.0);
  so->P_colptr.assign(n_var + 1, 0);
  std::vector<std::pair<std::pair<int, int>, double>> pe(Pm.begin(), Pm.end());
  std::sort(pe.begin(), pe.end(), [](const auto& x, const auto& y) {
    return x.first.second != y.first.second ? x.first.second < y.first.second : x.first.first < y.first.first;
  });
  for (const auto& x : pe) {
    const int i = x.first.first, j = x.first.second;
    so->P_rowind.push_back(i);
    so->P_val.push_back(B.D[i] * x.second * B.D[j]);
    ++so->P_colptr[j + 1];
    Po[i] += x.second * B.o[j];
    if (i != j) Po[j] += x.second * B.o[i];
  }
  for (int c = 0; c < n_var; ++c) so->P_colptr[c + 1] += so->P_colptr[c];

  cudaError_t e = cudaSuccess;
  bool uniq = finish(B.A, n_var, so->A_colptr, so->A_rowind, so->dA, so, B.A.nrow, e) &&
              finish(B.G, n_var, so->G_colptr, so->G_rowind, so->dG, so, B.n_nonneg, e);
  auto up = [&](auto& v) {
    auto* p = upload(v, e);
    if (p) so->allocs.push_back((void*)p);
    return p;
  };
  so->consts = up(B.consts);
  so->D = up(B.D);
  so->o = up(B.o);
  so->Po = up(Po);
  so->colz = up(B.colz);
  if (!uniq) {
    free_socp(so);
    return set_error(CISCVX_EINVAL, "internal: duplicate SOCP entry");
  }
  if (e != cudaSuccess) {
    free_socp(so);
    return set_error(e == cudaErrorMemoryAllocation ? CISCVX_ENOMEM : CISCVX_ECUDA, "socp tables: %s",
                     cudaGetErrorString(e));
  }
  so->dims.n_var = n_var;
  so->dims.n_eq = B.A.nrow;
  so->dims.n_ineq = B.G.nrow;
  so->dims.n_nonneg = B.n_nonneg;
  so->dims.n_soc = B.n_soc;
  so->dims.nnz_A = (long long)B.A.e.size();
  so->dims.nnz_G = (long long)B.G.e.size();
  so->dims.nnz_P = (long long)so->P_val.size();
  *out = so;
  return set_error(CISCVX_OK, "");
}

void ciscvx_socp_destroy(ciscvx_socp* so) {
  if (so) free_socp(so);
}

ciscvx_status ciscvx_socp_get_dims(const ciscvx_socp* so, ciscvx_socp_dims* dims) {
  if (!so || !dims) return set_error(CISCVX_EINVAL, "null socp or dims");
  *dims = so->dims;
  return set_error(CISCVX_OK, "");
}

ciscvx_status ciscvx_socp_structure(const ciscvx_socp* so, int* A_colptr, int* A_rowind, int* G_colptr,
                                    int* G_rowind, int* P_colptr, int* P_rowind, double* P_values) {
  if (!so) return set_error(CISCVX_EINVAL, "null socp");
  auto cp = [](const auto& v, auto* dst) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(so->A_colptr, A_colptr); cp(so->A_rowind, A_rowind);
  cp(so->G_colptr, G_colptr); cp(so->G_rowind, G_rowind);
  cp(so->P_colptr, P_colptr); cp(so->P_rowind, P_rowind);
  cp(so->P_val, P_values);
  return set_error(CISCVX_OK, "");
}

ciscvx_status ciscvx_socp_fill(const ciscvx_socp* so, int n_inst, const ciscvx_socp_inputs* in,
                               const ciscvx_socp_outputs* out, void* stream) {
  if (!so || !in || !out) return set_error(CISCVX_EINVAL, "null socp, inputs or outputs");
  if (n_inst < 1) return set_error(CISCVX_EINVAL, "n_inst must be >= 1 (got %d)", n_inst);
  if (in->phi_precision != CISCVX_FP64 && in->phi_precision != CISCVX_FP32_PHI)
    return set_error(CISCVX_EINVAL, "phi_precision must be CISCVX_FP64 or CISCVX_FP32_PHI");
  const int nc = so->nc;
  if (!in->Xp || !in->Xm || !in->s || (so->nu > 0 && !in->U) || !in->A || !in->S || !in->defect || !in->g ||
      !in->Gvm || !in->Gth || (so->nu > 0 && (!in->Bm || !in->Bp)))
    return set_error(CISCVX_EINVAL, "null required input");
  if (nc > 0 && (!in->Phi || !in->Gam || !in->Gphi || !in->theta || !in->dtheta || !in->psi || !in->dpsi))
    return set_error(CISCVX_EINVAL, "null contact input (Phi, Gam, Gphi, theta, dtheta, psi, dpsi)");
  if (!out->A_values || !out->b || !out->G_values || !out->h || !out->c || !out->rho_A || !out->rho_G)
    return set_error(CISCVX_EINVAL, "null output");
  SocpIO I;
  std::memset(&I, 0, sizeof I);
  const int N = so->N, nxt = so->nxt, nu = so->nu, nq = so->nq;
  I.N = N; I.nxt = nxt; I.nu = nu; I.nb = so->nb; I.nc = nc; I.npsi = so->npsi; I.ny = so->ny; I.nq = nq;
  I.n_var = so->dims.n_var; I.node_layout = so->layout == CISCVX_FOH_NODE;
  I.phi64 = in->phi_precision == CISCVX_FP64;
  I.sX = (long long)(N + 1) * nxt;
  I.sU = so->layout == CISCVX_FOH_NODE ? (long long)(N + 1) * nu : (long long)N * 2 * nu;
  I.sS = N;
  I.sPhi = (long long)(N + 1) * 2 * nc;
  I.sGam = (long long)(N + 1) * nc;
  I.sA = (long long)N * nxt * nxt;
  I.sB = (long long)N * nxt * nu;
  I.sSv = (long long)N * nxt;
  I.sDef = (long long)N * nxt;
  I.sG = (long long)(N + 1) * nxt;
  I.sGvm = (long long)(N + 1) * nq * nq;
  I.sGth = (long long)(N + 1) * nq * so->nb;
  I.sGphi = (long long)(N + 1) * nq * 2 * nc;
  I.sGpx = (long long)(N + 1) * nq * nc;
  I.sTh = (long long)(N + 1) * 8 * nc;
  I.sDth = (long long)(N + 1) * nc * 8 * CISCVX_NODE_THETA_COLS;
  I.sPsi = (long long)N * so->npsi;
  I.sDpsi = (long long)N * so->npsi * so->ny;
  I.Xp = in->Xp; I.Xm = in->Xm; I.U = in->U; I.s = in->s; I.Phi = in->Phi; I.Gam = in->Gam;
  I.defect = in->defect; I.g = in->g; I.Gvm = in->Gvm; I.Gth = in->Gth; I.Gphi = in->Gphi; I.Gpx = in->Gpx;
  I.theta = in->theta; I.dtheta = in->dtheta; I.psi = in->psi; I.dpsi = in->dpsi;
  I.A = in->A; I.Bm = in->Bm; I.Bp = in->Bp; I.S = in->S;
  I.consts = so->consts; I.colz = so->colz; I.D = so->D; I.o = so->o; I.Po = so->Po;
  I.w_px = so->w_px; I.w_ep = so->w_ep;
  cudaStream_t st = (cudaStream_t)stream;
  const int bs = 256;
  auto grid = [&](long long n) { return (unsigned)((n + bs - 1) / bs); };
  const long long nA = (long long)n_inst * so->dA.nrow, nG = (long long)n_inst * so->dG.nrow;
  if (nA) k_socp_rows<<<grid(nA), bs, 0, st>>>(I, so->dA, n_inst, out->rho_A, out->b);
  if (nG) k_socp_rows<<<grid(nG), bs, 0, st>>>(I, so->dG, n_inst, out->rho_G, out->h);
  const long long vA = (long long)n_inst * so->dA.nnz, vG = (long long)n_inst * so->dG.nnz;
  if (vA) k_socp_values<<<grid(vA), bs, 0, st>>>(I, so->dA, n_inst, out->rho_A, out->A_values);
  if (vG) k_socp_values<<<grid(vG), bs, 0, st>>>(I, so->dG, n_inst, out->rho_G, out->G_values);
  k_socp_c<<<grid((long long)n_inst * I.n_var), bs, 0, st>>>(I, n_inst, out->c);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "socp launch: %s", cudaGetErrorString(e));
  return set_error(CISCVX_OK, "");
}

}  // extern "C"
