// socp.cu — the convex subproblem of one prox-linear SCP iteration (Sec. V)
// in the canonical SOCP form of a conic solver, assembled on the GPU from the
// linearization outputs (Sec. VI: CSC matrices, row normalization, affine
// variable scaling).  The variables, rows, convex set, objective and scaling
// are the ones include/ciscvx.h states for ciscvx_socp_*.
//
// Two phases.  The symbolic phase (host, once per (model, N, layout)) lays out
// the columns and rows and lists every structural entry with a 64-bit source
// descriptor: which output array holds its value, at which offset within one
// instance's part, or a constant.  It keeps the rows that depend on the
// iterate in a SELL-32 view (for the row pass) and all entries sorted into CSC
// order (for the value pass), and precomputes everything that does not depend
// on the iterate: the column scales and offsets, P, P o, and the scales and
// right-hand sides of the rows made of constants.
// The numeric phase (device, per call, any number of instances of that shape,
// IPB instances per thread):
//   zhat:   thread per column: the scaled iterate (zbar - o) / D, into c
//   rows:   thread per linearized row: rho = 1 / max |value D| over its
//           problem-variable entries, and rho (sum value D zhat - residual)
//   fixed:  the precomputed rho and right-hand side of the constant rows
//   values: thread per CSC entry: value * D[col] * rho[row]
//   c:      thread per column: D (P o - w_px zbar), or w_ep
// The descriptors are shared by all instances and stay in L2; every output is
// written once, coalesced.  FP64 throughout; the FP64 pipe bounds the row and
// value passes, so FP32 sources are widened and signs flipped on the integer
// pipe.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"

using namespace ciscvx;

namespace {

// ---------------------------------------------------------------- sources ---
// A 64-bit descriptor: bits 60..63 the array (kind), bit 59 negate, bits
// 0..58 the element offset within one instance's part of that array (or the
// index of a constant).  Three kind spaces: entry sources (SRC_*), column
// iterates (Z_*), row residuals (R_*).
enum : unsigned {
  SRC_CONST = 0, SRC_A, SRC_BM, SRC_BP, SRC_S, SRC_GVM, SRC_GTH, SRC_GPHI, SRC_GPX, SRC_DTH, SRC_DPSI, SRC_N
};
enum : unsigned { Z_SLACK = 0, Z_XP, Z_XM, Z_PHI, Z_GAM, Z_U, Z_S, Z_N };
enum : unsigned { R_CONST = 0, R_G, R_DYN, R_TH, R_PSI };

constexpr int SOCP_MAXK = (1 << 25) - 1;
constexpr uint64_t OFF_MASK = (1ull << 59) - 1;

inline uint64_t enc(unsigned kind, uint64_t off, bool neg = false) {
  return ((uint64_t)kind << 60) | ((uint64_t)(neg ? 1 : 0) << 59) | (off & OFF_MASK);
}
__host__ __device__ inline unsigned d_kind(uint64_t d) { return (unsigned)(d >> 60); }
__host__ __device__ inline bool d_neg(uint64_t d) { return (d >> 59) & 1u; }
__host__ __device__ inline long long d_off(uint64_t d) { return (long long)(d & OFF_MASK); }

// Device copy of one matrix's tables.
struct MatDev {
  int nrow;
  long long nnz;
  // the rows that depend on the iterate (linearized constraints), problem-
  // variable entries only, in SELL-32 order: groups of 32 rows (one warp),
  // entry j of the group's row `lane` at gptr[group] + 32 j + lane, padded to
  // the group's longest row with zero entries; rows sorted by length within
  // windows of SELL_WINDOW rows so that a group's rows are of similar length
  int n_lin;                 // such rows (padded to a multiple of 32)
  const int* lrow;           // [n_lin] their row indices (-1: padding)
  const long long* gptr;     // [n_lin / 32 + 1] first slot of each group
  const uint64_t* lsrc;      // source of each slot
  const int* lcol;           // its column
  const double* lD;          // its column scale (0 in padding)
  const uint64_t* lres;      // [n_lin] residual source (R_*) of each row
  // rows of constants only: rho and rho (h - G o) do not depend on the iterate
  int n_fix;
  const int* frow;           // [n_fix]
  const double* frho;        // [n_fix]
  const double* frhs;        // [n_fix]
  const int* crow;           // [nnz] row of each CSC entry
  const uint64_t* csrc;      // [nnz] source of each CSC entry
  const double* cscale;      // [nnz] D[col] (constants: the signed value times D[col])
};


// Per-call pointers and per-instance strides (elements), indexed by kind.
struct SocpIO {
  const void* sp[SRC_N];     // entry-source arrays
  long long ss[SRC_N];       // their per-instance strides
  unsigned f32;              // bit k: array k holds FP32
  const double* zp[Z_N];     // iterate arrays
  long long zs[Z_N];
  const double *g, *defect, *Xp, *Xm, *theta, *psi;
  long long sG, sDef, sX, sTh, sPsi;
  int nxt, n_var;
  const double* consts;
  const uint64_t* colz;  // [n_var] iterate source of each column
  const double* D;       // [n_var]
  const double* o;       // [n_var]
  const double* Po;      // [n_var] P o
  double w_px, w_ep;
};

// The per-kind pointer tables, copied to shared memory by each block: lanes
// of one warp index them with different kinds, which the kernel-parameter
// (constant) bank would serve one address at a time.
struct KindTab {
  const void* sp[SRC_N];
  long long ss[SRC_N];
  const double* zp[Z_N];
  long long zs[Z_N];
  unsigned f32;
};

__device__ __forceinline__ void load_tab(const SocpIO& I, KindTab& K) {
  const int t = threadIdx.x;
  if (t < SRC_N) {
    K.sp[t] = I.sp[t];
    K.ss[t] = I.ss[t];
  }
  if (t < Z_N) {
    K.zp[t] = I.zp[t];
    K.zs[t] = I.zs[t];
  }
  if (t == 0) K.f32 = I.f32;
  __syncthreads();
}

// The entry's value, its sign applied by flipping the sign bit.
__device__ __forceinline__ double fetch(const SocpIO& I, const KindTab& K, long inst, uint64_t d) {
  const unsigned kind = d_kind(d);
  const long long off = d_off(d);
  const unsigned long long neg = (unsigned long long)d_neg(d);
  if (kind == SRC_CONST) return __longlong_as_double(__double_as_longlong(I.consts[off]) ^ (long long)(neg << 63));
  const long long idx = inst * K.ss[kind] + off;
  if ((K.f32 >> kind) & 1u) return widen(__float_as_uint(((const float*)K.sp[kind])[idx]) ^ (unsigned)(neg << 31));
  return __longlong_as_double(__double_as_longlong(((const double*)K.sp[kind])[idx]) ^ (long long)(neg << 63));
}

__device__ __forceinline__ double zbar_at(const KindTab& K, long inst, uint64_t d) {
  return K.zp[d_kind(d)][inst * K.zs[d_kind(d)] + d_off(d)];
}

__device__ double residual_at(const SocpIO& I, long inst, uint64_t d) {
  const long long off = d_off(d);
  switch (d_kind(d)) {
    case R_G: return I.g[inst * I.sG + off];
    case R_DYN:  // F~(x~+_k, U_k, s_k) - x~-_{k+1}, with F~ = defect + x~+_{k+1}; off = k n_x~ + r
      return I.defect[inst * I.sDef + off] + I.Xp[inst * I.sX + off + I.nxt] - I.Xm[inst * I.sX + off + I.nxt];
    case R_TH: return I.theta[inst * I.sTh + off];
    case R_PSI: return I.psi[inst * I.sPsi + off];
    default: return I.consts[off];
  }
}

constexpr int SELL_WINDOW = 256;
constexpr int IPB = 4;  // instances per thread: the tables are read once for all of
                        // them, and each thread has IPB independent gathers in flight

// Scaled iterate zhat = (zbar - o) / D per (instance, column), 0 on slacks,
// written into the caller's c (the column pass overwrites it at the end).
__global__ void __launch_bounds__(256) k_socp_zhat(const __grid_constant__ SocpIO I, int n_inst, double* zhat) {
  __shared__ KindTab K;
  load_tab(I, K);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= I.n_var) return;
  const uint64_t zc = I.colz[j];
  const double idj = 1.0 / I.D[j], oj = I.o[j];
  for (long base = (long)blockIdx.y * IPB; base < n_inst; base += (long)gridDim.y * IPB)
#pragma unroll
    for (int i = 0; i < IPB; ++i)
      if (base + i < n_inst)
        zhat[(base + i) * I.n_var + j] = d_kind(zc) == Z_SLACK ? 0.0 : (zbar_at(K, base + i, zc) - oj) * idj;
}

// Row pass over the linearized rows: thread per (row, IPB instances).  With
// m = value x D: rho = 1 / max |m| (the max taken on the bit patterns of
// the magnitudes, which order like the values), and
// rhs = rho (sum m zhat - residual) = rho (J zbar - residual - J o).
__global__ void __launch_bounds__(256) k_socp_rows(const __grid_constant__ SocpIO I, MatDev T, int n_inst,
                                                   const double* zhat, double* rho_out, double* rhs_out) {
  __shared__ KindTab K;
  load_tab(I, K);
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= T.n_lin) return;
  const int r = T.lrow[w];
  const long long g0 = T.gptr[w >> 5], g1 = T.gptr[(w >> 5) + 1];
  const uint64_t rd = T.lres[w];
  for (long base = (long)blockIdx.y * IPB; base < n_inst; base += (long)gridDim.y * IPB) {
    unsigned long long mx[IPB];
    double acc[IPB];
#pragma unroll
    for (int i = 0; i < IPB; ++i) {
      mx[i] = 0ull;
      acc[i] = 0.0;
    }
    for (long long e = g0 + (w & 31); e < g1; e += 32) {
      const uint64_t d = T.lsrc[e];
      const int c = T.lcol[e];
      const double dc = T.lD[e];
#pragma unroll
      for (int i = 0; i < IPB; ++i) {
        if (base + i >= n_inst) break;
        const double m = fetch(I, K, base + i, d) * dc;
        mx[i] = ullmax(mx[i], (unsigned long long)__double_as_longlong(m) & 0x7FFFFFFFFFFFFFFFull);
        acc[i] = fma(m, zhat[(base + i) * I.n_var + c], acc[i]);
      }
    }
    if (r < 0) continue;  // padding row
#pragma unroll
    for (int i = 0; i < IPB; ++i) {
      if (base + i >= n_inst) break;
      const long inst = base + i;
      const double nrm = __longlong_as_double((long long)mx[i]);
      const double rho = nrm > 0.0 ? 1.0 / nrm : 1.0;
      rho_out[inst * T.nrow + r] = rho;
      rhs_out[inst * T.nrow + r] = rho * (acc[i] - residual_at(I, inst, rd));
    }
  }
}

// Rows of constants: their precomputed rho and right-hand side, per instance.
__global__ void __launch_bounds__(256) k_socp_fixed(MatDev T, int n_inst, double* rho_out, double* rhs_out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= T.n_fix) return;
  const int r = T.frow[w];
  const double rho = T.frho[w], rhs = T.frhs[w];
  for (long inst = blockIdx.y; inst < n_inst; inst += gridDim.y) {
    rho_out[inst * T.nrow + r] = rho;
    rhs_out[inst * T.nrow + r] = rhs;
  }
}

// Value pass: thread per (CSC entry, IPB instances).
__global__ void __launch_bounds__(256) k_socp_values(const __grid_constant__ SocpIO I, MatDev T, int n_inst,
                                                      const double* rho, double* val) {
  __shared__ KindTab K;
  load_tab(I, K);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= T.nnz) return;
  const uint64_t d = T.csrc[e];
  const double sc = T.cscale[e];
  const int row = T.crow[e];
  const bool cst = d_kind(d) == SRC_CONST;
  for (long base = (long)blockIdx.y * IPB; base < n_inst; base += (long)gridDim.y * IPB) {
    double v[IPB];
#pragma unroll
    for (int i = 0; i < IPB; ++i) {
      v[i] = 0.0;
      if (base + i < n_inst) v[i] = (cst ? sc : fetch(I, K, base + i, d) * sc) * rho[(base + i) * T.nrow + row];
    }
#pragma unroll
    for (int i = 0; i < IPB; ++i)
      if (base + i < n_inst) val[(base + i) * T.nnz + e] = v[i];
  }
}

// Column pass: c, thread per (column, IPB instances).
__global__ void __launch_bounds__(256) k_socp_c(const __grid_constant__ SocpIO I, int n_inst, double* c) {
  __shared__ KindTab K;
  load_tab(I, K);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= I.n_var) return;
  const uint64_t zc = I.colz[j];
  const double dj = I.D[j], poj = I.Po[j];
  for (long base = (long)blockIdx.y * IPB; base < n_inst; base += (long)gridDim.y * IPB)
#pragma unroll
    for (int i = 0; i < IPB; ++i)
      if (base + i < n_inst)
        c[(base + i) * I.n_var + j] = d_kind(zc) == Z_SLACK ? I.w_ep : dj * (poj - I.w_px * zbar_at(K, base + i, zc));
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

  bool compact = false;  // A, Bm, Bp inputs hold the pattern's nonzeros only

  Builder(const DevModel& m, int N_, int layout) : M(m), N(N_) {
    nxt = M.nxt; nu = M.nu; nb = M.nb; nj = M.nj; nc = M.nc;
    nq = 3 * nb; nx = 6 * nb; ny = nxt - nx;
    aux = M.aux != 0; jelim = M.jelim != 0; terrain = M.ta != 0.0;
    npsi = aux ? 3 * nc : nc;
    node = layout == CISCVX_FOH_NODE;
    // every model has a structural pattern (coupled links: column-major, the
    // integrated columns full); the dynamics rows take only its entries
    has_pattern = true;
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
  uint64_t one(bool neg = false) { return enc(SRC_CONST, cst(1.0), neg); }
  uint64_t value(double v) { return enc(SRC_CONST, cst(v)); }
  uint64_t rconst(double v) { return enc(R_CONST, cst(v)); }

  // entry source: element (k, off) of an output block, as a per-instance offset
  uint64_t desc(unsigned kind, long k, unsigned off, bool neg = false) const {
    long long blk = 0;
    switch (kind) {
      case SRC_A: blk = compact ? (long long)M.nnzA : (long long)nxt * nxt; break;
      case SRC_BM: case SRC_BP: blk = compact ? (long long)M.nnzB : (long long)nxt * nu; break;
      case SRC_S: blk = nxt; break;
      case SRC_GVM: blk = (long long)nq * nq; break;
      case SRC_GTH: blk = (long long)nq * nb; break;
      case SRC_GPHI: blk = (long long)nq * 2 * nc; break;
      case SRC_GPX: blk = (long long)nq * nc; break;
      case SRC_DTH: blk = (long long)nc * 8 * CISCVX_NODE_THETA_COLS; break;
      case SRC_DPSI: blk = (long long)npsi * ny; break;
    }
    return enc(kind, (uint64_t)(k * blk + off), neg);
  }
  // row residual: element (k, off) of g, defect, theta or psi
  uint64_t rdesc(unsigned kind, long k, unsigned off) const {
    const long long blk = kind == R_TH ? 8LL * nc : kind == R_PSI ? (long long)npsi : (long long)nxt;
    return enc(kind, (uint64_t)(k * blk + off));
  }
  // column iterate: component i of node / interval k (ZB_UL, ZB_UR: the
  // per-interval control layout's u_L, u_R)
  enum : unsigned { ZB_UL = 100, ZB_UR = 101 };
  uint64_t zdesc(unsigned zk, long k, int i) const {
    switch (zk) {
      case Z_XP: case Z_XM: return enc(zk, (uint64_t)(k * nxt + i));
      case Z_PHI: return enc(zk, (uint64_t)(k * 2 * nc + i));
      case Z_GAM: return enc(zk, (uint64_t)(k * nc + i));
      case Z_U: return enc(Z_U, (uint64_t)(k * nu + i));
      case ZB_UL: return enc(Z_U, (uint64_t)(2 * k * nu + i));
      case ZB_UR: return enc(Z_U, (uint64_t)((2 * k + 1) * nu + i));
      case Z_S: return enc(Z_S, (uint64_t)k);
    }
    return 0;
  }

  // columns: n of them, iterate source kind zk at index k (components 0..n-1),
  // scale/offset vectors sc/of of length n (null = identity) or slack
  int take(std::vector<int>& v, int n, unsigned zk, long k, const double* sc, const double* of) {
    const int c0 = (int)colz.size();
    v.push_back(c0);
    for (int i = 0; i < n; ++i) {
      colz.push_back(zk == Z_SLACK ? 0 : zdesc(zk, k, i));
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
          take(c_uL, nu, ZB_UL, k, P.scale_u, P.offset_u);
          take(c_uR, nu, ZB_UR, k, P.scale_u, P.offset_u);
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
    cst(0.0);  // the padding entries of the SELL layout point at it
    for (int k = 0; k <= N; ++k) {
      // G~ rows of node k
      for (int r = 0; r < nxt; ++r) {
        const int row = A.begin_row(rdesc(R_G, k, (unsigned)r));
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
          const int row = A.begin_row(rdesc(R_DYN, k, (unsigned)r));
          if (has_pattern) {
            for (size_t e = 0; e < par.size(); ++e)
              if (par[e] == r)
                A.add(row, c_xp[k] + pac[e], desc(SRC_A, k, (unsigned)(compact ? e : r * nxt + pac[e])));
          } else {
            for (int c = 0; c < nxt; ++c) A.add(row, c_xp[k] + c, desc(SRC_A, k, (unsigned)(r * nxt + c)));
          }
          A.add(row, c_xm[k + 1] + r, one(true));
          auto badd = [&](int q, unsigned off) {
            A.add(row, uL(k) + q, desc(SRC_BM, k, off));
            A.add(row, uR(k) + q, desc(SRC_BP, k, off));
          };
          if (has_pattern) {
            for (size_t e = 0; e < pbr.size(); ++e)
              if (pbr[e] == r) badd(pbc[e], (unsigned)(compact ? e : r * nu + pbc[e]));
          } else {
            for (int q = 0; q < nu; ++q) badd(q, (unsigned)(r * nu + q));
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
          const int row = G.begin_row(rdesc(R_TH, k, (unsigned)(8 * i + j)));
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
          const int row = G.begin_row(rdesc(R_PSI, k, (unsigned)r));
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
  int nnzA, nnzB;  // per-interval sizes of compact A and B- / B+ (0: dense)
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
bool finish(const HostMat& H, const Builder& B, std::vector<int>& colptr, std::vector<int>& rowind,
            MatDev& T, ciscvx_socp* so, int soc0, cudaError_t& e) {
  const int n_var = (int)B.colz.size();
  const long long nnz = (long long)H.e.size();
  std::vector<int> rowptr(H.nrow + 1, 0), crow(nnz);
  std::vector<uint64_t> csrc(nnz);
  std::vector<double> cscale(nnz);
  for (long long i = 0; i < nnz; ++i) ++rowptr[H.e[i].row + 1];
  for (int r = 0; r < H.nrow; ++r) rowptr[r + 1] += rowptr[r];
  auto is_problem = [&](int col) { return d_kind(B.colz[col]) != Z_SLACK; };
  auto cval = [&](uint64_t d) { return (d_neg(d) ? -1.0 : 1.0) * B.consts[d_off(d)]; };
  // rows that depend on the iterate, and rows of constants (rho and h precomputed)
  std::vector<int> lin, lrow, lcol, frow;
  std::vector<long long> gptr{0};
  std::vector<uint64_t> lsrc, lres;
  std::vector<double> lD, frho, frhs, fnrm(H.nrow, 0.0);
  auto nprob = [&](int r) {
    int n = 0;
    for (int i = rowptr[r]; i < rowptr[r + 1]; ++i) n += is_problem(H.e[i].col);
    return n;
  };
  for (int r = 0; r < H.nrow; ++r) {
    if (d_kind(H.res[r]) != R_CONST) {
      lin.push_back(r);
    } else {
      for (int i = rowptr[r]; i < rowptr[r + 1]; ++i) {
        const Entry& x = H.e[i];
        if (d_kind(x.src) != SRC_CONST) return false;  // constant rows hold constants only
        if (is_problem(x.col)) fnrm[r] = std::max(fnrm[r], std::fabs(cval(x.src) * B.D[x.col]));
      }
    }
  }
  // SELL-32 layout of the linearized rows
  for (size_t w0 = 0; w0 < lin.size(); w0 += SELL_WINDOW) {
    const size_t w1 = std::min(lin.size(), w0 + SELL_WINDOW);
    std::stable_sort(lin.begin() + w0, lin.begin() + w1, [&](int a, int b) { return nprob(a) > nprob(b); });
  }
  while (lin.size() % 32) lin.push_back(-1);
  const uint64_t zero = enc(SRC_CONST, (uint64_t)std::distance(
      B.consts.begin(), std::find(B.consts.begin(), B.consts.end(), 0.0)));
  for (size_t g = 0; g < lin.size(); g += 32) {
    int width = 0;
    for (int l = 0; l < 32; ++l) width = std::max(width, lin[g + l] < 0 ? 0 : nprob(lin[g + l]));
    const size_t base = lsrc.size();
    lsrc.resize(base + 32 * (size_t)width, zero);
    lcol.resize(base + 32 * (size_t)width, 0);
    lD.resize(base + 32 * (size_t)width, 0.0);
    for (int l = 0; l < 32; ++l) {
      const int r = lin[g + l];
      lrow.push_back(r);
      lres.push_back(r < 0 ? 0 : H.res[r]);
      if (r < 0) continue;
      int j = 0;
      for (int i = rowptr[r]; i < rowptr[r + 1]; ++i) {
        const Entry& x = H.e[i];
        if (!is_problem(x.col)) continue;
        const size_t slot = base + 32 * (size_t)j + l;
        lsrc[slot] = x.src;
        lcol[slot] = x.col;
        lD[slot] = B.D[x.col];
        ++j;
      }
    }
    gptr.push_back((long long)lsrc.size());
  }
  for (int r = 0; r < H.nrow; ++r) {
    if (d_kind(H.res[r]) != R_CONST) continue;
    double nrm = fnrm[r];
    if (r >= soc0) nrm = std::max(nrm, fnrm[soc0 + ((r - soc0) ^ 1)]);  // a Q^2 block shares its scale
    double go = 0.0;
    for (int i = rowptr[r]; i < rowptr[r + 1]; ++i)
      if (is_problem(H.e[i].col)) go += cval(H.e[i].src) * B.o[H.e[i].col];
    const double rho = nrm > 0.0 ? 1.0 / nrm : 1.0;
    frow.push_back(r);
    frho.push_back(rho);
    frhs.push_back(rho * (B.consts[d_off(H.res[r])] - go));
  }
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
    csrc[i] = x.src;
    // the column scale, with a constant's signed value folded in
    cscale[i] = B.D[x.col] * (d_kind(x.src) == SRC_CONST ? cval(x.src) : 1.0);
    rowind[i] = x.row;
    ++colptr[x.col + 1];
  }
  for (int c = 0; c < n_var; ++c) colptr[c + 1] += colptr[c];
  T.nrow = H.nrow;
  T.nnz = nnz;
  T.n_lin = (int)lrow.size();
  T.n_fix = (int)frow.size();
  auto up = [&](auto& v) {
    auto* p = upload(v, e);
    if (p) so->allocs.push_back((void*)p);
    return p;
  };
  T.lrow = up(lrow);
  T.gptr = up(gptr);
  T.lsrc = up(lsrc);
  T.lcol = up(lcol);
  T.lD = up(lD);
  T.lres = up(lres);
  T.frow = up(frow);
  T.frho = up(frho);
  T.frhs = up(frhs);
  T.crow = up(crow);
  T.csrc = up(csrc);
  T.cscale = up(cscale);
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

  if (P->phi_format != CISCVX_OUT_DENSE && P->phi_format != CISCVX_OUT_COMPACT)
    return set_error(CISCVX_EINVAL, "unknown phi_format %d", P->phi_format);
  Builder B(M, N, layout);
  B.compact = P->phi_format == CISCVX_OUT_COMPACT;
  if (B.compact && !B.has_pattern)
    return set_error(CISCVX_EUNSUPPORTED, "compact inputs need a model with a structural pattern");
  B.columns(*P);
  B.rows(*P);
  const int n_var = (int)B.colz.size();
  if ((long long)B.A.e.size() > INT32_MAX || (long long)B.G.e.size() > INT32_MAX)
    return set_error(CISCVX_EUNSUPPORTED, "more than 2^31 - 1 entries in a matrix");

  ciscvx_socp* so = new ciscvx_socp();
  so->N = N; so->layout = layout; so->device = m->device;
  so->nxt = M.nxt; so->nu = M.nu; so->nb = M.nb; so->nc = M.nc; so->npsi = B.npsi; so->ny = B.ny;
  so->nq = B.nq; so->w_px = P->w_px; so->w_ep = P->w_ep;
  so->nnzA = B.compact ? M.nnzA : 0;
  so->nnzB = B.compact ? M.nnzB : 0;

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
  bool uniq = finish(B.A, B, so->A_colptr, so->A_rowind, so->dA, so, B.A.nrow, e) &&
              finish(B.G, B, so->G_colptr, so->G_rowind, so->dG, so, B.n_nonneg, e);
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
    return set_error(CISCVX_EINVAL, "internal: duplicate SOCP entry or a non-constant fixed row");
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
  const long long N = so->N, nxt = so->nxt, nu = so->nu, nq = so->nq, nb = so->nb, npsi = so->npsi, ny = so->ny;
  const bool f32 = in->phi_precision == CISCVX_FP32_PHI;
  auto src = [&](unsigned k, const void* p, long long stride) {
    I.sp[k] = p;
    I.ss[k] = stride;
  };
  src(SRC_A, in->A, so->nnzA ? N * so->nnzA : N * nxt * nxt);
  src(SRC_BM, in->Bm, so->nnzB ? N * so->nnzB : N * nxt * nu);
  src(SRC_BP, in->Bp, so->nnzB ? N * so->nnzB : N * nxt * nu);
  src(SRC_S, in->S, N * nxt);
  src(SRC_GVM, in->Gvm, (N + 1) * nq * nq);
  src(SRC_GTH, in->Gth, (N + 1) * nq * nb);
  src(SRC_GPHI, in->Gphi, (N + 1) * nq * 2 * nc);
  src(SRC_GPX, in->Gpx, (N + 1) * nq * nc);
  src(SRC_DTH, in->dtheta, (N + 1) * nc * 8 * CISCVX_NODE_THETA_COLS);
  src(SRC_DPSI, in->dpsi, N * npsi * ny);
  I.f32 = f32 ? (1u << SRC_A) | (1u << SRC_BM) | (1u << SRC_BP) | (1u << SRC_S) : 0u;
  auto zsrc = [&](unsigned k, const double* p, long long stride) {
    I.zp[k] = p;
    I.zs[k] = stride;
  };
  zsrc(Z_XP, in->Xp, (N + 1) * nxt);
  zsrc(Z_XM, in->Xm, (N + 1) * nxt);
  zsrc(Z_PHI, in->Phi, (N + 1) * 2 * nc);
  zsrc(Z_GAM, in->Gam, (N + 1) * nc);
  zsrc(Z_U, in->U, so->layout == CISCVX_FOH_NODE ? (N + 1) * nu : N * 2 * nu);
  zsrc(Z_S, in->s, N);
  I.g = in->g; I.sG = (N + 1) * nxt;
  I.defect = in->defect; I.sDef = N * nxt;
  I.Xp = in->Xp; I.Xm = in->Xm; I.sX = (N + 1) * nxt;
  I.theta = in->theta; I.sTh = (N + 1) * 8 * nc;
  I.psi = in->psi; I.sPsi = N * npsi;
  I.nxt = (int)nxt; I.n_var = so->dims.n_var;
  I.consts = so->consts; I.colz = so->colz; I.D = so->D; I.o = so->o; I.Po = so->Po;
  I.w_px = so->w_px; I.w_ep = so->w_ep;
  cudaStream_t st = (cudaStream_t)stream;
  const int bs = 256;
  const unsigned gy = (unsigned)std::min((n_inst + IPB - 1) / IPB, 65535);
  auto grid = [&](long long n, int per) { return dim3((unsigned)((n + per - 1) / per), gy); };
  // zhat into c, the row passes read it, the column pass overwrites it with c
  k_socp_zhat<<<grid(I.n_var, bs), bs, 0, st>>>(I, n_inst, out->c);
  for (int w = 0; w < 2; ++w) {
    const MatDev& T = w == 0 ? so->dA : so->dG;
    double* rho = w == 0 ? out->rho_A : out->rho_G;
    double* rhs = w == 0 ? out->b : out->h;
    if (T.n_lin) k_socp_rows<<<grid(T.n_lin, bs), bs, 0, st>>>(I, T, n_inst, out->c, rho, rhs);
    if (T.n_fix)
      k_socp_fixed<<<dim3((unsigned)((T.n_fix + bs - 1) / bs), (unsigned)std::min(n_inst, 65535)), bs, 0, st>>>(
          T, n_inst, rho, rhs);
  }
  for (int w = 0; w < 2; ++w) {
    const MatDev& T = w == 0 ? so->dA : so->dG;
    if (T.nnz)
      k_socp_values<<<grid(T.nnz, bs), bs, 0, st>>>(I, T, n_inst, w == 0 ? out->rho_A : out->rho_G,
                                                     w == 0 ? out->A_values : out->G_values);
  }
  k_socp_c<<<grid(I.n_var, bs), bs, 0, st>>>(I, n_inst, out->c);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "socp launch: %s", cudaGetErrorString(e));
  return set_error(CISCVX_OK, "");
}

}  // extern "C"
