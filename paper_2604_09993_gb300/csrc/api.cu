// api.cu — host side of the C ABI declared in include/ciscvx.h.
//
// Validation, the per-link device tables (coefficients of every input on every
// link, see common.cuh), the device status word, thread-local error messages
// and the launches.  Compute calls allocate nothing.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>
#include <new>
#include <string>

#include "coupled.cuh"

using namespace ciscvx;

namespace {

thread_local std::string g_err;

ciscvx_status fail(ciscvx_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

ciscvx_status ok() {
  g_err.clear();
  return CISCVX_OK;
}

bool finite2(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]); }

// Input i of link B exerts a torque on it (the Eq. (12) model's gamma exerts
// no force at all).
bool input_torque(const DevBody& B, int i) { return B.p[i] != 0.0 || B.q[i] != 0.0 || B.t[i] != 0.0; }

// Input i of a foot link enters its contact's lambda^c row (Eq. (12) model):
// through v_x or the rotation, or directly (phi_t, gamma).
bool input_lambda(const DevBody& B, int i) {
  const int d = B.idx[i] - B.cin;
  return B.ax[i] != 0.0 || input_torque(B, i) || d == 0 || d == 2;
}

// Adds input `q` acting on link `b` with the given coefficients.
ciscvx_status add_input(DevModel& M, int b, int q, double ax, double ay, double p, double qq,
                        double t) {
  DevBody& B = M.body[b];
  if (B.nin >= MAXIN)
    return fail(CISCVX_EUNSUPPORTED, "link %d has more than %d inputs acting on it", b, MAXIN);
  const int i = B.nin++;
  B.idx[i] = q;
  B.ax[i] = ax; B.ay[i] = ay; B.p[i] = p; B.q[i] = qq; B.t[i] = t;
  return CISCVX_OK;
}

// Symbolic part of the node kernel's factorization of K = C' M^-1 C'^T (for
// forests of at most NODE_MAXJ joints): a children-first order of the joints
// (depth-first post-order from the roots), each row's first stored column
// (the earliest joint sharing a link with it) and the skyline offsets.
void node_symbolic(DevModel& M) {
  const int nj = M.nj, nb = M.nb;
  if (!M.tree || nj > NODE_MAXJ) return;
  for (int b = 0; b < nb; ++b)
    if (M.nadj[b] > NODE_MAXADJ) return;
  // joint whose child is link b (or -1)
  int pj[MAXB];
  for (int b = 0; b < nb; ++b) pj[b] = -1;
  for (int j = 0; j < nj; ++j) pj[M.jchi[j]] = j;
  int pos = 0;
  bool done[MAXJ] = {false};
  // iterative post-order: a joint is emitted once every joint hanging below its child link is
  int stack[MAXJ], sp = 0;
  for (int r = 0; r < nj; ++r) {
    if (pj[M.jpar[r]] >= 0) continue;  // not a root
    stack[sp++] = r;
    while (sp > 0) {
      const int j = stack[sp - 1];
      int next = -1;
      for (int c = 0; c < nj; ++c)
        if (!done[c] && M.jpar[c] == M.jchi[j]) { next = c; break; }
      if (next >= 0) { stack[sp++] = next; continue; }
      done[j] = true;
      M.nord[pos] = j;
      M.npos[j] = pos++;
      --sp;
    }
  }
  for (int j = 0; j < nj; ++j)
    if (!done[j]) { M.nord[pos] = j; M.npos[j] = pos++; }  // unreachable for a forest
  const int nk = 2 * nj;
  int off = 0;
  for (int i = 0; i < nk; ++i) {
    const int j = M.nord[i >> 1];
    int first = M.npos[j];
    for (int q = 0; q < nj; ++q) {
      const bool share = M.jchi[q] == M.jchi[j] || M.jchi[q] == M.jpar[j] ||
                         M.jpar[q] == M.jchi[j] || M.jpar[q] == M.jpar[j];
      if (share && M.npos[q] < first) first = M.npos[q];
    }
    M.nf[i] = 2 * first;
    M.noff[i] = off;
    off += i - M.nf[i] + 1;
  }
  M.noff[nk] = off;
  for (int b = 0; b < nb; ++b) {
    int lo = nk;
    for (int t = 0; t < M.nadj[b] && t < NODE_MAXADJ; ++t) lo = std::min(lo, 2 * M.npos[M.adj[b][t] >> 1]);
    M.lmin[b] = lo;
  }
}

ciscvx_status build_tables(const ciscvx_model_desc* d, DevModel& M) {
  std::memset(&M, 0, sizeof M);
  const int nb = d->n_bodies, nj = d->n_joints, nc = d->n_contacts;
  M.nb = nb; M.nj = nj; M.nc = nc;
  M.aux = d->aux_model;
  M.jelim = d->joint_forces;
  M.scheme = d->scheme;
  M.ta = d->terrain_amp;
  M.tk = d->terrain_wavenumber;
  if (M.ta == 0.0) M.tk = 0.0;
  M.ny = (M.aux ? 5 : 1) * nc;
  M.nxt = 6 * nb + M.ny;
  M.nu = (M.jelim ? 1 : 3) * nj + 3 * nc;
  M.g = d->gravity;
  M.tree = 1;
  for (int b = 0; b < nb; ++b) {
    M.body[b].contact = -1;
    M.body[b].cin = -1;
    M.mass[b] = d->bodies[b].mass;
    M.inertia[b] = d->bodies[b].inertia;
    M.minv[b] = 1.0 / d->bodies[b].mass;
    M.iinv[b] = 1.0 / d->bodies[b].inertia;
  }
  for (int j = 0; j < nj; ++j) {
    const ciscvx_joint_desc& J = d->joints[j];
    for (int role = 0; role < 2; ++role) {
      const int b = role ? J.parent : J.child;
      if (b >= 0 && b < nb) {
        if (M.nadj[b] < NODE_MAXADJ) M.adj[b][M.nadj[b]] = (j << 1) | role;
        ++M.nadj[b];  // counts past NODE_MAXADJ mark the model as outside the node kernel
      }
    }
    M.jpar[j] = J.parent;
    M.jchi[j] = J.child;
    M.jrp[j][0] = J.rho_parent[0]; M.jrp[j][1] = J.rho_parent[1];
    M.jrc[j][0] = J.rho_child[0]; M.jrc[j][1] = J.rho_child[1];
    for (int i = 0; i < j; ++i)
      if (d->joints[i].child == J.child) M.tree = 0;
  }
  for (int b = 0; b < nb; ++b) {
    const double m = d->bodies[b].mass, I = d->bodies[b].inertia;
    if (!(std::isfinite(m) && m > 0) || !(std::isfinite(I) && I > 0))
      return fail(CISCVX_EINVAL, "link %d: mass and inertia must be finite and > 0", b);
  }
  for (int j = 0; j < nj; ++j) {
    const ciscvx_joint_desc& J = d->joints[j];
    if (J.parent < 0 || J.parent >= nb || J.child < 0 || J.child >= nb || J.parent == J.child)
      return fail(CISCVX_EINVAL, "joint %d: parent/child must be distinct links in [0,%d)", j, nb);
    if (!finite2(J.rho_parent) || !finite2(J.rho_child))
      return fail(CISCVX_EINVAL, "joint %d: non-finite anchor", j);
    const int c = J.child, p = J.parent;
    const double mc = d->bodies[c].mass, Ic = d->bodies[c].inertia;
    const double mp = d->bodies[p].mass, Ip = d->bodies[p].inertia;
    const double cx = J.rho_child[0], cy = J.rho_child[1];
    const double px = J.rho_parent[0], py = J.rho_parent[1];
    ciscvx_status st;
    // torque: +tau on the child, -tau on the parent
    if ((st = add_input(M, c, j, 0, 0, 0, 0, 1.0 / Ic))) return st;
    if ((st = add_input(M, p, j, 0, 0, 0, 0, -1.0 / Ip))) return st;
    if (M.jelim) continue;  // reaction forces are not inputs (coupled path)
    // lambda_x: +e_x on the child at rho_c, -e_x on the parent at rho_p
    //   rho x e_x = -rho_y, rho . e_x = rho_x
    if ((st = add_input(M, c, nj + 2 * j, 1.0 / mc, 0, -cy / Ic, cx / Ic, 0))) return st;
    if ((st = add_input(M, p, nj + 2 * j, -1.0 / mp, 0, py / Ip, -px / Ip, 0))) return st;
    // lambda_y: rho x e_y = rho_x, rho . e_y = rho_y
    if ((st = add_input(M, c, nj + 2 * j + 1, 0, 1.0 / mc, cx / Ic, cy / Ic, 0))) return st;
    if ((st = add_input(M, p, nj + 2 * j + 1, 0, -1.0 / mp, -px / Ip, -py / Ip, 0))) return st;
  }
  for (int i = 0; i < nc; ++i) {
    const ciscvx_contact_desc& C = d->contacts[i];
    if (C.body < 0 || C.body >= nb) return fail(CISCVX_EINVAL, "contact %d: bad link %d", i, C.body);
    if (!finite2(C.rho) || !std::isfinite(C.mu) || C.mu < 0)
      return fail(CISCVX_EINVAL, "contact %d: non-finite point or negative mu", i);
    DevBody& B = M.body[C.body];
    if (B.contact >= 0)
      return fail(CISCVX_EUNSUPPORTED, "link %d carries more than one contact", C.body);
    B.contact = i;
    B.cin = (M.jelim ? 1 : 3) * nj + 3 * i;
    B.crho[0] = C.rho[0]; B.crho[1] = C.rho[1];
    B.mu = C.mu;
    const double m = d->bodies[C.body].mass, I = d->bodies[C.body].inertia;
    const double rx = C.rho[0], ry = C.rho[1];
    ciscvx_status st;
    if (M.aux) {
      // Eq. (12) model: phi_t: +e_x;  phi_n: +e_y;  gamma: no force (it enters the auxiliary state only)
      if ((st = add_input(M, C.body, B.cin, 1.0 / m, 0, -ry / I, rx / I, 0))) return st;
      if ((st = add_input(M, C.body, B.cin + 1, 0, 1.0 / m, rx / I, ry / I, 0))) return st;
      if ((st = add_input(M, C.body, B.cin + 2, 0, 0, 0, 0, 0))) return st;
    } else {
      // lambda_n: +e_y;  lambda_t+: +e_x;  lambda_t-: -e_x
      if ((st = add_input(M, C.body, B.cin, 0, 1.0 / m, rx / I, ry / I, 0))) return st;
      if ((st = add_input(M, C.body, B.cin + 1, 1.0 / m, 0, -ry / I, rx / I, 0))) return st;
      if ((st = add_input(M, C.body, B.cin + 2, -1.0 / m, 0, ry / I, -rx / I, 0))) return st;
    }
  }
  // VJP slots: link b's inputs occupy slots [slot0, slot0 + nin)
  int slot = 0;
  for (int b = 0; b < nb; ++b) {
    M.body[b].slot0 = slot;
    for (int i = 0; i < M.body[b].nin; ++i) {
      const int q = M.body[b].idx[i];
      if (M.in_n[q] >= 2) return fail(CISCVX_EINVAL, "input %d acts on more than two links", q);
      M.in_slot[q][M.in_n[q]++] = slot + i;
    }
    slot += M.body[b].nin;
  }
  M.nslot = slot;
  // compact output offsets (see common.cuh for the entry order)
  int aoff = 0, boff = 0;
  for (int b = 0; b < nb; ++b) {
    DevBody& B = M.body[b];
    const bool cross = M.aux && B.contact >= 0;
    B.a_off = aoff;
    B.b_off = boff;
    aoff += A_PER_LINK + (B.contact >= 0 ? A_PER_FOOT : 0) + (cross ? A_PER_CROSS : 0);
    for (int i = 0; i < B.nin; ++i)
      boff += (input_torque(B, i) ? 2 : 0) + (B.ax[i] != 0.0 ? 2 : 0) + (B.ay[i] != 0.0 ? 2 : 0) +
              (B.contact >= 0 ? 1 : 0);
    if (cross) {
      for (int i = 0; i < B.nin; ++i) boff += input_lambda(B, i) ? 1 : 0;
      boff += B_CROSS_FIXED;
    }
  }
  M.nnzA = aoff;
  M.nnzB = boff;
  if (cpl_needed(M)) {  // coupled links: the column-major pattern of fill_pattern
    M.nnzA = 0;
    for (int c = 0; c < M.nxt; ++c) M.nnzA += cpl_col_nnz(M, c);
    M.nnzB = M.nxt * M.nu;
  }
  node_symbolic(M);
  return CISCVX_OK;
}

// Checks of the description that come before the tables are built.
ciscvx_status check_desc(const ciscvx_model_desc* desc) {
  if (desc->n_bodies < 1 || desc->n_joints < 0 || desc->n_contacts < 0)
    return fail(CISCVX_EINVAL, "need n_bodies >= 1, n_joints >= 0, n_contacts >= 0");
  if (!desc->bodies || (desc->n_joints > 0 && !desc->joints) ||
      (desc->n_contacts > 0 && !desc->contacts))
    return fail(CISCVX_EINVAL, "null body/joint/contact array");
  if (desc->n_bodies > MAXB || desc->n_joints > MAXJ || desc->n_contacts > MAXB)
    return fail(CISCVX_EUNSUPPORTED, "at most %d links, %d joints, %d contacts", MAXB, MAXJ, MAXB);
  if (!std::isfinite(desc->gravity)) return fail(CISCVX_EINVAL, "non-finite gravity");
  if (desc->aux_model != CISCVX_AUX_PENALTY && desc->aux_model != CISCVX_AUX_CROSS)
    return fail(CISCVX_EINVAL, "unknown aux_model %d", desc->aux_model);
  if (desc->joint_forces != CISCVX_JOINT_FORCE_INPUT && desc->joint_forces != CISCVX_JOINT_FORCE_ELIMINATED)
    return fail(CISCVX_EINVAL, "unknown joint_forces %d", desc->joint_forces);
  if (desc->scheme != CISCVX_RK4 && desc->scheme != CISCVX_RKF45)
    return fail(CISCVX_EINVAL, "unknown scheme %d", desc->scheme);
  if (!std::isfinite(desc->terrain_amp) || !std::isfinite(desc->terrain_wavenumber))
    return fail(CISCVX_EINVAL, "non-finite terrain parameters");
  return CISCVX_OK;
}

// The compact pattern of the built tables, in the order the kernels store it
// (see common.cuh; for a model with coupled links column-major, see
// cpl_col_kind); the arrays may be null.
void fill_pattern(const DevModel& M, int32_t* ar, int32_t* ac, int32_t* br, int32_t* bc) {
  if (cpl_needed(M)) {
    int j = 0;
    for (int c = 0; c < M.nxt; ++c) {
      const int kind = cpl_col_kind(M, c);
      auto put = [&](int r) { if (ar) ar[j] = r; if (ac) ac[j] = c; ++j; };
      if (kind == 0) for (int r = 0; r < M.nxt; ++r) put(r);
      else if (kind == 2) { put(c - 3 * M.nb); put(c); }
      else put(c);
    }
    for (int q = 0, e = 0; q < M.nu; ++q)
      for (int r = 0; r < M.nxt; ++r, ++e) { if (br) br[e] = r; if (bc) bc[e] = q; }
    return;
  }
  const int nb = M.nb;
  for (int b = 0; b < nb; ++b) {
    const DevBody& B = M.body[b];
    const bool cross = M.aux && B.contact >= 0;
    const int px = 3 * b, py = px + 1, th = px + 2;
    const int vx = 3 * nb + 3 * b, vy = vx + 1, om = vx + 2;
    // the contact's path-penalty row, and (Eq. (12) model) its first cross row
    const int y = B.contact >= 0 ? 6 * nb + (M.aux ? 4 * M.nc : 0) + B.contact : -1;
    const int c0 = cross ? 6 * nb + 4 * B.contact : -1;
    const int arow[22] = {px, px, py, py, th, th, vx, vy, om, om, y, y, y, y, y,
                          c0, c0 + 1, c0 + 2, c0 + 3, c0 + 1, c0 + 1, c0 + 1};
    const int acol[22] = {px, vx, py, vy, th, om, vx, vy, th, om, py, th, vy, om, y,
                          c0, c0 + 1, c0 + 2, c0 + 3, vx, th, om};
    const int na = A_PER_LINK + (y >= 0 ? A_PER_FOOT : 0) + (cross ? A_PER_CROSS : 0);
    for (int j = 0; j < na; ++j) {
      if (ar) ar[B.a_off + j] = arow[j];
      if (ac) ac[B.a_off + j] = acol[j];
    }
    int o = B.b_off;
    auto put = [&](int r, int q) {
      if (br) br[o] = r;
      if (bc) bc[o] = q;
      ++o;
    };
    for (int i = 0; i < B.nin; ++i) {
      const bool nx = B.ax[i] != 0.0, ny = B.ay[i] != 0.0, tq = input_torque(B, i);
      if (nx) put(px, B.idx[i]);
      if (ny) put(py, B.idx[i]);
      if (tq) put(th, B.idx[i]);
      if (nx) put(vx, B.idx[i]);
      if (ny) put(vy, B.idx[i]);
      if (tq) put(om, B.idx[i]);
      if (y >= 0) put(y, B.idx[i]);
    }
    if (cross) {
      for (int i = 0; i < B.nin; ++i)
        if (input_lambda(B, i)) put(c0 + 1, B.idx[i]);
      put(c0, B.cin + 1);
      put(c0 + 2, B.cin + 2);
      put(c0 + 3, B.cin);
      put(c0 + 3, B.cin + 1);
    }
  }
}

bool layout_ok(int layout) { return layout == CISCVX_FOH_NODE || layout == CISCVX_FOH_INTERVAL; }

ciscvx_status check_common(const ciscvx_model* m, int N, int n_sub, int precision, int layout,
                           const double* X, const double* U, const double* s) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  if (N < 1) return fail(CISCVX_EINVAL, "N must be >= 1 (got %d)", N);
  if (n_sub < 1) return fail(CISCVX_EINVAL, "n_sub must be >= 1 (got %d)", n_sub);
  if (!layout_ok(layout)) return fail(CISCVX_EINVAL, "unknown control layout %d", layout);
  if (precision == CISCVX_TF32_TC || precision == CISCVX_BF16_TC)
    return fail(CISCVX_EUNSUPPORTED, "tensor-core precisions are not provided by this library");
  if (precision != CISCVX_FP64 && precision != CISCVX_FP32_PHI)
    return fail(CISCVX_EINVAL, "unknown precision %d", precision);
  if (!X || !s || (m->host.nu > 0 && !U)) return fail(CISCVX_EINVAL, "null input array");
  return CISCVX_OK;
}

ciscvx_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CISCVX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

// The compact pattern for the other translation units (SOCP canonicalization).
void ciscvx::model_pattern(const DevModel& M, int32_t* ar, int32_t* ac, int32_t* br, int32_t* bc) {
  fill_pattern(M, ar, ac, br, bc);
}

// Sets this thread's last-error message for entry points defined in other files.
ciscvx_status ciscvx::set_error(ciscvx_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

extern "C" {

int ciscvx_version(void) { return CISCVX_VERSION_MAJOR * 1000 + CISCVX_VERSION_MINOR; }

const char* ciscvx_last_error(void) { return g_err.c_str(); }

ciscvx_status ciscvx_model_create(const ciscvx_model_desc* desc, ciscvx_model** out) {
  if (!desc || !out) return fail(CISCVX_EINVAL, "null argument");
  *out = nullptr;
  ciscvx_status st = check_desc(desc);
  if (st != CISCVX_OK) return st;
  ciscvx_model* m = new (std::nothrow) ciscvx_model;
  if (!m) return fail(CISCVX_ENOMEM, "host allocation failed");
  st = build_tables(desc, m->host);
  if (st != CISCVX_OK) { delete m; return st; }
  m->cpl = nullptr;
  if (cpl_needed(m->host)) {
    m->cpl = new (std::nothrow) CplTab;
    if (!m->cpl) { delete m; return fail(CISCVX_ENOMEM, "host allocation failed"); }
    const char* why = cpl_build(m->host, *m->cpl);
    if (why) {
      delete m->cpl;
      delete m;
      return fail(CISCVX_EUNSUPPORTED, "%s", why);
    }
  }
  m->dev = nullptr;
  m->status = nullptr;
  m->zpat = nullptr;
  cudaGetDevice(&m->device);
  cudaError_t e = cudaMalloc(&m->dev, sizeof(DevModel));
  if (e == cudaSuccess) e = cudaMalloc(&m->status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(m->dev, &m->host, sizeof(DevModel), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(unsigned));
  if (e == cudaSuccess && (m->host.aux || m->cpl)) {
    // the compact pattern by rows, for z with compact outputs
    const DevModel& M = m->host;
    std::vector<int32_t> ar(M.nnzA), ac(M.nnzA), br(M.nnzB), bc(M.nnzB);
    fill_pattern(M, ar.data(), ac.data(), br.data(), bc.data());
    std::vector<int32_t> zp;
    auto by_rows = [&](const std::vector<int32_t>& rr, const std::vector<int32_t>& cc) {
      std::vector<int32_t> off(M.nxt + 1, 0);
      for (int32_t r : rr) ++off[r + 1];
      for (int r = 0; r < M.nxt; ++r) off[r + 1] += off[r];
      std::vector<int32_t> ent(2 * rr.size());
      std::vector<int32_t> pos(off.begin(), off.end() - 1);
      for (size_t j = 0; j < rr.size(); ++j) {
        const int32_t at = pos[rr[j]]++;
        ent[2 * at] = (int32_t)j;
        ent[2 * at + 1] = cc[j];
      }
      zp.insert(zp.end(), off.begin(), off.end());
      zp.insert(zp.end(), ent.begin(), ent.end());
    };
    by_rows(ar, ac);
    by_rows(br, bc);
    e = cudaMalloc(&m->zpat, zp.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(m->zpat, zp.data(), zp.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    if (m->dev) cudaFree(m->dev);
    if (m->status) cudaFree(m->status);
    if (m->zpat) cudaFree(m->zpat);
    delete m->cpl;
    delete m;
    return e == cudaErrorMemoryAllocation ? fail(CISCVX_ENOMEM, "device allocation failed")
                                          : cuda_fail(e, "model upload");
  }
  *out = m;
  return ok();
}

void ciscvx_model_destroy(ciscvx_model* m) {
  if (!m) return;
  if (m->zpat) cudaFree(m->zpat);
  if (m->dev) cudaFree(m->dev);
  if (m->status) cudaFree(m->status);
  delete m->cpl;
  delete m;
}

ciscvx_status ciscvx_model_pattern(const ciscvx_model_desc* desc, int* nnz_a, int* nnz_b,
                                   int32_t* a_row, int32_t* a_col, int32_t* b_row,
                                   int32_t* b_col) {
  if (!desc) return fail(CISCVX_EINVAL, "null description");
  ciscvx_status st = check_desc(desc);
  if (st != CISCVX_OK) return st;
  DevModel* M = new (std::nothrow) DevModel;
  if (!M) return fail(CISCVX_ENOMEM, "host allocation failed");
  st = build_tables(desc, *M);
  if (st == CISCVX_OK) {
    if (nnz_a) *nnz_a = M->nnzA;
    if (nnz_b) *nnz_b = M->nnzB;
    fill_pattern(*M, a_row, a_col, b_row, b_col);
  }
  delete M;
  return st == CISCVX_OK ? ok() : st;
}

ciscvx_status ciscvx_model_nnz(const ciscvx_model* m, int* nnz_a, int* nnz_b) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  if (nnz_a) *nnz_a = m->host.nnzA;
  if (nnz_b) *nnz_b = m->host.nnzB;
  return ok();
}

ciscvx_status ciscvx_model_dims(const ciscvx_model* m, int* n_x, int* n_y, int* n_u) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  if (n_x) *n_x = 6 * m->host.nb;
  if (n_y) *n_y = m->host.ny;
  if (n_u) *n_u = m->host.nu;
  return ok();
}

ciscvx_status ciscvx_workspace_size(const ciscvx_model* m, ciscvx_op op, int N,
                                    ciscvx_u_layout layout, size_t* bytes) {
  if (!m || !bytes) return fail(CISCVX_EINVAL, "null argument");
  if (N < 1) return fail(CISCVX_EINVAL, "N must be >= 1");
  if (!layout_ok(layout)) return fail(CISCVX_EINVAL, "unknown control layout %d", (int)layout);
  if (op == CISCVX_OP_DISCRETIZE) {
    if (m->cpl)
      return fail(CISCVX_EUNSUPPORTED, "the scratch of a model with coupled links depends on n_sub and "
                                       "the precision: use ciscvx_discretize_workspace_size");
    *bytes = 0;
  }
  else if (op == CISCVX_OP_VJP) {
    if (m->cpl)
      return fail(CISCVX_EUNSUPPORTED, "the scratch of the coupled-path adjoint depends on n_sub and "
                                       "the precision: use ciscvx_discretize_workspace_size");
    *bytes = vjp_workspace_bytes(m->host.nb, m->host.nu, m->host.nslot, N, layout);
  }
  else return fail(CISCVX_EINVAL, "unknown op %d", (int)op);
  return ok();
}

ciscvx_status ciscvx_discretize_workspace_size(const ciscvx_model* m, ciscvx_op op, int N,
                                               int n_sub, ciscvx_precision precision,
                                               ciscvx_u_layout layout, size_t* min_bytes,
                                               size_t* full_bytes) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  if (N < 1 || n_sub < 1) return fail(CISCVX_EINVAL, "need N >= 1 and n_sub >= 1");
  if (precision != CISCVX_FP64 && precision != CISCVX_FP32_PHI && precision != CISCVX_TF32_TC &&
      precision != CISCVX_BF16_TC)
    return fail(CISCVX_EINVAL, "unknown precision %d", (int)precision);
  if (!layout_ok(layout)) return fail(CISCVX_EINVAL, "unknown control layout %d", (int)layout);
  if (op != CISCVX_OP_DISCRETIZE && op != CISCVX_OP_VJP) return fail(CISCVX_EINVAL, "unknown op %d", (int)op);
  size_t lo = 0, hi = 0;
  if (op == CISCVX_OP_DISCRETIZE) {
    if (m->cpl) {
      const size_t per = cpl_interval_bytes(*m->cpl, n_sub, precision);
      lo = per * (size_t)std::min(N, 32);
      hi = per * (size_t)N;
    }
  } else if (m->cpl) {  // reverse-mode adjoint of the coupled path
    lo = cpl_adjoint_bytes(*m->cpl, std::min(N, 32), n_sub, precision);
    hi = cpl_adjoint_bytes(*m->cpl, N, n_sub, precision);
  } else {
    lo = hi = vjp_workspace_bytes(m->host.nb, m->host.nu, m->host.nslot, N, layout);
  }
  if (min_bytes) *min_bytes = lo;
  if (full_bytes) *full_bytes = hi;
  return ok();
}

ciscvx_status ciscvx_discretize(const ciscvx_model* m, int N, int n_sub,
                                ciscvx_precision precision, ciscvx_u_layout layout,
                                const double* X, const double* U, const double* s, void* A,
                                void* Bm, void* Bp, void* S, double* defect, double* penalty,
                                double* z, void* workspace, size_t ws_bytes, void* stream) {
  ciscvx_status st = check_common(m, N, n_sub, precision, layout, X, U, s);
  if (st != CISCVX_OK) return st;
  if (!A || !S || !defect) return fail(CISCVX_EINVAL, "null output array");
  if (m->host.nu > 0 && (!Bm || !Bp)) return fail(CISCVX_EINVAL, "null B- / B+");
  if (m->host.nc > 0 && !penalty) return fail(CISCVX_EINVAL, "null penalty");
  if (m->cpl) {
    const size_t per = cpl_interval_bytes(*m->cpl, n_sub, precision);
    const size_t need = per * (size_t)std::min(N, 32);
    if (!workspace || ws_bytes < need)
      return fail(CISCVX_EINVAL, "workspace of at least %zu bytes needed (got %zu)", need, ws_bytes);
    if (((uintptr_t)workspace & 15) != 0) return fail(CISCVX_EINVAL, "workspace must be 16-byte aligned");
    const long chunk = (long)std::min<size_t>(ws_bytes / per, (size_t)N);
    cudaError_t e = launch_coupled(*m->cpl, N, n_sub, precision, layout, X, U, s, A, Bm, Bp, S,
                                   defect, penalty, workspace, chunk, m->status, (cudaStream_t)stream);
    if (e == cudaSuccess && z)
      e = launch_affine_z(m->host, N, precision, layout, X, U, s, A, Bm, Bp, S, defect, z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "coupled discretize launch");
    return ok();
  }
  // the Eq. (12) model's kernels do not form z; it comes from the outputs
  const bool post_z = m->host.aux && z;
  cudaError_t e = launch_discretize(m->dev, m->host.nb, N, n_sub, precision, layout, false, m->host.aux != 0, X, U,
                                    s, A, Bm, Bp, S, defect, penalty, post_z ? nullptr : z, m->status,
                                    (cudaStream_t)stream);
  if (e == cudaSuccess && post_z)
    e = launch_affine_z(m->host, N, precision, layout, X, U, s, A, Bm, Bp, S, defect, z, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "discretize launch");
  return ok();
}

ciscvx_status ciscvx_discretize_compact(const ciscvx_model* m, int N, int n_sub,
                                        ciscvx_precision precision, ciscvx_u_layout layout,
                                        const double* X, const double* U, const double* s,
                                        void* A, void* Bm, void* Bp, void* S, double* defect,
                                        double* penalty, double* z, void* workspace, size_t ws_bytes,
                                        void* stream) {
  ciscvx_status st = check_common(m, N, n_sub, precision, layout, X, U, s);
  if (st != CISCVX_OK) return st;
  if (!A || !S || !defect) return fail(CISCVX_EINVAL, "null output array");
  if (m->host.nnzB > 0 && (!Bm || !Bp)) return fail(CISCVX_EINVAL, "null B- / B+");
  if (m->host.nc > 0 && !penalty) return fail(CISCVX_EINVAL, "null penalty");
  if (m->cpl) {  // the coupled path writing the column-major compact layout
    const size_t per = cpl_interval_bytes(*m->cpl, n_sub, precision);
    const size_t need = per * (size_t)std::min(N, 32);
    if (!workspace || ws_bytes < need)
      return fail(CISCVX_EINVAL, "workspace of at least %zu bytes needed (got %zu)", need, ws_bytes);
    if (((uintptr_t)workspace & 15) != 0) return fail(CISCVX_EINVAL, "workspace must be 16-byte aligned");
    const long chunk = (long)std::min<size_t>(ws_bytes / per, (size_t)N);
    cudaError_t e = launch_coupled(*m->cpl, N, n_sub, precision, layout, X, U, s, A, Bm, Bp, S, defect,
                                   penalty, workspace, chunk, m->status, (cudaStream_t)stream, nullptr,
                                   nullptr, true);
    if (e == cudaSuccess && z)
      e = launch_affine_z_compact(m->host, N, precision, layout, X, U, s, A, Bm, Bp, S, defect, m->zpat, z,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "coupled discretize launch");
    return ok();
  }
  // the Eq. (12) model's kernels do not form z: a post-pass over the compact
  // outputs and the pattern by rows does
  const bool post_z = m->host.aux && z;
  cudaError_t e = launch_discretize(m->dev, m->host.nb, N, n_sub, precision, layout, true, m->host.aux != 0, X,
                                    U, s, A, Bm, Bp, S, defect, penalty, post_z ? nullptr : z, m->status,
                                    (cudaStream_t)stream);
  if (e == cudaSuccess && post_z)
    e = launch_affine_z_compact(m->host, N, precision, layout, X, U, s, A, Bm, Bp, S, defect, m->zpat, z,
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "discretize launch");
  return ok();
}

ciscvx_status ciscvx_discretize_vjp(const ciscvx_model* m, int N, int n_sub,
                                    ciscvx_precision precision, ciscvx_u_layout layout,
                                    const double* X, const double* U, const double* s,
                                    const double* w, const double* rho, double* gX, double* gU,
                                    double* gs, double* L, void* workspace, size_t ws_bytes,
                                    void* stream) {
  ciscvx_status st = check_common(m, N, n_sub, precision, layout, X, U, s);
  if (st != CISCVX_OK) return st;
  if (!w || (m->host.nc > 0 && !rho)) return fail(CISCVX_EINVAL, "null cotangent array");
  if (!gX || !gs || (m->host.nu > 0 && !gU)) return fail(CISCVX_EINVAL, "null gradient array");
  if (m->cpl) {  // reverse-mode adjoint of the coupled path
    const size_t need = cpl_adjoint_bytes(*m->cpl, std::min(N, 32), n_sub, precision);
    if (!workspace || ws_bytes < need)
      return fail(CISCVX_EINVAL, "workspace of at least %zu bytes needed (got %zu)", need, ws_bytes);
    if (((uintptr_t)workspace & 15) != 0) return fail(CISCVX_EINVAL, "workspace must be 16-byte aligned");
    cudaError_t e = launch_coupled_vjp(*m->cpl, N, n_sub, precision, layout, X, U, s, w, rho, gX, gU, gs, L,
                                       workspace, ws_bytes, m->status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "coupled adjoint launch");
    return ok();
  }
  if (n_sub > MAXSUB_VJP)
    return fail(CISCVX_EUNSUPPORTED, "VJP supports at most %d substeps (got %d)", MAXSUB_VJP, n_sub);
  const size_t need = vjp_workspace_bytes(m->host.nb, m->host.nu, m->host.nslot, N, layout);
  if (!workspace || ws_bytes < need)
    return fail(CISCVX_EINVAL, "workspace of %zu bytes needed (got %zu)", need, ws_bytes);
  if (((uintptr_t)workspace & 15) != 0) return fail(CISCVX_EINVAL, "workspace must be 16-byte aligned");
  cudaError_t e = launch_vjp(m->dev, m->host.nb, m->host.nxt, m->host.nu, m->host.nslot, N, n_sub,
                             precision, layout, X, U, s, w, rho, gX, gU, gs, L, workspace,
                             m->status, m->host.aux != 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vjp launch");
  return ok();
}

ciscvx_status ciscvx_node_linearize(const ciscvx_model* m, int n, const double* Xp,
                                    const double* Xm, const double* Phi, const double* Gam,
                                    const ciscvx_node_params* params, double* g, double* Gvm,
                                    double* Gth, double* Gphi, double* Gpx, double* theta,
                                    double* dtheta, void* stream) {
  if (!m || !params) return fail(CISCVX_EINVAL, "null model or params");
  if (n < 1) return fail(CISCVX_EINVAL, "n_nodes must be >= 1 (got %d)", n);
  const DevModel& M = m->host;
  if (!M.tree)
    return fail(CISCVX_EUNSUPPORTED, "node constraints need every link to be the child of at most one joint");
  if (M.nj > NODE_MAXJ)
    return fail(CISCVX_EUNSUPPORTED, "node constraints support at most %d joints", NODE_MAXJ);
  for (int b = 0; b < M.nb; ++b)
    if (M.nadj[b] > NODE_MAXADJ)
      return fail(CISCVX_EUNSUPPORTED, "node constraints support at most %d joints on one link", NODE_MAXADJ);
  if (!(std::isfinite(params->delta) && params->delta > 0.0))
    return fail(CISCVX_EINVAL, "delta must be finite and > 0");
  if (!Xp || !Xm || !g) return fail(CISCVX_EINVAL, "null state or residual array");
  if (M.nc > 0 && (!Phi || !Gam || !theta || !params->restitution))
    return fail(CISCVX_EINVAL, "null impulse, multiplier, theta or restitution array");
  NodeParams P;
  std::memset(&P, 0, sizeof P);
  P.delta = params->delta;
  for (int i = 0; i < M.nc; ++i) {
    const double e = params->restitution[i];
    if (!(std::isfinite(e) && e >= 0.0)) return fail(CISCVX_EINVAL, "restitution %d must be finite and >= 0", i);
    P.e[i] = e;
  }
  if (node_smem_per_warp(M) > 220u * 1024u)
    return fail(CISCVX_EUNSUPPORTED, "model too large for the node kernel's shared memory");
  cudaError_t e = launch_node(M, m->dev, n, Xp, Xm, Phi, Gam, P, g, Gvm, Gth, Gphi, Gpx, theta,
                              dtheta, m->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "node launch");
  return ok();
}

ciscvx_status ciscvx_psi_rows(const ciscvx_model* m, int* n_psi) {
  if (!m || !n_psi) return fail(CISCVX_EINVAL, "null model or output");
  *n_psi = psi_rows(m->host);
  return ok();
}

ciscvx_status ciscvx_psi_linearize(const ciscvx_model* m, int N, const double* Xp, const double* Xm,
                                   double delta, double epsilon, double* psi, double* dpsi,
                                   void* stream) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  if (N < 1) return fail(CISCVX_EINVAL, "N must be >= 1 (got %d)", N);
  if (!(std::isfinite(delta) && delta > 0.0)) return fail(CISCVX_EINVAL, "delta must be finite and > 0");
  if (!(std::isfinite(epsilon) && epsilon >= 0.0))
    return fail(CISCVX_EINVAL, "epsilon must be finite and >= 0");
  const DevModel& M = m->host;
  if (psi_rows(M) == 0) return ok();
  if (!Xp || !Xm || !psi) return fail(CISCVX_EINVAL, "null state or psi array");
  cudaError_t e = launch_psi(M, N, Xp, Xm, delta, epsilon, psi, dpsi, m->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "psi launch");
  return ok();
}

ciscvx_status ciscvx_sync_status(const ciscvx_model* m, void* stream) {
  if (!m) return fail(CISCVX_EINVAL, "null model");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, m->status, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (h & ST_NONFINITE) return fail(CISCVX_ENONFINITE, "non-finite state or block produced");
  return ok();
}

}  // extern "C"
