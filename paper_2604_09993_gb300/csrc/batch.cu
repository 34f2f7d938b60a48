// batch.cu — batched heterogeneous discretization and VJP (many independent
// instances: different robots, horizons N and substep counts) in one launch.
//
// Work decomposition (built on the host when the plan is created):
//  * bucket = (model, n_sub); every interval of every instance in the bucket
//    is an entry (instance, k);
//  * group = 32 consecutive entries of one bucket (may span instances), so a
//    warp's 32 lanes run the same link program with the same trip counts;
//  * item = group x link; items are ordered by estimated cost (n_sub, doubled
//    for foot links), largest first, and a persistent grid pulls them from a
//    device counter (no waits: each warp takes the next index with one
//    atomicAdd and stops when the list is exhausted).
// The launch sequence (counter reset + kernel) is captured into a CUDA graph
// once per set of buffers and replayed.  An autotuner times launch shapes.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_common.cuh"
#include "coupled.cuh"

namespace ciscvx {

// CMP: compact A/Bm/Bp (structural nonzeros only; strides nnzA / nnzB).
// AUX: some model of the batch uses the Eq. (12) auxiliary state (its foot
// links take the CROSS path); a separate instantiation keeps that path's
// registers out of the common kernels.
template <typename TP, int OCC, bool CMP, bool AUX = false>
__global__ void __launch_bounds__(Occ<OCC>::T, Occ<OCC>::B) k_batch_disc(BatchCommon c, const double* __restrict__ X,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ s, TP* A, TP* Bm,
                                                    TP* Bp, TP* S, double* defect,
                                                    double* penalty) {
  int iter = 0;
  for (;;) {
    const int item = next_item(c, iter);
    if (item >= c.n_items) break;
    disc_item<TP, CMP, AUX>(c, item, X, U, s, A, Bm, Bp, S, defect, penalty);
  }
}

template <typename TP, int OCC, bool AUX = false>
__global__ void __launch_bounds__(Occ<OCC>::T, Occ<OCC>::B) k_batch_vjp(BatchCommon c, const double* __restrict__ X,
                                                   const double* __restrict__ U,
                                                   const double* __restrict__ s,
                                                   const double* __restrict__ w,
                                                   const double* __restrict__ rho, double* gX,
                                                   double* part, double* ps, double* pL) {
  int iter = 0;
  for (;;) {
    const int item = next_item(c, iter);
    if (item >= c.n_items) break;
    vjp_item<TP, AUX>(c, item, X, U, s, w, rho, gX, part, ps, pL);
  }
}

constexpr int FINB = 256;

// One CTA per instance: dL/dU (node layout sums the u_L part of interval k and
// the u_R part of interval k-1), dL/ds and L, all in a fixed summation order.
__global__ void __launch_bounds__(FINB) k_batch_vjp_finish(const DevModel* const* models,
                                                           const DevInst* inst, int layout,
                                                           const double* __restrict__ part,
                                                           const double* __restrict__ ps,
                                                           const double* __restrict__ pL,
                                                           double* gU, double* gs, double* L) {
  __shared__ double red[FINB];
  const DevInst I = inst[blockIdx.x];
  if (I.contract) return;  // written by the coupled path's adjoint
  const DevModel& M = *models[I.model];
  const int nu = M.nu, nslot = M.nslot, nb = M.nb, N = I.N;
  const double* P = part + I.part;
  const long nrow = (layout == CISCVX_FOH_NODE) ? (long)N + 1 : 2L * N;
  for (long idx = threadIdx.x; idx < nrow * nu; idx += FINB) {
    const long r = idx / nu;
    const int q = (int)(idx - r * nu);
    const int n = M.in_n[q];
    double v = 0.0;
    if (layout == CISCVX_FOH_NODE) {
      if (r < N) for (int t = 0; t < n; ++t) v += P[(size_t)r * nslot * 2 + 2 * M.in_slot[q][t]];
      if (r > 0) for (int t = 0; t < n; ++t) v += P[(size_t)(r - 1) * nslot * 2 + 2 * M.in_slot[q][t] + 1];
    } else {
      const long k = r >> 1;
      const int side = (int)(r & 1);
      for (int t = 0; t < n; ++t) v += P[(size_t)k * nslot * 2 + 2 * M.in_slot[q][t] + side];
    }
    gU[I.u + idx] = v;
  }
  double Lacc = 0.0;
  for (int k = threadIdx.x; k < N; k += FINB) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) {
      v += ps[I.pb + (long)k * nb + b];
      Lacc += pL[I.pb + (long)k * nb + b];
    }
    gs[I.s + k] = v;
  }
  if (L) {
    red[threadIdx.x] = Lacc;
    __syncthreads();
    for (int o = FINB / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) L[blockIdx.x] = red[0];
  }
}

}  // namespace ciscvx

using namespace ciscvx;

// Work tables for the instances split into consecutive chunks (the pipelined
// host executor runs chunk by chunk; one chunk = the whole batch otherwise).
struct ChunkTables {
  int K = 0;                        // number of chunks these tables describe
  int2* d_entries = nullptr;
  int4* d_groups = nullptr;
  int2* d_items_lpt = nullptr;
  int2* d_items_nat = nullptr;
  int2* d_items_sm = nullptr;
  std::vector<int> item_off;        // [K+1] items of chunk c: [item_off[c], item_off[c+1])
  std::vector<int> entry_off;       // [K+1] per-link entries (intervals) of chunk c
  std::vector<int> foot_cnt;        // [K] foot-link items at the head of chunk c's items_sm
  int split_sm = 0;                 // SMs that take the foot-link queue first (lpt_order 2)
  std::vector<int> inst_off;        // [K+1] instances of chunk c
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> ev;      // 1 start + 3 per chunk
};

struct ciscvx_batch_plan {
  int n_inst = 0, n_models = 0, prec = 0, layout = 0, device = 0, sm_count = 0, max_nsub = 0;
  bool compact = false;  // CISCVX_OUT_COMPACT
  bool all_nu0 = true, all_nc0 = true;
  bool any_aux = false;  // some model uses the Eq. (12) auxiliary state (AUX kernel instantiations)
  bool any_cpl = false;  // some model has coupled links (coupled path, its own adjoint)
  // coupled-path groups: instances of one coupled model with one n_sub, as
  // (instance, k) entries; one stage-data workspace shared in stream order
  struct CplGroup {
    int model, nsub, first, count;
  };
  std::vector<CplGroup> cpl_groups;
  int2* d_cpl_entries = nullptr;
  void* d_cpl_ws = nullptr;
  size_t cpl_ws_bytes = 0;
  std::vector<const ciscvx_model*> models;
  std::vector<DevInst> inst;
  ciscvx_batch_sizes sizes{};
  size_t part_total = 0, pb_total = 0;
  int n_items = 0;
  std::vector<int2> items_lpt, items_nat;
  int max_nsub_adj = 0;        // largest n_sub among the per-link instances (the adjoint kernel's)
  size_t cpl_adj_ws = 0;       // bytes of VJP workspace the coupled adjoint needs (after the partial sums)
  std::string key;
  // device tables
  const DevModel** d_models = nullptr;
  DevInst* d_inst = nullptr;
  int2* d_entries = nullptr;
  int4* d_groups = nullptr;
  int2* d_items_lpt = nullptr;
  int2* d_items_nat = nullptr;
  int* d_queue = nullptr;  // [0..1]: discretize, [2..3]: vjp (two counters each: lpt_order 2 uses both)
  int2* d_items_sm = nullptr;  // lpt_order 2: foot-link items, then the others (bucket order)
  int n_foot_items = 0, split_sm = 0;
  int n_entries = 0;  // per-link intervals (entries) of the batch
  // dense outputs of the fused pass staged as compact values and widened by
  // k_expand_dense (expand.cu): per model, the compact index of every dense
  // entry of A and of B-/B+ (-1: structural zero); stage_vals = the largest
  // nnz_A + 2 nnz_B over the per-link models
  int* d_maps = nullptr;
  const int** d_map_a = nullptr;
  const int** d_map_b = nullptr;
  int stage_vals = 0;
  bool stage_ok = false;
  unsigned* d_status = nullptr;
  ciscvx_tune tune{4, 2, 1, 1, 0};
  ciscvx_tune tune_fused{4, 2, 1, 0, 0, 0};  // launch shape of the fused discretize+VJP pass
  ChunkTables chunks;  // tables of the last chunk count used by ciscvx_batch_run_host
  // graph cache
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  ciscvx_batch_io graph_io{};
  ciscvx_tune graph_tune{};
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, ciscvx_tune> g_tune_cache;

bool tune_ok(const ciscvx_tune& t) {
  return (t.warps_per_cta == 1 || t.warps_per_cta == 2 || t.warps_per_cta == 4 ||
          t.warps_per_cta == 8) &&
         t.ctas_per_sm >= 0 && t.ctas_per_sm <= 32 && t.occupancy >= 0 && t.occupancy <= 2 &&
         t.lpt_order >= 0 && t.lpt_order <= 2 &&
         (t.occupancy == 0 || t.warps_per_cta <= 4) && (t.split == 0 || (t.split == 1 && t.occupancy == 0));
}

void free_chunks(ChunkTables& t) {
  cudaFree(t.d_entries);
  cudaFree(t.d_groups);
  cudaFree(t.d_items_lpt);
  cudaFree(t.d_items_nat);
  cudaFree(t.d_items_sm);
  for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
  if (t.s_in) cudaStreamDestroy(t.s_in);
  if (t.s_comp) cudaStreamDestroy(t.s_comp);
  if (t.s_out) cudaStreamDestroy(t.s_out);
  t = ChunkTables();
}

void free_plan(ciscvx_batch_plan* p) {
  if (!p) return;
  free_chunks(p->chunks);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->d_models);
  cudaFree(p->d_inst);
  cudaFree(p->d_entries);
  cudaFree(p->d_groups);
  cudaFree(p->d_items_lpt);
  cudaFree(p->d_items_nat);
  cudaFree(p->d_items_sm);
  cudaFree(p->d_maps);
  cudaFree(p->d_map_a);
  cudaFree(p->d_map_b);
  cudaFree(p->d_queue);
  cudaFree(p->d_status);
  cudaFree(p->d_cpl_entries);
  cudaFree(p->d_cpl_ws);
  delete p;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  const size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)dst, n);
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Host work decomposition of instances [inst_off[c], inst_off[c+1]) for each
// chunk c: bucket (model, n_sub) -> entries (instance, k) -> groups of 32 ->
// items (group x link), items of each chunk contiguous, in cost order (lpt),
// in bucket order (nat), or as two queues (sm: the foot-link items in bucket
// order, then the others in bucket order; foot_cnt[c] of them are foot-link
// items).  Also returns the tuning key of the whole batch and the estimated
// cost of the foot-link and of all items.
struct HostDecomp {
  std::vector<int2> entries, items_lpt, items_nat, items_sm;
  std::vector<int4> groups;
  std::vector<int> item_off, foot_cnt, entry_off;
  double foot_cost = 0.0, all_cost = 0.0;
  std::string key;
};

std::string model_signature(const DevModel& M);

HostDecomp decompose(const ciscvx_batch_plan* p, const std::vector<int>& inst_off) {
  HostDecomp d;
  const int K = (int)inst_off.size() - 1;
  d.item_off.push_back(0);
  d.entry_off.push_back(0);
  for (int c = 0; c < K; ++c) {
    std::map<std::pair<int, int>, std::vector<int>> buckets;
    for (int i = inst_off[c]; i < inst_off[c + 1]; ++i)
      if (!p->models[p->inst[i].model]->cpl)  // coupled models take the coupled path
        buckets[{p->inst[i].model, p->inst[i].nsub}].push_back(i);
    std::vector<std::pair<long long, int2>> costed;
    for (auto& kv : buckets) {
      const int m = kv.first.first, ns = kv.first.second;
      const DevModel& M = p->models[m]->host;
      const int first = (int)d.entries.size();
      for (int i : kv.second)
        for (int k = 0; k < p->inst[i].N; ++k) d.entries.push_back(make_int2(i, k));
      const int cnt = (int)d.entries.size() - first;
      for (int g0 = 0; g0 < cnt; g0 += 32) {
        const int gi = (int)d.groups.size();
        d.groups.push_back(make_int4(m, ns, first + g0, std::min(32, cnt - g0)));
        for (int b = 0; b < M.nb; ++b)
          costed.push_back({(long long)ns * (M.body[b].contact >= 0 ? 2 : 1), make_int2(gi, b)});
      }
      if (K == 1) {
        int lg = 0;
        while ((1 << lg) < cnt) ++lg;
        d.key += model_signature(M) + "@" + std::to_string(ns) + "x2^" + std::to_string(lg) + ";";
      }
    }
    for (auto& x : costed) d.items_nat.push_back(x.second);
    int nfoot = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (auto& x : costed) {
        const int4 g = d.groups[x.second.x];
        const bool foot = p->models[g.x]->host.body[x.second.y].contact >= 0;
        if (foot != (pass == 0)) continue;
        d.items_sm.push_back(x.second);
        if (foot) { ++nfoot; d.foot_cost += (double)x.first; }
        d.all_cost += (double)x.first;
      }
    d.foot_cnt.push_back(nfoot);
    std::stable_sort(costed.begin(), costed.end(),
                     [](const std::pair<long long, int2>& a, const std::pair<long long, int2>& b) {
                       return a.first > b.first;
                     });
    for (auto& x : costed) d.items_lpt.push_back(x.second);
    d.item_off.push_back((int)d.items_lpt.size());
    d.entry_off.push_back((int)d.entries.size());
  }
  return d;
}

// SMs that take the foot-link queue first under lpt_order 2: their share of
// the estimated cost, at least one SM for each queue.
int split_sms(const ciscvx_batch_plan* p, const HostDecomp& d) {
  if (d.all_cost <= 0.0 || p->sm_count < 2) return 0;
  const int f = (int)std::lround(p->sm_count * d.foot_cost / d.all_cost);
  return std::min(std::max(f, 1), p->sm_count - 1);
}

BatchCommon common_of(const ciscvx_batch_plan* p, int queue_slot, const ciscvx_tune& t) {
  BatchCommon c;
  c.models = p->d_models;
  c.inst = p->d_inst;
  c.entries = p->d_entries;
  c.groups = p->d_groups;
  c.items = t.lpt_order == 2 ? p->d_items_sm : (t.lpt_order ? p->d_items_lpt : p->d_items_nat);
  c.n_items = p->n_items;
  c.persistent = t.ctas_per_sm > 0;
  c.two_q = (t.lpt_order == 2 && c.persistent) ? 1 : 0;
  c.n_first = p->n_foot_items;
  c.split_sm = p->split_sm;
  c.sm_count = p->sm_count;
  c.queue = p->d_queue + 2 * queue_slot;
  c.status = p->d_status;
  c.layout = p->layout;
  c.ck_smem = 0;
  c.stage_dense = 0;
  c.e0 = 0;
  c.e1 = p->n_entries;
  return c;
}

// BatchCommon for chunk c of the chunked tables.
BatchCommon common_chunk(const ciscvx_batch_plan* p, int queue_slot, int c, const ciscvx_tune& tu) {
  BatchCommon b = common_of(p, queue_slot, tu);
  const ChunkTables& t = p->chunks;
  b.entries = t.d_entries;
  b.groups = t.d_groups;
  b.items = (tu.lpt_order == 2 ? t.d_items_sm : (tu.lpt_order ? t.d_items_lpt : t.d_items_nat)) + t.item_off[c];
  b.n_items = t.item_off[c + 1] - t.item_off[c];
  b.n_first = t.foot_cnt[c];
  b.split_sm = t.split_sm;
  b.e0 = t.entry_off[c];
  b.e1 = t.entry_off[c + 1];
  return b;
}

void grid_for(const ciscvx_batch_plan* p, const ciscvx_tune& t, int n_items, unsigned& blocks,
              unsigned& threads) {
  threads = 32u * (unsigned)t.warps_per_cta;
  if (t.ctas_per_sm > 0) {
    blocks = (unsigned)(p->sm_count * t.ctas_per_sm);
  } else {
    blocks = (unsigned)((n_items + t.warps_per_cta - 1) / t.warps_per_cta);
  }
  if (blocks == 0) blocks = 1;
}

cudaError_t launch_disc_c(ciscvx_batch_plan* p, const BatchCommon& c, const ciscvx_batch_io* io,
                          cudaStream_t st) {
  if (c.persistent) {
    cudaError_t e = cudaMemsetAsync(c.queue, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  unsigned blocks, threads;
  grid_for(p, p->tune, c.n_items, blocks, threads);
#define CISCVX_DISC1(TP, OCC, CMP)                                                            \
  k_batch_disc<TP, OCC, CMP><<<blocks, threads, 0, st>>>(c, io->X, io->U, io->s, (TP*)io->A,   \
                                                         (TP*)io->Bm, (TP*)io->Bp, (TP*)io->S,  \
                                                         io->defect, io->penalty)
#define CISCVX_DISC(TP, OCC)                     \
  do {                                           \
    if (p->compact) CISCVX_DISC1(TP, OCC, true); \
    else CISCVX_DISC1(TP, OCC, false);           \
  } while (0)
  const int occ = p->tune.occupancy;
  if (p->any_aux) {  // Eq. (12) model in the batch: no register cap
#define CISCVX_DISC_AUX(TP, CMP)                                                             \
  k_batch_disc<TP, 0, CMP, true><<<blocks, threads, 0, st>>>(c, io->X, io->U, io->s, (TP*)io->A, \
                                                             (TP*)io->Bm, (TP*)io->Bp, (TP*)io->S, \
                                                             io->defect, io->penalty)
    if (p->prec == CISCVX_FP64) {
      if (p->compact) CISCVX_DISC_AUX(double, true); else CISCVX_DISC_AUX(double, false);
    } else {
      if (p->compact) CISCVX_DISC_AUX(float, true); else CISCVX_DISC_AUX(float, false);
    }
#undef CISCVX_DISC_AUX
    return cudaGetLastError();
  }
  if (p->prec == CISCVX_FP64) {
    if (occ == 1) CISCVX_DISC(double, 1);
    else if (occ == 2) CISCVX_DISC(double, 2);
    else CISCVX_DISC(double, 0);
  } else {
    if (occ == 1) CISCVX_DISC(float, 1);
    else if (occ == 2) CISCVX_DISC(float, 2);
    else CISCVX_DISC(float, 0);
  }
#undef CISCVX_DISC
#undef CISCVX_DISC1
  return cudaGetLastError();
}

// Coupled-path groups of the plan (after the per-link items).
cudaError_t launch_cpl_groups(ciscvx_batch_plan* p, const ciscvx_batch_io* io, cudaStream_t st) {
  for (const auto& g : p->cpl_groups) {
    const CplTab& T = *p->models[g.model]->cpl;
    const size_t per = cpl_interval_bytes(T, g.nsub, p->prec);
    const long chunk = (long)std::min<size_t>((size_t)g.count, p->cpl_ws_bytes / per);
    cudaError_t e = launch_coupled(T, g.count, g.nsub, p->prec, p->layout, io->X, io->U, io->s, io->A,
                                   io->Bm, io->Bp, io->S, io->defect, io->penalty, p->d_cpl_ws, chunk,
                                   p->d_status, st, p->d_cpl_entries + g.first, p->d_inst, p->compact);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_disc(ciscvx_batch_plan* p, const ciscvx_batch_io* io, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (p->n_items > 0) e = launch_disc_c(p, common_of(p, 0, p->tune), io, st);
  if (e == cudaSuccess && !p->cpl_groups.empty()) e = launch_cpl_groups(p, io, st);
  return e;
}

// VJP kernel over the items of `c`, then the per-instance finish over
// instances [i0, i1) (their partials are complete once the kernel is done).
cudaError_t launch_vjp_c(ciscvx_batch_plan* p, const BatchCommon& c, const ciscvx_batch_vjp_io* io,
                         double* part, double* ps, double* pL, int i0, int i1, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (c.persistent) e = cudaMemsetAsync(c.queue, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  unsigned blocks, threads;
  grid_for(p, p->tune, c.n_items, blocks, threads);
#define CISCVX_VJP(TP, OCC)                                                                   \
  k_batch_vjp<TP, OCC><<<blocks, threads, 0, s>>>(c, io->X, io->U, io->s, io->w, io->rho, io->gX, \
                                                  part, ps, pL)
  const int occ = p->tune.occupancy;
  if (p->any_aux) {  // Eq. (12) model in the batch: no register cap
    if (p->prec == CISCVX_FP64)
      k_batch_vjp<double, 0, true><<<blocks, threads, 0, s>>>(c, io->X, io->U, io->s, io->w, io->rho,
                                                              io->gX, part, ps, pL);
    else
      k_batch_vjp<float, 0, true><<<blocks, threads, 0, s>>>(c, io->X, io->U, io->s, io->w, io->rho,
                                                             io->gX, part, ps, pL);
  } else if (p->prec == CISCVX_FP64) {
    if (occ == 1) CISCVX_VJP(double, 1);
    else if (occ == 2) CISCVX_VJP(double, 2);
    else CISCVX_VJP(double, 0);
  } else {
    if (occ == 1) CISCVX_VJP(float, 1);
    else if (occ == 2) CISCVX_VJP(float, 2);
    else CISCVX_VJP(float, 0);
  }
#undef CISCVX_VJP
  e = cudaGetLastError();
  if (e == cudaSuccess && i1 > i0)
    k_batch_vjp_finish<<<i1 - i0, FINB, 0, s>>>(p->d_models, p->d_inst + i0, p->layout, part, ps,
                                                pL, io->gU, io->gs, io->L ? io->L + i0 : nullptr);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// Offset of the coupled adjoint's part of the VJP workspace (after the
// per-link adjoint's partial sums, 16-byte aligned).
size_t cpl_ws_offset(const ciscvx_batch_plan* p) {
  return (sizeof(double) * (p->part_total + 2 * p->pb_total) + 15) & ~(size_t)15;
}

// The reverse-mode adjoint of the coupled path for the coupled-link
// instances, one after another in stream order, each in chunks of what fits
// in the workspace.
cudaError_t launch_coupled_vjps(ciscvx_batch_plan* p, const ciscvx_batch_vjp_io* io, void* ws,
                                size_t ws_bytes, cudaStream_t s) {
  for (int i = 0; i < p->n_inst; ++i) {
    const DevInst& I = p->inst[i];
    if (!I.contract) continue;
    const ciscvx_model* m = p->models[I.model];
    const bool nu = m->host.nu > 0, nc = m->host.nc > 0;
    cudaError_t e = launch_coupled_vjp(*m->cpl, I.N, I.nsub, p->prec, p->layout, io->X + I.x,
                                       nu ? io->U + I.u : nullptr, io->s + I.s, io->w + I.v,
                                       nc ? io->rho + I.p : nullptr, io->gX + I.x,
                                       nu ? io->gU + I.u : nullptr, io->gs + I.s, io->L ? io->L + i : nullptr,
                                       ws, ws_bytes, p->d_status, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The coupled instances of [i0, i1) one after another: linearized, and with
// `vjp` also their VJP from the same nominal pass (defined below).
cudaError_t run_coupled_range(ciscvx_batch_plan* p, const ciscvx_batch_io* io, const ciscvx_batch_vjp_io* vjp,
                              void* ws, size_t ws_bytes, int i0, int i1, cudaStream_t st);

// Discretize + VJP of the items of `c` in one pass, then the per-instance
// finish over instances [i0, i1).  vio's X, U, s are not used (io's are).
cudaError_t launch_fused_c(ciscvx_batch_plan* p, const BatchCommon& c, const ciscvx_batch_io* io,
                           const ciscvx_batch_vjp_io* vio, double* part, double* ps, double* pL,
                           int i0, int i1, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (c.persistent) e = cudaMemsetAsync(c.queue, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  unsigned blocks, threads;
  if (p->tune_fused.split) {  // linearization and adjoint of each item on two warps
    BatchCommon cs = c;
    cs.n_items = 2 * c.n_items;
    cs.two_q = 0;  // one counter over the doubled item list
    grid_for(p, p->tune_fused, cs.n_items, blocks, threads);
    e = launch_disc_vjp_split(cs, c.n_items, p->prec, p->compact, p->any_aux, blocks, threads, io->X, io->U,
                              io->s, io->A, io->Bm, io->Bp, io->S, io->defect, io->penalty, vio->w,
                              vio->rho, vio->gX, part, ps, pL, s);
    if (e == cudaSuccess && i1 > i0)
      k_batch_vjp_finish<<<i1 - i0, FINB, 0, s>>>(p->d_models, p->d_inst + i0, p->layout, part, ps,
                                                  pL, vio->gU, vio->gs, vio->L ? vio->L + i0 : nullptr);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
  }
  grid_for(p, p->tune_fused, c.n_items, blocks, threads);
  // FP32 pass: the checkpoints (4 FP32 anchors per substep and thread) in
  // shared memory when a block's fit in the default 48 KB
  BatchCommon cf = c;
  size_t smem = 0;
  const size_t ck_bytes = (size_t)threads * 4 * sizeof(float) * (size_t)p->max_nsub_adj;
  if (p->prec == CISCVX_FP32_PHI && p->max_nsub_adj > 0 && ck_bytes <= 48u * 1024u) {
    cf.ck_smem = 1;
    smem = ck_bytes;
  }
  // dense outputs: the kernel stages each interval's compact values at the
  // start of its dense blocks (one store per structural nonzero) and
  // k_expand_dense widens them with coalesced stores (expand.cu)
  const bool stage = !p->compact && p->stage_ok;
  cf.stage_dense = stage ? 1 : 0;
  e = launch_disc_vjp_fused(cf, p->prec, p->tune_fused.occupancy, p->compact || stage, p->any_aux, blocks, threads,
                            io->X, io->U, io->s, io->A, io->Bm, io->Bp, io->S, io->defect, io->penalty,
                            vio->w, vio->rho, vio->gX, part, ps, pL, smem, s);
  if (e == cudaSuccess && stage)
    e = launch_expand_dense(cf, p->prec, p->d_map_a, p->d_map_b, p->stage_vals, io->A, io->Bm, io->Bp, s);
  if (e == cudaSuccess && i1 > i0)
    k_batch_vjp_finish<<<i1 - i0, FINB, 0, s>>>(p->d_models, p->d_inst + i0, p->layout, part, ps,
                                                pL, vio->gU, vio->gs, vio->L ? vio->L + i0 : nullptr);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// Checks of a VJP io and workspace shared by the VJP entry points.
ciscvx_status check_vjp(const ciscvx_batch_plan* p, const ciscvx_batch_vjp_io* io, bool need_x,
                        const void* workspace, size_t ws_bytes) {
  if (!p || !io) return set_error(CISCVX_EINVAL, "null plan or io");
  if ((need_x && (!io->X || !io->s)) || !io->w || !io->gX || !io->gs)
    return set_error(CISCVX_EINVAL, "null required buffer in ciscvx_batch_vjp_io");
  if (!p->all_nu0 && ((need_x && !io->U) || !io->gU)) return set_error(CISCVX_EINVAL, "null U / gU");
  if (!p->all_nc0 && !io->rho) return set_error(CISCVX_EINVAL, "null rho");
  if (p->max_nsub_adj > MAXSUB_VJP)
    return set_error(CISCVX_EUNSUPPORTED, "VJP supports at most %d substeps (plan has %d)",
                     MAXSUB_VJP, p->max_nsub_adj);
  const size_t need = cpl_ws_offset(p) + p->cpl_adj_ws;
  if (!workspace || ws_bytes < need)
    return set_error(CISCVX_EINVAL, "workspace of %zu bytes needed (got %zu)", need, ws_bytes);
  if (((uintptr_t)workspace & 15) != 0) return set_error(CISCVX_EINVAL, "workspace must be 16-byte aligned");
  return CISCVX_OK;
}

bool same_io(const ciscvx_batch_io& a, const ciscvx_batch_io& b) {
  return std::memcmp(&a, &b, sizeof a) == 0;
}

bool same_tune(const ciscvx_tune& a, const ciscvx_tune& b) {
  return std::memcmp(&a, &b, sizeof a) == 0;
}

ciscvx_status check_io(const ciscvx_batch_plan* p, const ciscvx_batch_io* io) {
  if (!p || !io) return set_error(CISCVX_EINVAL, "null plan or io");
  if (!io->X || !io->s || !io->A || !io->S || !io->defect)
    return set_error(CISCVX_EINVAL, "null required buffer in ciscvx_batch_io");
  if (!p->all_nu0 && (!io->U || !io->Bm || !io->Bp))
    return set_error(CISCVX_EINVAL, "null U / Bm / Bp");
  if (!p->all_nc0 && !io->penalty) return set_error(CISCVX_EINVAL, "null penalty");
  return CISCVX_OK;
}

std::string model_signature(const DevModel& M) {
  std::string s = std::to_string(M.nb) + "." + std::to_string(M.nj) + "." + std::to_string(M.nc);
  for (int b = 0; b < M.nb; ++b)
    s += "/" + std::to_string(M.body[b].nin) + (M.body[b].contact >= 0 ? "f" : "");
  return s;
}

}  // namespace

extern "C" {

ciscvx_status ciscvx_batch_plan_create(const ciscvx_model* const* models, int n_models,
                                       const int* model_idx, const int* N, const int* n_sub,
                                       int n_inst, ciscvx_precision precision,
                                       ciscvx_u_layout layout, ciscvx_out_format format,
                                       const ciscvx_tune* tune, ciscvx_batch_plan** out) {
  if (!out) return set_error(CISCVX_EINVAL, "null out");
  *out = nullptr;
  if (!models || n_models < 1 || !model_idx || !N || !n_sub || n_inst < 1)
    return set_error(CISCVX_EINVAL, "need models, n_models >= 1, n_inst >= 1 and per-instance arrays");
  if (layout != CISCVX_FOH_NODE && layout != CISCVX_FOH_INTERVAL)
    return set_error(CISCVX_EINVAL, "unknown control layout %d", (int)layout);
  if (precision == CISCVX_TF32_TC || precision == CISCVX_BF16_TC)
    return set_error(CISCVX_EUNSUPPORTED, "tensor-core precisions are not provided by this library");
  if (precision != CISCVX_FP64 && precision != CISCVX_FP32_PHI)
    return set_error(CISCVX_EINVAL, "unknown precision %d", (int)precision);
  if (format != CISCVX_OUT_DENSE && format != CISCVX_OUT_COMPACT)
    return set_error(CISCVX_EINVAL, "unknown output format %d", (int)format);
  if (tune && !tune_ok(*tune)) return set_error(CISCVX_EINVAL, "invalid ciscvx_tune");
  for (int m = 0; m < n_models; ++m)
    if (!models[m]) return set_error(CISCVX_EINVAL, "null model %d", m);
  for (int i = 0; i < n_inst; ++i) {
    if (model_idx[i] < 0 || model_idx[i] >= n_models)
      return set_error(CISCVX_EINVAL, "instance %d: model index %d out of range", i, model_idx[i]);
    if (N[i] < 1 || n_sub[i] < 1)
      return set_error(CISCVX_EINVAL, "instance %d: N and n_sub must be >= 1", i);
  }
  ciscvx_batch_plan* p = new (std::nothrow) ciscvx_batch_plan;
  if (!p) return set_error(CISCVX_ENOMEM, "host allocation failed");
  p->n_inst = n_inst;
  p->n_models = n_models;
  p->prec = precision;
  p->layout = layout;
  p->compact = (format == CISCVX_OUT_COMPACT);
  p->models.assign(models, models + n_models);
  if (tune) {
    p->tune = *tune;
    p->tune_fused = *tune;
    p->tune_fused.use_graph = 0;
  }
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (p->sm_count < 1) p->sm_count = 1;

  // packed offsets, instance order
  p->inst.resize(n_inst);
  ciscvx_batch_sizes& z = p->sizes;
  std::memset(&z, 0, sizeof z);
  for (int i = 0; i < n_inst; ++i) {
    const DevModel& M = models[model_idx[i]]->host;
    DevInst& I = p->inst[i];
    I.model = model_idx[i];
    I.N = N[i];
    I.nsub = n_sub[i];
    I.x = (long long)z.X; I.u = (long long)z.U; I.s = (long long)z.s; I.a = (long long)z.A;
    I.b = (long long)z.B; I.v = (long long)z.S; I.p = (long long)z.penalty;
    I.part = (long long)p->part_total;
    I.pb = (long long)p->pb_total;
    const size_t n = (size_t)N[i], nxt = M.nxt, nu = M.nu, nc = M.nc;
    z.X += (n + 1) * nxt;
    z.U += (layout == CISCVX_FOH_NODE ? (n + 1) : 2 * n) * nu;
    z.s += n;
    z.A += n * (p->compact ? (size_t)M.nnzA : nxt * nxt);
    z.B += n * (p->compact ? (size_t)M.nnzB : nxt * nu);
    z.S += n * nxt;
    z.defect += n * nxt;
    z.penalty += n * nc;
    p->part_total += n * (size_t)M.nslot * 2;
    p->pb_total += n * (size_t)M.nb;
    p->max_nsub = std::max(p->max_nsub, n_sub[i]);
    if (nu) p->all_nu0 = false;
    if (nc) p->all_nc0 = false;
    if (M.aux && !models[model_idx[i]]->cpl) p->any_aux = true;
    if (models[model_idx[i]]->cpl) p->any_cpl = true;
    I.contract = models[model_idx[i]]->cpl ? 1 : 0;
    if (I.contract) {  // the coupled path's adjoint, chunked to at most 4096 intervals
      const CplTab* T = models[model_idx[i]]->cpl;
      p->cpl_adj_ws = std::max(p->cpl_adj_ws, cpl_adjoint_bytes(*T, std::min<long>(N[i], 4096), n_sub[i], precision));
    } else {
      p->max_nsub_adj = std::max(p->max_nsub_adj, n_sub[i]);
    }
  }
  z.L = (size_t)n_inst;

  // work decomposition of the whole batch (one chunk)
  HostDecomp dec = decompose(p, {0, n_inst});
  p->key = std::to_string(precision) + "|" + std::to_string(layout) + "|" +
           (p->compact ? "c|" : "d|") + dec.key;
  p->n_items = (int)dec.items_lpt.size();
  p->n_foot_items = dec.foot_cnt.empty() ? 0 : dec.foot_cnt[0];
  p->split_sm = split_sms(p, dec);
  p->items_lpt = dec.items_lpt;
  p->items_nat = dec.items_nat;
  p->n_entries = (int)dec.entries.size();
  const std::vector<int2>& entries = dec.entries;
  const std::vector<int4>& groups = dec.groups;

  // coupled-path groups: (model, n_sub) -> (instance, k) entries; the stage-data
  // workspace holds one chunk of the largest group
  std::vector<int2> cpl_entries;
  {
    std::map<std::pair<int, int>, std::vector<int>> buckets;
    for (int i = 0; i < n_inst; ++i)
      if (models[p->inst[i].model]->cpl) buckets[{p->inst[i].model, p->inst[i].nsub}].push_back(i);
    size_t ws = 0;
    for (auto& kv : buckets) {
      ciscvx_batch_plan::CplGroup g{kv.first.first, kv.first.second, (int)cpl_entries.size(), 0};
      for (int i : kv.second)
        for (int k = 0; k < p->inst[i].N; ++k) cpl_entries.push_back(make_int2(i, k));
      g.count = (int)cpl_entries.size() - g.first;
      const CplTab& T = *models[g.model]->cpl;
      ws = std::max(ws, cpl_interval_bytes(T, g.nsub, precision) * (size_t)std::min(g.count, 32768));
      p->cpl_groups.push_back(g);
      cudaError_t pe = cpl_prepare(T, precision);  // compile the specialized kernels before any capture
      if (pe != cudaSuccess) {
        free_plan(p);
        return set_error(CISCVX_ECUDA, "coupled kernels: %s", cudaGetErrorString(pe));
      }
    }
    p->cpl_ws_bytes = ws;
  }

  std::vector<const DevModel*> dm(n_models);
  for (int m = 0; m < n_models; ++m) dm[m] = models[m]->dev;
  cudaError_t e = upload(&p->d_models, dm);
  if (e == cudaSuccess && !cpl_entries.empty()) e = upload(&p->d_cpl_entries, cpl_entries);
  if (e == cudaSuccess && p->cpl_ws_bytes) e = cudaMalloc(&p->d_cpl_ws, p->cpl_ws_bytes);
  if (e == cudaSuccess) e = upload(&p->d_inst, p->inst);
  if (e == cudaSuccess) e = upload(&p->d_entries, entries);
  if (e == cudaSuccess) e = upload(&p->d_groups, groups);
  if (e == cudaSuccess) e = upload(&p->d_items_lpt, p->items_lpt);
  if (e == cudaSuccess) e = upload(&p->d_items_nat, p->items_nat);
  if (e == cudaSuccess) e = upload(&p->d_items_sm, dec.items_sm);
  if (e == cudaSuccess && !p->compact && p->n_entries > 0 && precision == CISCVX_FP32_PHI) {
    // dense FP32 outputs: the per-model maps that widen staged compact values
    // (the FP64 path keeps the in-kernel zeroing: its doubled expand traffic
    // measured slower, 352 against 342 ms on the 4096 x 400 x 20 sweep)
    std::vector<int> maps;
    std::vector<size_t> oa(n_models, 0), ob(n_models, 0);
    int vals = 0;
    for (int m = 0; m < n_models; ++m) {
      const DevModel& M = models[m]->host;
      if (models[m]->cpl) continue;
      std::vector<int32_t> ar(M.nnzA), ac(M.nnzA), br(M.nnzB), bc(M.nnzB);
      model_pattern(M, ar.data(), ac.data(), br.data(), bc.data());
      maps.resize((maps.size() + 3) / 4 * 4, -1);  // 16-byte aligned map starts
      oa[m] = maps.size();
      maps.resize(maps.size() + (size_t)M.nxt * M.nxt, -1);
      for (int j = 0; j < M.nnzA; ++j) maps[oa[m] + (size_t)ar[j] * M.nxt + ac[j]] = j;
      maps.resize((maps.size() + 3) / 4 * 4, -1);
      ob[m] = maps.size();
      maps.resize(maps.size() + (size_t)M.nxt * M.nu, -1);
      for (int j = 0; j < M.nnzB; ++j) maps[ob[m] + (size_t)br[j] * M.nu + bc[j]] = j;
      vals = std::max(vals, M.nnzA + 2 * M.nnzB);
    }
    const size_t el = precision == CISCVX_FP64 ? sizeof(double) : sizeof(float);
    if (vals > 0 && 4u * (size_t)vals * el <= 200u * 1024u) {
      e = upload(&p->d_maps, maps);
      std::vector<const int*> pa(n_models, nullptr), pb(n_models, nullptr);
      for (int m = 0; m < n_models && e == cudaSuccess; ++m)
        if (!models[m]->cpl) { pa[m] = p->d_maps + oa[m]; pb[m] = p->d_maps + ob[m]; }
      if (e == cudaSuccess) e = upload(&p->d_map_a, pa);
      if (e == cudaSuccess) e = upload(&p->d_map_b, pb);
      p->stage_vals = vals;
      p->stage_ok = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->d_queue, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_plan(p);
    return set_error(e == cudaErrorMemoryAllocation ? CISCVX_ENOMEM : CISCVX_ECUDA,
                     "plan upload: %s", cudaGetErrorString(e));
  }
  *out = p;
  return CISCVX_OK;
}

void ciscvx_batch_plan_destroy(ciscvx_batch_plan* plan) { free_plan(plan); }

ciscvx_status ciscvx_batch_sizes_get(const ciscvx_batch_plan* p, ciscvx_batch_sizes* out) {
  if (!p || !out) return set_error(CISCVX_EINVAL, "null argument");
  *out = p->sizes;
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_offsets(const ciscvx_batch_plan* p, int i, ciscvx_batch_sizes* out) {
  if (!p || !out) return set_error(CISCVX_EINVAL, "null argument");
  if (i < 0 || i >= p->n_inst) return set_error(CISCVX_EINVAL, "instance %d out of range", i);
  const DevInst& I = p->inst[i];
  out->X = (size_t)I.x; out->U = (size_t)I.u; out->s = (size_t)I.s; out->A = (size_t)I.a;
  out->B = (size_t)I.b; out->S = (size_t)I.v; out->defect = (size_t)I.v;
  out->penalty = (size_t)I.p; out->L = (size_t)i;
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_get_tune(const ciscvx_batch_plan* p, ciscvx_tune* out) {
  if (!p || !out) return set_error(CISCVX_EINVAL, "null argument");
  *out = p->tune;
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_discretize(ciscvx_batch_plan* p, const ciscvx_batch_io* io,
                                      void* stream) {
  ciscvx_status st = check_io(p, io);
  if (st != CISCVX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!p->tune.use_graph) {
    e = launch_disc(p, io, s);
    if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    return CISCVX_OK;
  }
  if (!p->exec || !same_io(p->graph_io, *io) || !same_tune(p->graph_tune, p->tune)) {
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = launch_disc(p, io, p->cap);
      e = cudaStreamEndCapture(p->cap, &g);
      if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->exec = nullptr;
      return set_error(CISCVX_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    p->graph_io = *io;
    p->graph_tune = p->tune;
  }
  e = cudaGraphLaunch(p->exec, s);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_vjp_workspace_size(const ciscvx_batch_plan* p, size_t* bytes) {
  if (!p || !bytes) return set_error(CISCVX_EINVAL, "null argument");
  *bytes = cpl_ws_offset(p) + p->cpl_adj_ws;
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_vjp_workspace_sizes(const ciscvx_batch_plan* p, size_t* min_bytes, size_t* full_bytes) {
  if (!p || !min_bytes || !full_bytes) return set_error(CISCVX_EINVAL, "null argument");
  *min_bytes = cpl_ws_offset(p) + p->cpl_adj_ws;
  *full_bytes = *min_bytes;
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_discretize_vjp(ciscvx_batch_plan* p, const ciscvx_batch_vjp_io* io,
                                          void* workspace, size_t ws_bytes, void* stream) {
  ciscvx_status st = check_vjp(p, io, true, workspace, ws_bytes);
  if (st != CISCVX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)workspace;
  double* ps = part + p->part_total;
  double* pL = ps + p->pb_total;
  cudaError_t e = launch_vjp_c(p, common_of(p, 1, p->tune), io, part, ps, pL, 0, p->n_inst, s);
  if (e == cudaSuccess && p->any_cpl)
    e = launch_coupled_vjps(p, io, (char*)workspace + cpl_ws_offset(p), ws_bytes - cpl_ws_offset(p), s);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "batch vjp launch: %s", cudaGetErrorString(e));
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_discretize_and_vjp(ciscvx_batch_plan* p, const ciscvx_batch_io* io,
                                              const ciscvx_batch_vjp_io* vjp, void* workspace,
                                              size_t ws_bytes, void* stream) {
  ciscvx_status st = check_io(p, io);
  if (st == CISCVX_OK) st = check_vjp(p, vjp, false, workspace, ws_bytes);
  if (st != CISCVX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)workspace;
  double* ps = part + p->part_total;
  double* pL = ps + p->pb_total;
  cudaError_t e = launch_fused_c(p, common_of(p, 0, p->tune_fused), io, vjp, part, ps, pL, 0, p->n_inst, s);
  // coupled instances: linearization and VJP from one nominal pass each, in
  // the coupled part of the workspace
  if (e == cudaSuccess && p->any_cpl)
    e = run_coupled_range(p, io, vjp, (char*)workspace + cpl_ws_offset(p), ws_bytes - cpl_ws_offset(p), 0,
                          p->n_inst, s);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "fused launch: %s", cudaGetErrorString(e));
  return CISCVX_OK;
}

}  // extern "C"

namespace {

const ciscvx_tune kTuneCandidates[] = {
    {4, 2, 1, 0, 0}, {8, 1, 1, 0, 0}, {2, 4, 1, 0, 0}, {1, 8, 1, 0, 0}, {4, 0, 1, 0, 0},
    {4, 2, 0, 0, 0}, {4, 3, 1, 0, 1}, {2, 6, 1, 0, 1}, {4, 4, 1, 0, 2}, {2, 8, 1, 0, 2},
    {4, 0, 1, 0, 1}, {4, 0, 1, 0, 2},
    // SM-partitioned foot-link / other-link queues (lpt_order 2)
    {4, 3, 2, 0, 1}, {4, 2, 2, 0, 0}, {4, 4, 2, 0, 2},
};
// Split-form candidates of the fused pass (small batches only).
const ciscvx_tune kSplitCandidates[] = {{1, 0, 1, 0, 0, 1}, {2, 0, 1, 0, 0, 1}, {4, 0, 1, 0, 0, 1}};

// The tuner's choices can persist across processes in a text file named by
// CISCVX_TUNE_CACHE: one line per key, "key<TAB>warps ctas lpt graph occupancy
// split" (lines without the split field read as split 0).
// It is read once, at the first autotune of the process; every new choice is
// appended.  Lines that do not parse into a valid tune are ignored.
bool g_tune_file_read = false;

const char* tune_file() {
  const char* f = std::getenv("CISCVX_TUNE_CACHE");
  return (f && f[0]) ? f : nullptr;
}

void read_tune_file() {  // g_tune_mu held
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = tune_file();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[4096];
  while (std::fgets(line, sizeof line, f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    *tab = '\0';
    ciscvx_tune t{};
    const int got = std::sscanf(tab + 1, "%d %d %d %d %d %d", &t.warps_per_cta, &t.ctas_per_sm, &t.lpt_order,
                                &t.use_graph, &t.occupancy, &t.split);
    if (got == 5) t.split = 0;  // a line written before the split form existed
    if ((got == 5 || got == 6) && tune_ok(t))
      g_tune_cache[line] = t;
  }
  std::fclose(f);
}

void append_tune_file(const std::string& key, const ciscvx_tune& t) {  // g_tune_mu held
  const char* path = tune_file();
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s\t%d %d %d %d %d %d\n", key.c_str(), t.warps_per_cta, t.ctas_per_sm, t.lpt_order,
               t.use_graph, t.occupancy, t.split);
  std::fclose(f);
}

// Times launch() under every candidate written into *slot (warm-up + 2 timed
// calls each; with_split adds the split-form candidates), keeps the fastest
// there, caches it under `key` (and in the CISCVX_TUNE_CACHE file, if set).
template <class Launch>
ciscvx_status autotune_slot(ciscvx_batch_plan* p, ciscvx_tune* slot, const std::string& tag,
                            cudaStream_t s, const Launch& launch, ciscvx_tune* chosen,
                            bool with_split = false) {
  const int keep_graph = slot->use_graph;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->device);
  const std::string key = std::string(prop.name) + "|" + p->key + tag;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    read_tune_file();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *slot = it->second;
      slot->use_graph = keep_graph;
      if (chosen) *chosen = *slot;
      return CISCVX_OK;
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error(CISCVX_ECUDA, "event creation failed");
  float best = 1e30f;
  ciscvx_tune bt = *slot;
  cudaError_t e = cudaSuccess;
  std::vector<ciscvx_tune> cands(std::begin(kTuneCandidates), std::end(kTuneCandidates));
  if (with_split) cands.insert(cands.end(), std::begin(kSplitCandidates), std::end(kSplitCandidates));
  for (const ciscvx_tune& c : cands) {
    *slot = c;
    e = launch();  // warm-up
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bt = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  bt.use_graph = keep_graph;
  *slot = bt;
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "autotune: %s", cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = bt;
    append_tune_file(key, bt);
  }
  if (chosen) *chosen = bt;
  return CISCVX_OK;
}

}  // namespace

extern "C" {

ciscvx_status ciscvx_batch_autotune(ciscvx_batch_plan* p, const ciscvx_batch_io* io, void* stream,
                                    ciscvx_tune* chosen) {
  ciscvx_status st = check_io(p, io);
  if (st != CISCVX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return autotune_slot(p, &p->tune, "", s, [&]() { return launch_disc(p, io, s); }, chosen);
}

ciscvx_status ciscvx_batch_autotune_fused(ciscvx_batch_plan* p, const ciscvx_batch_io* io,
                                          const ciscvx_batch_vjp_io* vjp, void* workspace,
                                          size_t ws_bytes, void* stream, ciscvx_tune* chosen) {
  ciscvx_status st = check_io(p, io);
  if (st == CISCVX_OK) st = check_vjp(p, vjp, false, workspace, ws_bytes);
  if (st != CISCVX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* part = (double*)workspace;
  double* ps = part + p->part_total;
  double* pL = ps + p->pb_total;
  // the split form only where the fused pass has at most one warp per scheduler
  const bool with_split = p->n_items <= 4 * p->sm_count;
  return autotune_slot(p, &p->tune_fused, "|fused", s, [&]() {
    return launch_fused_c(p, common_of(p, 0, p->tune_fused), io, vjp, part, ps, pL, 0, p->n_inst, s);
  }, chosen, with_split);
}

ciscvx_status ciscvx_batch_get_tune_fused(const ciscvx_batch_plan* p, ciscvx_tune* out) {
  if (!p || !out) return set_error(CISCVX_EINVAL, "null argument");
  *out = p->tune_fused;
  return CISCVX_OK;
}

}  // extern "C"

namespace {

// Element offsets of instance i in the packed buffers (i == n_inst: the totals).
ciscvx_batch_sizes offsets_of(const ciscvx_batch_plan* p, int i) {
  if (i >= p->n_inst) return p->sizes;
  const DevInst& I = p->inst[i];
  ciscvx_batch_sizes o;
  o.X = (size_t)I.x; o.U = (size_t)I.u; o.s = (size_t)I.s; o.A = (size_t)I.a; o.B = (size_t)I.b;
  o.S = (size_t)I.v; o.defect = (size_t)I.v; o.penalty = (size_t)I.p; o.L = (size_t)i;
  return o;
}

// Chunk tables for K chunks of consecutive instances with balanced estimated
// cost (N * n_sub * links), built once per K and kept in the plan.
cudaError_t ensure_chunks(ciscvx_batch_plan* p, int K) {
  ChunkTables& t = p->chunks;
  if (t.K == K) return cudaSuccess;
  free_chunks(t);
  std::vector<double> cum(p->n_inst + 1, 0.0);
  for (int i = 0; i < p->n_inst; ++i)
    cum[i + 1] = cum[i] + (double)p->inst[i].N * p->inst[i].nsub * p->models[p->inst[i].model]->host.nb;
  std::vector<int> off(K + 1, 0);
  off[K] = p->n_inst;
  for (int c = 1; c < K; ++c) {
    const double target = cum[p->n_inst] * c / K;
    int i = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
    off[c] = std::min(std::max(i, off[c - 1] + 1), p->n_inst - (K - c));
  }
  HostDecomp d = decompose(p, off);
  cudaError_t e = upload(&t.d_entries, d.entries);
  if (e == cudaSuccess) e = upload(&t.d_groups, d.groups);
  if (e == cudaSuccess) e = upload(&t.d_items_lpt, d.items_lpt);
  if (e == cudaSuccess) e = upload(&t.d_items_nat, d.items_nat);
  if (e == cudaSuccess) e = upload(&t.d_items_sm, d.items_sm);
  t.foot_cnt = d.foot_cnt;
  t.entry_off = d.entry_off;
  t.split_sm = split_sms(p, d);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t.s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t.s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t.s_out, cudaStreamNonBlocking);
  for (int k = 0; k < 1 + 3 * K && e == cudaSuccess; ++k) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) t.ev.push_back(ev);
  }
  if (e != cudaSuccess) { free_chunks(t); return e; }
  t.K = K;
  t.item_off = d.item_off;
  t.inst_off = off;
  return cudaSuccess;
}

// The coupled-link instances of [i0, i1) one after another (host executor):
// the linearization into the device outputs at each instance's offsets
// (stage data in the plan's coupled workspace) and, with `vjp`, the
// reverse-mode adjoint into the VJP outputs (its scratch in `ws`).
cudaError_t run_coupled_range(ciscvx_batch_plan* p, const ciscvx_batch_io* io, const ciscvx_batch_vjp_io* vjp,
                              void* ws, size_t ws_bytes, int i0, int i1, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int i = i0; i < i1 && e == cudaSuccess; ++i) {
    const DevInst& I = p->inst[i];
    const ciscvx_model* m = p->models[I.model];
    if (!m->cpl) continue;
    const CplTab& T = *m->cpl;
    const bool nu = T.nu > 0, nc = T.nc > 0;
    const size_t el = p->prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
    const long chunk = std::max<long>(1, (long)std::min<size_t>((size_t)I.N, p->cpl_ws_bytes /
                                                                 cpl_interval_bytes(T, I.nsub, p->prec)));
    char* A = (char*)io->A + I.a * el;
    char* Bm = nu ? (char*)io->Bm + I.b * el : nullptr;
    char* Bp = nu ? (char*)io->Bp + I.b * el : nullptr;
    char* S = (char*)io->S + I.v * el;
    if (vjp)  // the linearization and the VJP from one nominal pass per chunk
      e = launch_coupled_and_vjp(T, I.N, I.nsub, p->prec, p->layout, io->X + I.x, nu ? io->U + I.u : nullptr,
                                 io->s + I.s, A, Bm, Bp, S, io->defect + I.v, nc ? io->penalty + I.p : nullptr,
                                 vjp->w + I.v, nc ? vjp->rho + I.p : nullptr, vjp->gX + I.x,
                                 nu ? vjp->gU + I.u : nullptr, vjp->gs + I.s, vjp->L ? vjp->L + i : nullptr, ws,
                                 ws_bytes, p->d_status, st, p->compact);
    else
      e = launch_coupled(T, I.N, I.nsub, p->prec, p->layout, io->X + I.x, nu ? io->U + I.u : nullptr,
                         io->s + I.s, A, Bm, Bp, S, io->defect + I.v, nc ? io->penalty + I.p : nullptr,
                         p->d_cpl_ws, chunk, p->d_status, st, nullptr, nullptr, p->compact);
  }
  return e;
}

cudaError_t copy_range(void* dst, const void* src, size_t elem, size_t lo, size_t hi,
                       cudaMemcpyKind kind, cudaStream_t st) {
  if (hi <= lo || !dst || !src) return cudaSuccess;
  return cudaMemcpyAsync((char*)dst + lo * elem, (const char*)src + lo * elem, (hi - lo) * elem,
                         kind, st);
}

}  // namespace

extern "C" {

ciscvx_status ciscvx_batch_run_host(ciscvx_batch_plan* p, int n_chunks, const ciscvx_batch_io* host,
                                    const ciscvx_batch_io* dev, const ciscvx_batch_vjp_io* host_vjp,
                                    const ciscvx_batch_vjp_io* dev_vjp, void* workspace,
                                    size_t ws_bytes, void* stream) {
  ciscvx_status st = check_io(p, dev);
  if (st != CISCVX_OK) return st;
  if (!host || !host->X || !host->s || !host->A || !host->S || !host->defect)
    return set_error(CISCVX_EINVAL, "null required host buffer");
  if (!p->all_nu0 && (!host->U || !host->Bm || !host->Bp)) return set_error(CISCVX_EINVAL, "null host U / Bm / Bp");
  if (!p->all_nc0 && !host->penalty) return set_error(CISCVX_EINVAL, "null host penalty");
  if (n_chunks < 1 || n_chunks > p->n_inst)
    return set_error(CISCVX_EINVAL, "n_chunks must be in [1, %d]", p->n_inst);
  const bool vjp = host_vjp != nullptr;
  double *part = nullptr, *ps = nullptr, *pL = nullptr;
  if (vjp) {
    if (!dev_vjp || !host_vjp->w || !host_vjp->gX || !host_vjp->gs || !dev_vjp->w || !dev_vjp->gX ||
        !dev_vjp->gs)
      return set_error(CISCVX_EINVAL, "null VJP buffer");
    if (!p->all_nu0 && (!host_vjp->gU || !dev_vjp->gU)) return set_error(CISCVX_EINVAL, "null gU");
    if (!p->all_nc0 && (!host_vjp->rho || !dev_vjp->rho)) return set_error(CISCVX_EINVAL, "null rho");
    if (p->max_nsub > MAXSUB_VJP)
      return set_error(CISCVX_EUNSUPPORTED, "VJP supports at most %d substeps", MAXSUB_VJP);
    // the adjoint's partial sums; with coupled instances also their adjoint's scratch
    const size_t need = p->any_cpl ? cpl_ws_offset(p) + p->cpl_adj_ws
                                   : sizeof(double) * (p->part_total + 2 * p->pb_total);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 15) != 0)
      return set_error(CISCVX_EINVAL, "16-byte aligned workspace of %zu bytes needed", need);
    part = (double*)workspace;
    ps = part + p->part_total;
    pL = ps + p->pb_total;
  }
  cudaError_t e = ensure_chunks(p, n_chunks);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "chunk tables: %s", cudaGetErrorString(e));
  ChunkTables& t = p->chunks;
  cudaStream_t user = (cudaStream_t)stream;
  const size_t phi = (p->prec == CISCVX_FP64) ? sizeof(double) : sizeof(float);
  const size_t d8 = sizeof(double);
  // the device-side VJP io: inputs/outputs in the device buffers
  ciscvx_batch_vjp_io dv{};
  if (vjp) {
    dv = *dev_vjp;
    dv.X = dev->X; dv.U = dev->U; dv.s = dev->s;
  }
  e = cudaEventRecord(t.ev[0], user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(t.s_in, t.ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(t.s_comp, t.ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(t.s_out, t.ev[0], 0);
  for (int c = 0; c < n_chunks && e == cudaSuccess; ++c) {
    const int i0 = t.inst_off[c], i1 = t.inst_off[c + 1];
    const ciscvx_batch_sizes a = offsets_of(p, i0), b = offsets_of(p, i1);
    cudaEvent_t ev_in = t.ev[1 + 3 * c], ev_comp = t.ev[2 + 3 * c], ev_out = t.ev[3 + 3 * c];
    // host -> device: this chunk's inputs
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
    e = copy_range((void*)dev->X, host->X, d8, a.X, b.X, h2d, t.s_in);
    if (e == cudaSuccess) e = copy_range((void*)dev->U, host->U, d8, a.U, b.U, h2d, t.s_in);
    if (e == cudaSuccess) e = copy_range((void*)dev->s, host->s, d8, a.s, b.s, h2d, t.s_in);
    if (vjp && e == cudaSuccess) e = copy_range((void*)dev_vjp->w, host_vjp->w, d8, a.defect, b.defect, h2d, t.s_in);
    if (vjp && e == cudaSuccess) e = copy_range((void*)dev_vjp->rho, host_vjp->rho, d8, a.penalty, b.penalty, h2d, t.s_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, t.s_in);
    // compute
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t.s_comp, ev_in, 0);
    if (e == cudaSuccess) {
      if (vjp) e = launch_fused_c(p, common_chunk(p, 0, c, p->tune_fused), dev, &dv, part, ps, pL, i0, i1, t.s_comp);
      else e = launch_disc_c(p, common_chunk(p, 0, c, p->tune), dev, t.s_comp);
      if (e == cudaSuccess && p->any_cpl)
        e = run_coupled_range(p, dev, vjp ? &dv : nullptr, vjp ? (char*)workspace + cpl_ws_offset(p) : nullptr,
                              vjp ? ws_bytes - cpl_ws_offset(p) : 0, i0, i1, t.s_comp);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp, t.s_comp);
    // device -> host: this chunk's outputs
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t.s_out, ev_comp, 0);
    if (e == cudaSuccess) e = copy_range(host->A, dev->A, phi, a.A, b.A, d2h, t.s_out);
    if (e == cudaSuccess) e = copy_range(host->Bm, dev->Bm, phi, a.B, b.B, d2h, t.s_out);
    if (e == cudaSuccess) e = copy_range(host->Bp, dev->Bp, phi, a.B, b.B, d2h, t.s_out);
    if (e == cudaSuccess) e = copy_range(host->S, dev->S, phi, a.S, b.S, d2h, t.s_out);
    if (e == cudaSuccess) e = copy_range(host->defect, dev->defect, d8, a.defect, b.defect, d2h, t.s_out);
    if (e == cudaSuccess) e = copy_range(host->penalty, dev->penalty, d8, a.penalty, b.penalty, d2h, t.s_out);
    if (vjp) {
      if (e == cudaSuccess) e = copy_range(host_vjp->gX, dev_vjp->gX, d8, a.X, b.X, d2h, t.s_out);
      if (e == cudaSuccess) e = copy_range(host_vjp->gU, dev_vjp->gU, d8, a.U, b.U, d2h, t.s_out);
      if (e == cudaSuccess) e = copy_range(host_vjp->gs, dev_vjp->gs, d8, a.s, b.s, d2h, t.s_out);
      if (e == cudaSuccess) e = copy_range(host_vjp->L, dev_vjp->L, d8, a.L, b.L, d2h, t.s_out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_out, t.s_out);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, t.ev[3 * n_chunks], 0);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "pipelined run: %s", cudaGetErrorString(e));
  return CISCVX_OK;
}

ciscvx_status ciscvx_batch_sync_status(const ciscvx_batch_plan* p, void* stream) {
  if (!p) return set_error(CISCVX_EINVAL, "null plan");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p->d_status, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(CISCVX_ECUDA, "status read: %s", cudaGetErrorString(e));
  if (h & ST_NONFINITE) return set_error(CISCVX_ENONFINITE, "non-finite state or block produced");
  return CISCVX_OK;
}

}  // extern "C"
