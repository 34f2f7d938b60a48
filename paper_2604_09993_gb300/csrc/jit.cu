// jit.cu — run-time specialization of the coupled path's tangent kernel.
//
// The tangent kernel's cost is dominated by runtime-indexed loops over the
// model's links, joints, contacts and rows.  For a given model shape
// (sizes, topology, row maps, skyline structure of K, stage-data layout,
// scheme, precision) this file writes a prelude of compile-time constants,
// appends the device source of cpl_tangent_jit.cuh (embedded at build time)
// and compiles it with NVRTC for the current GPU.  The robot's numbers (link
// inverses) stay kernel parameters, so every robot of a shape shares one
// compiled kernel; compiled kernels are cached per process by their source.
//
// NVRTC is loaded with dlopen and the driver entry points come through the
// runtime, so the library has no link-time dependency on either; when NVRTC
// is missing, compilation fails, or CISCVX_COUPLED_JIT=0 is set, the caller
// falls back to the generic kernel (same arithmetic).
#include <cuda.h>
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "coupled.cuh"
#include "cpl_jit_src.inc"  // kCplTangentJitSrc, kCplNominalJitSrc, kCplAdjointJitSrc (generated from the .cuh sources)

namespace ciscvx {

namespace {

// NVRTC entry points (dlopen)
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram* nvrtcProgram_t;
struct Nvrtc {
  nvrtcResult_t (*create)(nvrtcProgram_t*, const char*, const char*, int, const char* const*,
                          const char* const*);
  nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char* const*);
  nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t*);
  nvrtcResult_t (*log)(nvrtcProgram_t, char*);
  nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t*);
  nvrtcResult_t (*cubin)(nvrtcProgram_t, char*);
  nvrtcResult_t (*destroy)(nvrtcProgram_t*);
  bool ok = false;
};

// Driver entry points (through cudaGetDriverEntryPointByVersion)
struct Drv {
  CUresult (*load)(CUmodule*, const void*);
  CUresult (*get_fn)(CUfunction*, CUmodule, const char*);
  CUresult (*set_attr)(CUfunction, CUfunction_attribute, int);
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                     unsigned, CUstream, void**, void**);
  CUresult (*occ)(int*, CUfunction, int, size_t) = nullptr;  // optional
  bool ok = false;
};

std::mutex g_mu;
Nvrtc g_nvrtc;
Drv g_drv;
bool g_loaded = false;
std::map<std::string, CplJit> g_cache;

void load_apis() {
  if (g_loaded) return;
  g_loaded = true;
  const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
  void* h = nullptr;
  for (const char* nm : names)
    if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
  if (h) {
    g_nvrtc.create = (decltype(g_nvrtc.create))dlsym(h, "nvrtcCreateProgram");
    g_nvrtc.compile = (decltype(g_nvrtc.compile))dlsym(h, "nvrtcCompileProgram");
    g_nvrtc.log_size = (decltype(g_nvrtc.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    g_nvrtc.log = (decltype(g_nvrtc.log))dlsym(h, "nvrtcGetProgramLog");
    g_nvrtc.cubin_size = (decltype(g_nvrtc.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    g_nvrtc.cubin = (decltype(g_nvrtc.cubin))dlsym(h, "nvrtcGetCUBIN");
    g_nvrtc.destroy = (decltype(g_nvrtc.destroy))dlsym(h, "nvrtcDestroyProgram");
    g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.log_size && g_nvrtc.log &&
                 g_nvrtc.cubin_size && g_nvrtc.cubin && g_nvrtc.destroy;
  }
  auto entry = [](const char* sym, void** fn) {
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion(sym, fn, 13000, cudaEnableDefault, &q) == cudaSuccess &&
           q == cudaDriverEntryPointSuccess && *fn;
  };
  g_drv.ok = entry("cuModuleLoadData", (void**)&g_drv.load) &&
             entry("cuModuleGetFunction", (void**)&g_drv.get_fn) &&
             entry("cuFuncSetAttribute", (void**)&g_drv.set_attr) &&
             entry("cuLaunchKernel", (void**)&g_drv.launch);
  if (!entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void**)&g_drv.occ)) g_drv.occ = nullptr;
}

template <typename T>
void arr(std::ostringstream& o, const char* name, const T* v, int n) {
  o << "__device__ constexpr int " << name << "[" << (n > 0 ? n : 1) << "] = {";
  for (int i = 0; i < n; ++i) o << (i ? "," : "") << (int)v[i];
  if (n == 0) o << "0";
  o << "};\n";
}

void tab(std::ostringstream& o, const char* type, const char* name, const double* v, int n) {
  char buf[64];
  o << "__constant__ " << type << " " << name << "[" << n << "] = {";
  for (int i = 0; i < n; ++i) {
    std::snprintf(buf, sizeof buf, "%s(%s)%.17g", i ? "," : "", type, v[i]);
    o << buf;
  }
  o << "};\n";
}

std::string prelude(const CplTab& T, int prec, int bs) {
  std::ostringstream o;
  o << "#define CPL_TP " << (prec == CISCVX_FP64 ? "double" : "float") << "\n";
  o << "#define CPL_SCH " << T.scheme << "\n#define CPL_BS " << bs << "\n";
  o << "typedef CPL_TP TP;\n";
  o << "constexpr int NB = " << T.nb << ", NJ = " << T.nj << ", NC = " << T.nc << ", NXT = " << T.nxt
    << ", NU = " << T.nu << ", AUX = " << T.aux << ", JELIM = " << T.jelim << ", NK = " << T.nk
    << ", NL = " << T.nlive << ", NQD = " << T.nquad << ", CI0 = " << T.ci0 << ", CNT = " << T.cnt
    << ", NCF = " << T.ncf << ";\n";
  o << "constexpr int SD_ARM = " << T.sd_arm << ", SD_QW = " << T.sd_qw << ", SD_F = " << T.sd_F
    << ", SD_K = " << T.sd_K << ", SD_CON = " << T.sd_con << ", SD_SIZE = " << T.sd_size << ";\n";
  o << "constexpr int NSKY = " << T.nsky << ", PEN0 = " << T.pen0 << ";\n";
  o << "constexpr bool TERRAIN = " << (T.ta != 0.0 ? "true" : "false") << ";\n";
  arr(o, "JPAR", T.jpar, T.nj);
  arr(o, "JCHI", T.jchi, T.nj);
  arr(o, "NPOS", T.npos, T.nk ? T.nj : 0);
  arr(o, "NORD", T.nord, T.nk ? T.nj : 0);
  arr(o, "NF", T.nf, T.nk);
  arr(o, "NOFF", T.noff, T.nk ? T.nk + 1 : 0);
  arr(o, "CBODY", T.cbody, T.nc);
  arr(o, "CONTACT", T.contact, T.nb);
  arr(o, "LROW", T.lrow, T.nxt);
  arr(o, "QROW", T.qrow, T.nxt);
  std::vector<int> linv(T.nlive, -1), qinv(T.nquad > 0 ? T.nquad : 1, -1);
  for (int r = 0; r < T.nxt; ++r) {
    if (T.lrow[r] >= 0) linv[T.lrow[r]] = r;
    if (T.qrow[r] >= 0) qinv[T.qrow[r]] = r;
  }
  arr(o, "LINV", linv.data(), T.nlive);
  arr(o, "QINV", qinv.data(), T.nquad);
  // live rows whose derivative is a live velocity (theta, and p of contact
  // links): LVEL = the velocity's live index; the others are numbered by LDYN
  std::vector<int> ldyn(T.nlive, -1), lvel(T.nlive, -1);
  int nld = 0;
  for (int l = 0; l < T.nlive; ++l) {
    const int r = linv[l];
    if (r < 3 * T.nb && T.lrow[r + 3 * T.nb] >= 0) lvel[l] = T.lrow[r + 3 * T.nb];
    else ldyn[l] = nld++;
  }
  o << "constexpr int NLD = " << nld << ";\n";
  arr(o, "LDYN", ldyn.data(), T.nlive);
  arr(o, "LVEL", lvel.data(), T.nlive);
  arr(o, "CPERM", T.cperm, T.cnt);
  arr(o, "COLPTR", T.colptr, T.nxt + 1);  // compact A, column-major (CplTab::colptr)
  double a[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) a[6 * i + j] = T.a[i][j];
  tab(o, "TP", "TAB_A6", a, 36);
  tab(o, "TP", "TAB_B", T.b, 6);
  tab(o, "TP", "TAB_C", T.c, 6);
  tab(o, "TP", "TAB_BETA", T.beta, 6);
  tab(o, "double", "TABD_A6", a, 36);
  tab(o, "double", "TABD_B", T.b, 6);
  tab(o, "double", "TABD_C", T.c, 6);
  tab(o, "double", "TABD_BETA", T.beta, 6);
  double a2[36];  // the tableau squared: a kinematic row's stage value from its velocity's slopes
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
      for (int l = 0; l < 6; ++l) v += T.a[i][l] * T.a[l][j];
      a2[6 * i + j] = v;
    }
  tab(o, "double", "TABD_A26", a2, 36);
  o << "#define TAB_A(j, m) TAB_A6[6 * (j) + (m)]\n";
  o << "#define TABD_A(j, m) TABD_A6[6 * (j) + (m)]\n";
  o << "#define TABD_A2(j, m) TABD_A26[6 * (j) + (m)]\n";
  return o.str();
}

// Compiles `src` (cached) and returns its kernel `name`, or null.
const CplJit* compile(const std::string& src, const char* name, int bs, size_t smem);

}  // namespace

const CplJit* cpl_jit_tangent(const CplTab& T, int prec) {
  const char* env = std::getenv("CISCVX_COUPLED_JIT");
  if (env && env[0] == '0') return nullptr;
  const int bs = prec == CISCVX_FP64 ? 64 : 128;
  const size_t el = prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
  const size_t smem = T.scheme ? (size_t)5 * T.nlive * bs * el : 0;
  return compile(prelude(T, prec, bs) + kCplTangentJitSrc, "cpl_tangent", bs, smem);
}

const CplJit* cpl_jit_nominal(const CplTab& T, int prec) {
  const char* env = std::getenv("CISCVX_COUPLED_JIT");
  if (env && env[0] == '0') return nullptr;
  // per lane: K's skyline, the stored slopes (plus the RK4 accumulator), the
  // quadrature rows and the lever arms, in doubles; one warp per block
  // (RKF45 stores the slopes of the live rows that are not kinematic: theta
  // and the contact links' p follow from their velocities' slopes)
  const int nks = T.scheme ? 5 : 1;
  int nkin = 0;
  for (int r = 0; r < 3 * T.nb; ++r) nkin += T.lrow[r] >= 0 && T.lrow[r + 3 * T.nb] >= 0;
  const int nkr = T.scheme ? T.nlive - nkin : T.nlive;
  const size_t elems = (size_t)T.nsky + nks * nkr + (nks == 1 ? T.nlive : 0) + T.nquad + 4 * T.nj;
  const size_t smem = elems * sizeof(double) * 32;
  if (smem > 200u * 1024u) return nullptr;
  std::string src = prelude(T, prec, 32) + "#define CPL_NW 1\n" + kCplNominalJitSrc;
  return compile(src, "cpl_nominal", 32, smem);
}

const CplJit* cpl_jit_adjoint(const CplTab& T, int prec) {
  const char* env = std::getenv("CISCVX_COUPLED_JIT");
  if (env && env[0] == '0') return nullptr;
  const int bs = prec == CISCVX_FP64 ? 32 : 64;
  const size_t el = prec == CISCVX_FP64 ? sizeof(double) : sizeof(float);
  const size_t smem = T.scheme ? (size_t)6 * T.nlive * bs * el : 0;  // RKF45's stage slope cotangents
  return compile(prelude(T, prec, bs) + kCplAdjointJitSrc, "cpl_adjoint", bs, smem);
}

namespace {

const CplJit* compile(const std::string& src0, const char* name, int bs, size_t smem) {
  // a loaded module belongs to the current device's context: key by device too
  int cur = 0;
  cudaGetDevice(&cur);
  const std::string src = "// device " + std::to_string(cur) + "\n" + src0;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(src);
  if (it != g_cache.end()) return it->second.fn ? &it->second : nullptr;
  CplJit& J = g_cache[src];  // a failed compile is cached too (fn stays null)
  load_apis();
  if (!g_nvrtc.ok || !g_drv.ok) return nullptr;
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  char arch[64];
  std::snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%d%s", major, minor,
                (major == 10 && minor == 3) ? "a" : "");
  // CISCVX_JIT_LOG also asks ptxas for the kernel's registers and spills
  const char* opts[] = {arch, "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
  const int nopt = std::getenv("CISCVX_JIT_LOG") ? 4 : 3;
  nvrtcProgram_t prog = nullptr;
  if (g_nvrtc.create(&prog, src.c_str(), "cpl_tangent_jit.cu", 0, nullptr, nullptr) != 0) return nullptr;
  const int rc = g_nvrtc.compile(prog, nopt, opts);
  if (rc != 0 || std::getenv("CISCVX_JIT_LOG")) {
    size_t n = 0;
    g_nvrtc.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) g_nvrtc.log(prog, &log[0]);
    std::fprintf(stderr, "ciscvx: coupled %s kernel compile %s\n%s\n", name, rc ? "failed" : "log", log.c_str());
  }
  if (rc != 0) { g_nvrtc.destroy(&prog); return nullptr; }
  size_t nb = 0;
  g_nvrtc.cubin_size(prog, &nb);
  std::vector<char> cubin(nb);
  g_nvrtc.cubin(prog, cubin.data());
  g_nvrtc.destroy(&prog);
  cudaFree(nullptr);  // the runtime's primary context is current on this thread
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
  if (g_drv.load(&mod, cubin.data()) != CUDA_SUCCESS) return nullptr;
  if (g_drv.get_fn(&fn, mod, name) != CUDA_SUCCESS) return nullptr;
  if (smem > 48u * 1024u &&
      g_drv.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
    return nullptr;
  J.fn = (void*)fn;
  J.bs = bs;
  J.smem = smem;
  int nblk = 0;
  if (g_drv.occ && g_drv.occ(&nblk, fn, bs, smem) == CUDA_SUCCESS) J.blocks_per_sm = nblk;
  return &J;
}

}  // namespace

cudaError_t cpl_jit_launch_nominal(const CplJit& J, const CplTab& T, long i0, long n, int nsub,
                                   int layout, const double* X, const double* U, const double* s,
                                   void* sd, void* A, double* defect, double* penalty,
                                   unsigned* status, cudaStream_t st, const int2* entries,
                                   const DevInst* inst, int cmp) {
  // NumN {mass, minv, iinv [NB]; jrp, jrc [max(NJ,1)][2]; crho [max(NC,1)][2]; mu [max(NC,1)]; g, ta, tk}
  std::vector<double> num;
  const int nj1 = T.nj > 0 ? T.nj : 1, nc1 = T.nc > 0 ? T.nc : 1;
  for (int b = 0; b < T.nb; ++b) num.push_back(T.mass[b]);
  for (int b = 0; b < T.nb; ++b) num.push_back(T.minv[b]);
  for (int b = 0; b < T.nb; ++b) num.push_back(T.iinv[b]);
  for (int j = 0; j < nj1; ++j) { num.push_back(j < T.nj ? T.jrp[j][0] : 0.0); num.push_back(j < T.nj ? T.jrp[j][1] : 0.0); }
  for (int j = 0; j < nj1; ++j) { num.push_back(j < T.nj ? T.jrc[j][0] : 0.0); num.push_back(j < T.nj ? T.jrc[j][1] : 0.0); }
  for (int i = 0; i < nc1; ++i) { num.push_back(i < T.nc ? T.crho[i][0] : 0.0); num.push_back(i < T.nc ? T.crho[i][1] : 0.0); }
  for (int i = 0; i < nc1; ++i) num.push_back(i < T.nc ? T.mu[i] : 0.0);
  num.push_back(T.g);
  num.push_back(T.ta);
  num.push_back(T.tk);
  void* args[] = {num.data(), &i0, &n, &nsub, &layout, &X, &U, &s, &sd, &A, &defect, &penalty, &status,
                  &entries, &inst, &cmp};
  const unsigned grid = (unsigned)((n + J.bs - 1) / J.bs);
  const CUresult r = g_drv.launch((CUfunction)J.fn, grid, 1, 1, J.bs, 1, 1, (unsigned)J.smem, (CUstream)st, args, nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t cpl_jit_launch(const CplJit& J, const CplTab& T, int prec, long i0, long n, int nsub,
                           const double* s, const void* sd, void* A, void* Bm, void* Bp, void* S,
                           unsigned* status, cudaStream_t st, int layout, const int2* entries,
                           const DevInst* inst, int cmp) {
  // Num {TP minv[NB]; TP iinv[NB];}
  unsigned char num[2 * MAXB * sizeof(double)];
  if (prec == CISCVX_FP64) {
    double* d = (double*)num;
    for (int b = 0; b < T.nb; ++b) { d[b] = T.minv[b]; d[T.nb + b] = T.iinv[b]; }
  } else {
    float* f = (float*)num;
    for (int b = 0; b < T.nb; ++b) { f[b] = T.minvf[b]; f[T.nb + b] = T.iinvf[b]; }
  }
  void* args[] = {num, &i0, &n, &nsub, &s, &sd, &A, &Bm, &Bp, &S, &status, &layout, &entries, &inst, &cmp};
  const long threads = n * T.cnt;
  const unsigned grid = (unsigned)((threads + J.bs - 1) / J.bs);
  const CUresult r = g_drv.launch((CUfunction)J.fn, grid, 1, 1, J.bs, 1, 1, (unsigned)J.smem, (CUstream)st, args, nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t cpl_jit_launch_adjoint(const CplJit& J, const CplTab& T, int prec, long i0, long n, long N, int nsub,
                                   const double* s, const void* sd, const double* w, const double* rho,
                                   double* gX, double* gs, double* ubar, unsigned* status, cudaStream_t st) {
  // NumA {TP minv[NB]; TP iinv[NB];}
  unsigned char num[2 * MAXB * sizeof(double)];
  if (prec == CISCVX_FP64) {
    double* d = (double*)num;
    for (int b = 0; b < T.nb; ++b) { d[b] = T.minv[b]; d[T.nb + b] = T.iinv[b]; }
  } else {
    float* f = (float*)num;
    for (int b = 0; b < T.nb; ++b) { f[b] = T.minvf[b]; f[T.nb + b] = T.iinvf[b]; }
  }
  void* args[] = {num, &i0, &n, &N, &nsub, &s, &sd, &w, &rho, &gX, &gs, &ubar, &status};
  const unsigned grid = (unsigned)((n + J.bs - 1) / J.bs);
  const CUresult r = g_drv.launch((CUfunction)J.fn, grid, 1, 1, J.bs, 1, 1, (unsigned)J.smem, (CUstream)st, args, nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace ciscvx
