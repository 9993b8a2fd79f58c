// Specialised fused-pass kernels: source generation per pass structure, NVRTC compilation
// (libnvrtc opened at run time), an on-disk cubin cache and loading through cudaLibrary.
//
// Every fused pass is a straight-line program of register phases. Its structure (tile size, register
// bits of each phase, op kinds and operand bits, shared-memory layouts) becomes compile-time code in a
// generated "Spec" struct; passes with the same structure share one kernel. Per-pass data that does not
// change the code (physical bit positions, the gate of every op) is passed at run time.
#include "jit.hpp"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <algorithm>
#include <map>
#include <atomic>
#include <mutex>
#include <thread>
#include <sstream>

#include "launch.hpp"

namespace qsim {

#include "jit_embed.inc"   // const char* kJitDeviceSource (jit_device.cuh as text)

// ------------------------------------------------------------------ NVRTC via dlopen
namespace {
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram* nvrtcProgram_t;
struct Nvrtc {
  void* h = nullptr;
  nvrtcResult_t (*create)(nvrtcProgram_t*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
  nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char* const*) = nullptr;
  nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t*) = nullptr;
  nvrtcResult_t (*log)(nvrtcProgram_t, char*) = nullptr;
  nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t*) = nullptr;
  nvrtcResult_t (*cubin)(nvrtcProgram_t, char*) = nullptr;
  nvrtcResult_t (*destroy)(nvrtcProgram_t*) = nullptr;
  nvrtcResult_t (*version)(int*, int*) = nullptr;
  std::string error;
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    std::vector<std::string> cand = {"libnvrtc.so.13", "libnvrtc.so"};
    if (const char* ch = getenv("CUDA_HOME")) cand.push_back(std::string(ch) + "/lib64/libnvrtc.so.13");
    cand.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    cand.push_back("/usr/local/cuda/lib64/libnvrtc.so");
    for (auto& c : cand) {
      n.h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL);
      if (n.h) break;
    }
    if (!n.h) {
      n.error = "cannot load libnvrtc (set CUDA_HOME): " + std::string(dlerror() ? dlerror() : "");
      return;
    }
#define QSIM_SYM(F, NAME)                                                       \
  n.F = reinterpret_cast<decltype(n.F)>(dlsym(n.h, NAME));                     \
  if (!n.F) {                                                                  \
    n.error = std::string("libnvrtc lacks ") + NAME;                           \
    n.h = nullptr;                                                             \
    return;                                                                    \
  }
    QSIM_SYM(create, "nvrtcCreateProgram")
    QSIM_SYM(compile, "nvrtcCompileProgram")
    QSIM_SYM(log_size, "nvrtcGetProgramLogSize")
    QSIM_SYM(log, "nvrtcGetProgramLog")
    QSIM_SYM(cubin_size, "nvrtcGetCUBINSize")
    QSIM_SYM(cubin, "nvrtcGetCUBIN")
    QSIM_SYM(destroy, "nvrtcDestroyProgram")
    QSIM_SYM(version, "nvrtcVersion")
#undef QSIM_SYM
  });
  return n;
}

typedef struct nvJitLink* nvJitLinkHandle_t;
struct JitLinker {
  void* h = nullptr;
  int (*create)(nvJitLinkHandle_t*, uint32_t, const char**) = nullptr;
  int (*destroy)(nvJitLinkHandle_t*) = nullptr;
  int (*add_data)(nvJitLinkHandle_t, int, const void*, size_t, const char*) = nullptr;
  int (*complete)(nvJitLinkHandle_t) = nullptr;
  int (*cubin_size)(nvJitLinkHandle_t, size_t*) = nullptr;
  int (*cubin)(nvJitLinkHandle_t, void*) = nullptr;
  int (*err_size)(nvJitLinkHandle_t, size_t*) = nullptr;
  int (*err_log)(nvJitLinkHandle_t, char*) = nullptr;
  std::string error;
};

JitLinker& jitlink() {
  static JitLinker n;
  static std::once_flag once;
  std::call_once(once, [] {
    std::vector<std::string> cand = {"libnvJitLink.so.13", "libnvJitLink.so"};
    if (const char* ch = getenv("CUDA_HOME")) cand.push_back(std::string(ch) + "/lib64/libnvJitLink.so.13");
    cand.push_back("/usr/local/cuda/lib64/libnvJitLink.so.13");
    for (auto& c : cand) {
      n.h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL);
      if (n.h) break;
    }
    if (!n.h) {
      n.error = "cannot load libnvJitLink (set CUDA_HOME)";
      return;
    }
#define QSIM_SYM(F, NAME)                                                       \
  n.F = reinterpret_cast<decltype(n.F)>(dlsym(n.h, NAME));                     \
  if (!n.F) {                                                                  \
    n.error = std::string("libnvJitLink lacks ") + NAME;                       \
    n.h = nullptr;                                                             \
    return;                                                                    \
  }
    QSIM_SYM(create, "__nvJitLinkCreate_13_0")
    QSIM_SYM(destroy, "__nvJitLinkDestroy_13_0")
    QSIM_SYM(add_data, "__nvJitLinkAddData_13_0")
    QSIM_SYM(complete, "__nvJitLinkComplete_13_0")
    QSIM_SYM(cubin_size, "__nvJitLinkGetLinkedCubinSize_13_0")
    QSIM_SYM(cubin, "__nvJitLinkGetLinkedCubin_13_0")
    QSIM_SYM(err_size, "__nvJitLinkGetErrorLogSize_13_0")
    QSIM_SYM(err_log, "__nvJitLinkGetErrorLog_13_0")
#undef QSIM_SYM
  });
  return n;
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ULL) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ULL;
  }
  return h;
}

std::string hex64(uint64_t v) {
  char b[17];
  snprintf(b, sizeof b, "%016llx", (unsigned long long)v);
  return b;
}

std::string cache_dir() {
  if (const char* e = getenv("QSIM_JIT_CACHE")) return e;
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&cache_dir), &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    size_t s = p.rfind('/');
    if (s != std::string::npos) return p.substr(0, s) + "/_jit_cache";
  }
  return "/tmp/qsim_jit_cache";
}

bool read_file(const std::string& path, std::string& out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream o;
  o << f.rdbuf();
  out = o.str();
  return true;
}

void write_file_atomic(const std::string& dir, const std::string& path, const std::string& data) {
  mkdir(dir.c_str(), 0755);
  std::string tmp = path + ".tmp." + std::to_string(getpid());
  {
    std::ofstream f(tmp, std::ios::binary);
    if (!f) return;
    f.write(data.data(), (std::streamsize)data.size());
  }
  rename(tmp.c_str(), path.c_str());
}

// shared-memory layout function of a DevLayout as C++ source
std::string lay_fn(const std::string& name, const DevLayout& L, int k) {
  std::ostringstream o;
  o << "  static __device__ __forceinline__ qj::u32 " << name << "(qj::u32 e) { return e";
  for (int j = 0; j < k; j++)
    if (L.m[j]) o << " ^ (((e >> " << j << ") & 1u) ? " << (unsigned)L.m[j] << "u : 0u)";
  o << "; }\n";
  return o.str();
}

uint32_t lay_eval(const DevLayout& L, int k, uint32_t e) {
  uint32_t s = e;
  for (int j = 0; j < k; j++)
    if ((e >> j) & 1u) s ^= L.m[j];
  return s;
}

}  // namespace

// ------------------------------------------------------------------ generation
// Ops of a phase in the order a pass runs them (backward: reversed), without the CNOTs that open the
// phase (forward order) with the control on a thread bit and the target on a register bit >= 1: those
// fold into the thread's addresses instead.
static std::vector<int> phase_order(const Schedule& s, const DevPhase& Ph, bool bwd, size_t* n_fold = nullptr) {
  size_t nf = 0;
  for (int oi = Ph.op_begin; oi < Ph.op_end; oi++) {
    const DevOp& op = s.ops[oi];
    if (op.kind != K_CNOT_RT || op.a < 1) break;
    nf++;
  }
  std::vector<int> order;
  for (int oi = Ph.op_begin + (int)nf; oi < Ph.op_end; oi++) order.push_back(oi);
  if (bwd) std::reverse(order.begin(), order.end());
  if (n_fold) *n_fold = nf;
  return order;
}

static bool is_diag_op(const DevOp& op) {
  return op.kind == K_RZ_R || op.kind == K_RZ_T || op.kind == K_CZ_RR || op.kind == K_CZ_RT || op.kind == K_CZ_TT;
}

// [x, y) ranges of a phase's op order that run as one merged diagonal factor per amplitude. The merged
// run costs a complex multiply per amplitude (two in the backward, where it also saves two FMAs of
// gradient and four of updates per RZ): worth it from 2 RZs backward, 4 forward.
static std::vector<std::pair<size_t, size_t>> diag_ranges(const Schedule& s, const std::vector<int>& order, bool bwd) {
  std::vector<std::pair<size_t, size_t>> r;
  if (!s.merge_diag) return r;
  for (size_t x = 0; x < order.size();) {
    size_t y = x;
    int n_rz = 0;
    while (y < order.size() && is_diag_op(s.ops[order[y]])) n_rz += s.ops[order[y++]].rot;
    if (n_rz >= (bwd ? 2 : 4)) {
      r.push_back({x, y});
      x = y;
    } else {
      x++;
    }
  }
  return r;
}

// Register bits of a merged run with a per-bit factor (an RZ or a register-thread CZ on them), sorted.
static std::vector<int> diag_used_bits(const Schedule& s, const std::vector<int>& run) {
  std::vector<int> used;
  for (int oi : run) {
    const DevOp& op = s.ops[oi];
    const int rb = op.kind == K_RZ_R ? op.a : op.kind == K_CZ_RT ? op.a : -1;
    if (rb >= 0 && std::find(used.begin(), used.end(), rb) == used.end()) used.push_back(rb);
  }
  std::sort(used.begin(), used.end());
  return used;
}

// One merged diagonal run of a pass with its factor table: for every value of the used register bits
// the product of the run's register-bit RZ factors, per sample, built in shared memory while a tile's
// loads are in flight. off: first element (in units of T); es: T values per entry (2: (re, im); 4:
// (re, re, im, im), the packed backward's FP32x2 operands).
// Runs whose table has more entries than the tile has threads (tiny tiles: a 5-qubit circuit's tile
// is one thread) form their factors in registers instead, by a butterfly over the used bits (tab false).
struct DiagRun {
  std::vector<int> ops;
  std::vector<int> used;
  int off = 0, es = 2;
  bool tab = true;
};

// The merged runs of a pass in the order the generated code meets them (phase steps, then op order).
static std::vector<DiagRun> pass_diag_runs(const Schedule& s, const DevPass& d, bool bwd, int* units = nullptr) {
  std::vector<DiagRun> runs;
  const int P = d.n_phases;
  const int es = bwd && s.packed_bwd ? 4 : 2;
  const int nthr = 1 << (d.k - d.R);
  int off = 0;
  for (int step = 0; step < P; step++) {
    const int ph = bwd ? P - 1 - step : step;
    const DevPhase& Ph = s.phases[d.phase0 + ph];
    const std::vector<int> order = phase_order(s, Ph, bwd);
    for (auto& xy : diag_ranges(s, order, bwd)) {
      DiagRun r;
      r.ops.assign(order.begin() + xy.first, order.begin() + xy.second);
      r.used = diag_used_bits(s, r.ops);
      r.es = es;
      r.tab = (1 << r.used.size()) <= nthr;
      r.off = r.tab ? off : -1;
      if (r.tab) off += es << r.used.size();
      runs.push_back(r);
    }
  }
  if (units) *units = off;
  return runs;
}

static int diag_table_units(const Schedule& s, const DevPass& d, bool bwd) {
  int u = 0;
  pass_diag_runs(s, d, bwd, &u);
  return u;
}

// Backward gradient partials live in shared memory until the end of the tile: one per gradient slot
// and group of 2^GS neighbouring threads, GS the smallest level (no shuffles at all for GS = 0) for
// which they fit in 32 KiB per CTA; deep passes, or many small tile groups in one CTA of a
// multi-circuit queue kernel, take GS up to a whole warp. cta: threads of the queue kernel's CTA
// (0: one tile per CTA).
static int grad_level(const DevPass& d, int dtype, int cta, int max_regs = 0, size_t tab_bytes = 0) {
  const size_t sc = dtype == QSIM_C128 ? 8 : 4;
  const size_t ng = d.n_gslots > 0 ? d.n_gslots : 1;
  const int lt = d.k - d.R;                      // log2 threads per tile
  const size_t groups = cta > 0 ? std::max<size_t>(1, (size_t)cta >> lt) : 1;
  size_t budget = cta > 0 ? 16 * 1024 : 32 * 1024;   // queue kernels: keep CTAs small (see multi.cpp)
  if (cta == 0 && max_regs > 0) {
    // a register cap asks for as many CTAs per SM as the registers allow: keep the shared memory of
    // one CTA (plus the 1 KiB the SM reserves per CTA) within 228 KiB divided by that count
    const size_t ctas = std::max<size_t>(1, 65536 / (((size_t)1 << lt) * (size_t)max_regs));
    const size_t per_cta = 228 * 1024 / ctas - 1024;
    const size_t fixed = 2 * ((2 * sc) << d.k) + (d.k + 2) * 8 + tab_bytes + (size_t)(d.n_ops + 1) * (sc + 1) + 48;
    budget = std::min(budget, per_cta > fixed ? per_cta - fixed : 0);
  }
  const int cap = std::min(lt, 5);
  for (int gs = 0; gs < cap; gs++)
    if (ng * ((size_t)1 << (lt - gs)) * sc * groups <= budget) return gs;
  return cap;
}

static std::string gen_spec_body(const Schedule& s, const DevPass& d, bool bwd, int cta = 0, bool prefix = false) {
  const int K = d.k, R = d.R, N = 1 << R, NTHR = 1 << (K - R);
  const int P = d.n_phases;
  std::ostringstream o;
  o << "  static constexpr int CTA = " << (cta > 0 ? cta : NTHR) << ";\n";
  o << "  static constexpr int NOPS = " << d.n_ops << ";\n";
  o << "  static constexpr int NGS = " << (bwd ? d.n_gslots : 0) << ";\n";
  int ntab = 0;
  const std::vector<DiagRun> druns = pass_diag_runs(s, d, bwd, &ntab);
  const size_t sc_bytes = s.dtype == QSIM_C128 ? 8 : 4;
  const int gs = bwd ? grad_level(d, s.dtype, cta, s.max_regs, (size_t)ntab * sc_bytes) : 0;
  o << "  static constexpr int GS = " << gs << ";\n";
  o << "  static constexpr int NTAB = " << ntab << ";\n";
  // factor tables of the merged diagonal runs (see DiagRun), from the sample's coefficients in global
  // memory; the barrier after the staging publishes them
  o << "  template <typename T> static __device__ __forceinline__ void build_tables(qj::Ctx<T>& c, const T* src) {\n"
    << "    (void)c; (void)src;\n";
  for (const DiagRun& r : druns) {
    if (!r.tab) continue;
    const int nu = (int)r.used.size();
    o << "    for (qj::u32 e = c.tid; e < " << (1u << nu) << "u; e += " << NTHR << "u) {\n"
      << "      T dr = T(1), di = T(0);\n";
    for (int k2 = 0; k2 < nu; k2++) {
      std::vector<int> lis;
      for (int oi : r.ops)
        if (s.ops[oi].kind == K_RZ_R && s.ops[oi].a == r.used[k2]) lis.push_back(oi - d.op0);
      if (lis.empty()) continue;
      o << "      { T ur = T(1), ui = T(0); const T sg = ((e >> " << k2 << ") & 1u) ? T(1) : T(-1);";
      for (int li : lis) o << " qj::cmul(ur, ui, T(1), sg * src[" << li << "]);";
      o << " qj::cmul(dr, di, ur, ui); }\n";
    }
    if (r.es == 4)
      o << "      T* t = c.tab + " << r.off << " + 4 * e; t[0] = dr; t[1] = dr; t[2] = di; t[3] = di;\n";
    else
      o << "      T* t = c.tab + " << r.off << " + 2 * e; t[0] = dr; t[1] = di;\n";
    o << "    }\n";
  }
  o << "  }\n";
  for (int i = 0; i <= P; i++) o << lay_fn("L" + std::to_string(i), s.layouts[d.lay0 + i], K);
  auto dep_of = [&](const DevPhase& ph, int i) {
    uint32_t e = 0;
    for (int r = 0; r < R; r++)
      if ((i >> r) & 1) e |= 1u << ph.rbit[r];
    return e;
  };
  // shared-memory element of a phase's register pair i in layout Lx = (thread part) ^ (constant part);
  // when the two parts cannot share a bit the XOR is an addition (the constant folds into the offset)
  auto disjoint = [&](const DevLayout& Lx, const DevPhase& ph) {
    uint32_t mt = 0, mr = 0;
    for (int jb = 0; jb < ph.n_tbits; jb++) mt |= lay_eval(Lx, K, 1u << ph.tbit[jb]);
    for (int r = 1; r < R; r++) mr |= lay_eval(Lx, K, 1u << ph.rbit[r]);
    return (mt & mr) == 0;
  };
  // <Z> bit map of the phase that stores to global memory (forward: the last phase)
  if (!bwd) {
    const DevPhase& lp = s.phases[d.phase0 + P - 1];
    o << "  static __device__ __forceinline__ int zmap(int j) {\n    switch (j) {\n";
    for (int r = 0; r < R; r++) o << "      case " << (int)lp.rbit[r] << ": return " << r << ";\n";
    for (int p = 0; p < lp.n_tbits; p++) o << "      case " << (int)lp.tbit[p] << ": return " << -1 - p << ";\n";
    o << "      default: return 0;\n    }\n  }\n";
  }
  // global offset of the thread's base element and of the register bits, for a phase, in the layout
  // the pass reads (out = false: a.L, c.base) or writes (out = true: a.Lo, c.base_out)
  auto gaddr = [&](const DevPhase& ph, const std::string& var, bool out) {
    const char* Lv = out ? "a.Lo" : "a.L";
    std::ostringstream g;
    g << "      qj::i64 " << var << " = " << (out ? "c.base_out" : "c.base") << ";\n";
    for (int jb = 0; jb < ph.n_tbits; jb++)
      g << "      if ((tid >> " << jb << ") & 1u) " << var << " |= (qj::i64)1 << " << Lv << "[" << (int)ph.tbit[jb] << "];\n";
    for (int r = 1; r < R; r++)
      g << "      const qj::i64 " << var << "u" << r << " = (qj::i64)1 << " << Lv << "[" << (int)ph.rbit[r] << "];\n";
    return g.str();
  };
  // address of register pair i from a base and the offsets <offs>u<r> (XOR: a folded base may
  // already carry a register bit)
  auto goff = [&](const std::string& base, const std::string& offs, int i) {
    std::string e = base;
    for (int r = 1; r < R; r++)
      if ((i >> r) & 1) e += " ^ " + offs + "u" + std::to_string(r);
    return "(" + e + ")";
  };
  // names of psi / lambda components of register element i in the backward
  const bool pk = bwd && s.packed_bwd;
  auto PR = [&](int i) { return pk ? "X[" + std::to_string(i) + "].x" : "pr[" + std::to_string(i) + "]"; };
  auto PQ = [&](int i) { return pk ? "Y[" + std::to_string(i) + "].x" : "pq[" + std::to_string(i) + "]"; };
  auto LR = [&](int i) { return pk ? "X[" + std::to_string(i) + "].y" : "lr[" + std::to_string(i) + "]"; };
  auto LQ = [&](int i) { return pk ? "Y[" + std::to_string(i) + "].y" : "lq[" + std::to_string(i) + "]"; };
  if (!bwd) {
    o << "  template <typename T> static __device__ __forceinline__ void fwd_phases(qj::Ctx<T>& c) {\n"
      << "    const qj::Args& a = *c.a;\n    const qj::u32 tid = c.tid;\n"
      << "    T re[" << N << "], im[" << N << "];\n";
  } else {
    o << "  template <typename T, typename A> static __device__ __forceinline__ void bwd_phases(qj::Ctx<T>& c, A* red) {\n"
      << "    const qj::Args& a = *c.a;\n    const qj::u32 tid = c.tid;\n";
    if (pk)   // (Re psi, Re lambda) and (Im psi, Im lambda) register pairs
      o << "    float2 X[" << N << "], Y[" << N << "];\n";
    else
      o << "    T pr[" << N << "], pq[" << N << "], lr[" << N << "], lq[" << N << "];\n";
    o << "    const qj::u32 lane = tid & 31u, warp = tid >> 5;\n    (void)lane; (void)warp;\n";
  }
  size_t run_i = 0;   // next entry of druns
  for (int step = 0; step < P; step++) {
    const int ph = bwd ? P - 1 - step : step;
    const DevPhase& Ph = s.phases[d.phase0 + ph];
    const int lin = bwd ? ph + 1 : ph, lout = bwd ? ph : ph + 1;
    const bool first = step == 0, last = step == P - 1;
    const DevLayout& Li = s.layouts[d.lay0 + lin];
    const DevLayout& Lo = s.layouts[d.lay0 + lout];
    o << "    { // phase " << ph << (first ? " (loads from global)" : "") << (last ? " (stores to global)" : "") << "\n";
    // CNOTs that open the phase (forward order) with the control on a thread bit and the target on a
    // register bit >= 1 are conditional register swaps; they become an XOR of the thread's base
    // address instead: at the load in the forward, at the store in the backward (applied last there).
    size_t n_fold = 0;
    const std::vector<int> order = phase_order(s, Ph, bwd, &n_fold);
    std::vector<const DevOp*> fold;
    for (size_t f = 0; f < n_fold; f++) fold.push_back(&s.ops[Ph.op_begin + (int)f]);
    auto fold_smem = [&](const DevLayout& Lx) {
      std::string t;
      for (const DevOp* op : fold)
        t += " ^ (((tb >> " + std::to_string(op->b) + ") & 1u) ? " +
             std::to_string(lay_eval(Lx, K, dep_of(Ph, 1 << op->a))) + "u : 0u)";
      return t;
    };
    auto fold_glob = [&](const std::string& base, const std::string& from) {
      std::string t = "      qj::i64 " + base + " = " + from + ";\n";
      for (const DevOp* op : fold)
        t += "      if ((tb >> " + std::to_string(op->b) + ") & 1u) " + base + " ^= " + from + "u" +
             std::to_string(op->a) + ";\n";
      return t;
    };
    // register bit r of a folded CNOT target holds the element with that bit flipped where the control is
    // set: the prefix factors of that qubit swap their two values there
    auto fold_swap = [&](int r) {
      std::string t = "0u";
      for (const DevOp* op : fold)
        if (op->a == r) t += " ^ ((tb >> " + std::to_string(op->b) + ") & 1u)";
      return t;
    };
    o << "      const qj::u32 tb = 0u";
    for (int jb = 0; jb < Ph.n_tbits; jb++) o << " | (((tid >> " << jb << ") & 1u) << " << (int)Ph.tbit[jb] << ")";
    o << ";\n      (void)tb;\n";
    if (first) o << gaddr(Ph, "gb", false);
    if (last) o << gaddr(Ph, "gs", true);
    // ---- load
    if (first) {
      if (!bwd) {
        // product-state prefix: psi(x) = prod_q phi_q(x_q), the tile-index and thread bits' factors in one
        // product, then a butterfly over the register bits
        if (prefix) {
        o << "      if (a.in == nullptr && a.phi != nullptr) {\n"
          << "        const T* ph = reinterpret_cast<const T*>(a.phi) + c.b * a.n * 4;\n"
          << "        T br, bi;\n        qj::phi_nonlocal<T>(a, ph, c.t, br, bi);\n";
        for (int jb = 0; jb < Ph.n_tbits; jb++)
          o << "        { const T* f = ph + 4 * a.Q[" << (int)Ph.tbit[jb] << "] + 2 * ((tid >> " << jb
            << ") & 1u); qj::cmul(br, bi, f[0], f[1]); }\n";
        o << "        re[0] = br; im[0] = bi;\n";
        for (int r = 0; r < R; r++)
          o << "        { const qj::u32 sw = " << fold_swap(r) << "; const T* f = ph + 4 * a.Q[" << (int)Ph.rbit[r]
            << "];\n          const T f0r = f[2 * sw], f0i = f[2 * sw + 1], f1r = f[2 - 2 * sw], f1i = f[3 - 2 * sw];\n"
            << "          for (int i = 0; i < " << (1 << r) << "; i++) { re[i + " << (1 << r) << "] = re[i]; im[i + "
            << (1 << r) << "] = im[i]; qj::cmul(re[i + " << (1 << r) << "], im[i + " << (1 << r)
            << "], f1r, f1i); qj::cmul(re[i], im[i], f0r, f0i); }\n        }\n";
        }
        o << (prefix ? "      } else if (a.in == nullptr) {\n" : "      if (a.in == nullptr) {\n");
        for (int i = 0; i < N; i++) o << "        re[" << i << "] = T(0); im[" << i << "] = T(0);\n";
        o << "        if (tb == 0u && c.t == 0) re[0] = T(1);\n      } else {\n"
          << "        const T* in = reinterpret_cast<const T*>(a.in);\n";
        o << fold_glob("gl", "gb");
        for (int i = 0; i < N; i += 2)
          o << "        qj::ldg_pair(in + 2 * " << goff("gl", "gb", i) << ", re[" << i << "], im[" << i << "], re[" << i + 1
            << "], im[" << i + 1 << "]);\n";
        o << "      }\n";
        o << "      qj::stage_fwd<T, " << NTHR << ", S_SELF>(c);\n      __syncthreads();\n";
      } else {
        o << "      {\n        const T* in = reinterpret_cast<const T*>(a.in);\n";
        for (int i = 0; i < N; i += 2)
          o << "        qj::ldg_pair(in + 2 * " << goff("gb", "gb", i) << ", " << PR(i) << ", " << PQ(i) << ", " << PR(i + 1)
            << ", " << PQ(i + 1) << ");\n";
        o << "      }\n      if (a.lam_in != nullptr) {\n        const T* li = reinterpret_cast<const T*>(a.lam_in);\n";
        for (int i = 0; i < N; i += 2)
          o << "        qj::ldg_pair(li + 2 * " << goff("gb", "gb", i) << ", " << LR(i) << ", " << LQ(i) << ", " << LR(i + 1)
            << ", " << LQ(i + 1) << ");\n";
        // lambda = d(e) psi, d(e) = gq[K] + sum_j (bit_j(e) ? -g_j : g_j)
        o << "      }\n      qj::stage_bwd<T, " << K << ", " << NTHR << ", S_SELF>(c);\n      __syncthreads();\n";
        o << "      if (a.lam_in == nullptr) {\n        T dt = c.gq[" << K << "];\n";
        for (int jb = 0; jb < Ph.n_tbits; jb++)
          o << "        dt += ((tid >> " << jb << ") & 1u) ? -c.gq[" << (int)Ph.tbit[jb] << "] : c.gq[" << (int)Ph.tbit[jb] << "];\n";
        // d(i) = dt + sum_r (bit r of i ? -g_r : g_r): the all-plus value, then a butterfly (subtract 2 g_r
        // for every set register bit), then lambda = d * psi, all in T
        o << "        T dd[" << N << "];\n        dd[0] = (T)(dt";
        for (int r = 0; r < R; r++) o << " + c.gq[" << (int)Ph.rbit[r] << "]";
        o << ");\n";
        for (int r = 0; r < R; r++)
          o << "        { const T m = T(2) * c.gq[" << (int)Ph.rbit[r] << "]; for (int i = 0; i < " << (1 << r)
            << "; i++) dd[i + " << (1 << r) << "] = dd[i] - m; }\n";
        for (int i = 0; i < N; i++)
          o << "        " << LR(i) << " = dd[" << i << "] * " << PR(i) << "; " << LQ(i) << " = dd[" << i << "] * " << PQ(i) << ";\n";
        o << "      }\n";
      }
    } else {
      const std::string fl = bwd ? std::string() : fold_smem(Li);
      const char* ad = fl.empty() && disjoint(Li, Ph) ? "true" : "false";
      o << "      const qj::u32 si = L" << lin << "(tb)" << fl << ";\n";
      for (int i = 0; i < N; i += 2) {
        const uint32_t cc = lay_eval(Li, K, dep_of(Ph, i));
        if (!bwd) {
          o << "      qj::ldpx<" << ad << ">(c.tile, si, " << cc << "u, re[" << i << "], im[" << i << "], re[" << i + 1 << "], im[" << i + 1 << "]);\n";
        } else if (pk) {
          o << "      qj::ldppx<" << ad << ">(c.tile, si, " << cc << "u, X[" << i << "], Y[" << i << "], X[" << i + 1 << "], Y[" << i + 1 << "]);\n";
        } else {
          o << "      qj::ldpx<" << ad << ">(c.tile, si, " << cc << "u, pr[" << i << "], pq[" << i << "], pr[" << i + 1 << "], pq[" << i + 1 << "]);\n";
          o << "      qj::ldpx<" << ad << ">(c.tile2, si, " << cc << "u, lr[" << i << "], lq[" << i << "], lr[" << i + 1 << "], lq[" << i + 1 << "]);\n";
        }
      }
    }
    // ---- ops
    // gradient partial of a rotation op (backward): one per thread, or summed over 2^gs lanes first
    auto emit_grad = [&](const DevOp& op, const std::string& expr) {
      if (gs == 0)
        o << "      red[" << op.gslot * NTHR << " + tid] = " << expr << ";\n";
      else
        o << "      { A g = qj::part_sum<" << (1 << gs) << ", A, CTA>(" << expr << "); if ((tid & " << ((1 << gs) - 1)
          << "u) == 0u) red[" << op.gslot * (NTHR >> gs) << " + (tid >> " << gs << ")] = g; }\n";
    };
    auto emit_op = [&](int oi) {
      const DevOp& op = s.ops[oi];
      const int li = oi - d.op0;
      const int SA = 1 << op.a, SB = 1 << op.b;
      // with a Pauli frame every rotation takes the tangent form (a literal 0 removes the other branch)
      std::string C = "c.cf[" + std::to_string(li) + "], " + (s.pauli_frame ? std::string("0") : "c.fm[" + std::to_string(li) + "]");
      std::string call;
      std::ostringstream g;
      switch (op.kind) {
        case K_RY_R:
          call = "qj::ry<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I, " + C + ");";
          g << "qj::g_ry<" << N << ", " << SA << ">(pr, pq, lr, lq)";
          break;
        case K_RX_R:
          call = "qj::rx<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I, " + C + ");";
          g << "qj::g_rx<" << N << ", " << SA << ">(pr, pq, lr, lq)";
          break;
        case K_RZ_R:
          call = "qj::rz<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I, " + C + ");";
          g << "qj::g_rz<" << N << ", " << SA << ">(pr, pq, lr, lq)";
          break;
        case K_H_R:
          call = "qj::hd<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I);";
          break;
        case K_X_R:
          call = "qj::swp<" + std::to_string(N) + ", " + std::to_string(SA) + ", 0>(%R, %I);";
          break;
        case K_RZ_T:
          call = "qj::rz_t<" + std::to_string(N) + ">(%R, %I, " + C + ", ((tb >> " + std::to_string(op.a) +
                 ") & 1u) ? T(-1) : T(1));";
          g << "((((tb >> " << (int)op.a << ") & 1u) ? A(-1) : A(1)) * qj::g_im<" << N << ">(pr, pq, lr, lq))";
          break;
        case K_CNOT_RR:
          call = "qj::swp<" + std::to_string(N) + ", " + std::to_string(SA) + ", " + std::to_string(SB) + ">(%R, %I);";
          break;
        case K_CNOT_RT:
          call = "qj::cnot_t<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I, ((tb >> " +
                 std::to_string(op.b) + ") & 1u) != 0u);";
          break;
        case K_CZ_RR:
          call = "qj::cz<" + std::to_string(N) + ", " + std::to_string(SA) + ", " + std::to_string(SB) + ">(%R, %I);";
          break;
        case K_CZ_RT:
          call = "qj::cz_t<" + std::to_string(N) + ", " + std::to_string(SA) + ">(%R, %I, ((tb >> " +
                 std::to_string(op.b) + ") & 1u) != 0u);";
          break;
        case K_CZ_TT:
          call = "if (((tb >> " + std::to_string(op.a) + ") & 1u) && ((tb >> " + std::to_string(op.b) +
                 ") & 1u)) qj::scal<" + std::to_string(N) + ">(%R, %I, T(-1));";
          break;
        case K_SCALE:
          call = "qj::scal<" + std::to_string(N) + ">(%R, %I, c.cf[" + std::to_string(li) + "]);";
          break;
      }
      if (pk) {   // packed backward: the same ops on (psi, lambda) pairs, tangent form only
        const std::string Ns = std::to_string(N), As = std::to_string(SA), Bs = std::to_string(SB);
        const std::string cf = "c.cf[" + std::to_string(li) + "]";
        const std::string tba = "((tb >> " + std::to_string(op.a) + ") & 1u)", tbb = "((tb >> " + std::to_string(op.b) + ") & 1u)";
        g.str("");
        switch (op.kind) {
          case K_RY_R: call = "qj::ry_p<" + Ns + ", " + As + ">(X, Y, " + cf + ");"; g << "qj::g_ry_p<" << N << ", " << SA << ">(X, Y)"; break;
          case K_RX_R: call = "qj::rx_p<" + Ns + ", " + As + ">(X, Y, " + cf + ");"; g << "qj::g_rx_p<" << N << ", " << SA << ">(X, Y)"; break;
          case K_RZ_R: call = "qj::rz_p<" + Ns + ", " + As + ">(X, Y, " + cf + ");"; g << "qj::g_rz_p<" << N << ", " << SA << ">(X, Y)"; break;
          case K_H_R: call = "qj::hd_p<" + Ns + ", " + As + ">(X, Y);"; break;
          case K_X_R: call = "qj::swp_p<" + Ns + ", " + As + ", 0>(X, Y);"; break;
          case K_RZ_T:
            call = "qj::rz_tp<" + Ns + ">(X, Y, " + cf + ", " + tba + " ? -1.f : 1.f);";
            g << "((" << tba << " ? -1.f : 1.f) * qj::g_im_p<" << N << ">(X, Y))";
            break;
          case K_CNOT_RR: call = "qj::swp_p<" + Ns + ", " + As + ", " + Bs + ">(X, Y);"; break;
          case K_CNOT_RT: call = "qj::cnot_tp<" + Ns + ", " + As + ">(X, Y, " + tbb + " != 0u);"; break;
          case K_CZ_RR: call = "qj::cz_p<" + Ns + ", " + As + ", " + Bs + ">(X, Y);"; break;
          case K_CZ_RT: call = "qj::cz_tp<" + Ns + ", " + As + ">(X, Y, " + tbb + " != 0u);"; break;
          case K_CZ_TT: call = "if (" + tba + " && " + tbb + ") qj::scal_p<" + Ns + ">(X, Y, -1.f);"; break;
          case K_SCALE: call = "qj::scal_p<" + Ns + ">(X, Y, " + cf + ");"; break;
        }
      }
      auto inst = [&](const char* rr, const char* ii) {
        std::string c2 = call;
        size_t p;
        while ((p = c2.find("%R")) != std::string::npos) c2.replace(p, 2, rr);
        while ((p = c2.find("%I")) != std::string::npos) c2.replace(p, 2, ii);
        return c2;
      };
      if (!bwd) {
        o << "      " << inst("re", "im") << "\n";
      } else {
        if (op.rot) emit_grad(op, g.str());
        if (pk) o << "      " << call << "\n";
        else o << "      " << inst("pr", "pq") << " " << inst("lr", "lq") << "\n";
      }
    };
    // A run of diagonal ops (tangent-form RZ: amplitude times 1 - i cs, cs = +-c by the qubit's bit; CZ:
    // sign flips) is one diagonal factor D per amplitude: the product of the run's register-bit RZ
    // factors for the amplitude's values of the used register bits (a table entry, per sample: see
    // DiagRun), times a thread-uniform part (RZ and CZ on thread bits) and the signs of register-thread
    // CZs; register-register CZs commute with the rest and are applied after.
    // Backward: conj(lambda) psi of every amplitude only gains the real factor 1 + c^2 from each RZ
    // undone, so all of the run's RZ gradients come from sums of w = Im(conj(lambda) psi) taken once at
    // the start, each times the product rho of 1 + c^2 of the run's RZs undone before it.
    auto emit_diag_run = [&](const DiagRun& dr) {
      const std::vector<int>& run = dr.ops;
      const std::vector<int>& used = dr.used;
      std::vector<int> wused;  // register bits with an RZ gradient (backward)
      bool has_t = false;      // a thread-uniform factor
      std::vector<std::pair<int, int>> czrt;   // (index in used, thread bit) of register-thread CZs
      for (int oi : run) {
        const DevOp& op = s.ops[oi];
        if (op.kind == K_RZ_R && std::find(wused.begin(), wused.end(), (int)op.a) == wused.end()) wused.push_back(op.a);
        if (op.kind == K_RZ_T || op.kind == K_CZ_TT) has_t = true;
        if (op.kind == K_CZ_RT)
          czrt.push_back({(int)(std::find(used.begin(), used.end(), (int)op.a) - used.begin()), (int)op.b});
      }
      const bool tab = dr.tab;
      auto uname = [&](int r, int b, char part) { return "u" + std::to_string(r) + "_" + std::to_string(b) + part; };
      o << "      { // diagonal run of " << run.size() << " ops\n";
      if (has_t || !tab) o << "        T tr = T(1), ti = T(0);\n";
      if (!tab)
        for (int r : used)
          o << "        T " << uname(r, 0, 'r') << " = T(1), " << uname(r, 0, 'i') << " = T(0), " << uname(r, 1, 'r')
            << " = T(1), " << uname(r, 1, 'i') << " = T(0);\n";
      if (bwd) {
        o << "        A wt = A(0);";
        for (size_t k2 = 0; k2 < wused.size(); k2++) o << " A w" << wused[k2] << " = A(0);";
        o << "\n";
        for (int i = 0; i < N; i++) {
          o << "        { const A w = (A)" << LR(i) << " * (A)" << PQ(i) << " - (A)" << LQ(i) << " * (A)" << PR(i) << "; wt += w;";
          for (int r : wused) o << " w" << r << ((i >> r) & 1 ? " -= w;" : " += w;");
          o << " }\n";
        }
        o << "        T rho = T(1);\n";
      }
      std::vector<const DevOp*> czrr;
      for (int oi : run) {
        const DevOp& op = s.ops[oi];
        const std::string cf = "c.cf[" + std::to_string(oi - d.op0) + "]";
        switch (op.kind) {
          case K_RZ_R:
            if (bwd) {
              emit_grad(op, "(A)w" + std::to_string(op.a) + " * (A)rho");
              o << "        rho *= T(1) + " << cf << " * " << cf << ";\n";
            }
            if (!tab)
              o << "        { const T cc = " << cf << "; qj::cmul(" << uname(op.a, 0, 'r') << ", " << uname(op.a, 0, 'i')
                << ", T(1), -cc); qj::cmul(" << uname(op.a, 1, 'r') << ", " << uname(op.a, 1, 'i') << ", T(1), cc); }\n";
            break;
          case K_RZ_T: {
            const std::string sg = "(((tb >> " + std::to_string(op.a) + ") & 1u) ? T(-1) : T(1))";
            if (bwd) {
              emit_grad(op, "(A)" + sg + " * (A)wt * (A)rho");
              o << "        rho *= T(1) + " << cf << " * " << cf << ";\n";
            }
            o << "        { const T cc = " << sg << " * " << cf << "; qj::cmul(tr, ti, T(1), -cc); }\n";
            break;
          }
          case K_CZ_TT:
            o << "        if (((tb >> " << (int)op.a << ") & 1u) && ((tb >> " << (int)op.b << ") & 1u)) { tr = -tr; ti = -ti; }\n";
            break;
          case K_CZ_RT:   // with a table: the entry's sign below
            if (!tab)
              o << "        if ((tb >> " << (int)op.b << ") & 1u) { " << uname(op.a, 1, 'r') << " = -" << uname(op.a, 1, 'r')
                << "; " << uname(op.a, 1, 'i') << " = -" << uname(op.a, 1, 'i') << "; }\n";
            break;
          default:   // K_CZ_RR
            czrr.push_back(&op);
            break;
        }
      }
      // every amplitude times its D: one table entry per value of the used bits (compressed index)
      const int nu = (int)used.size();
      if (!tab) {   // D over the used bits by a butterfly from the thread-uniform part
        o << "        T dr[" << (1 << nu) << "], di[" << (1 << nu) << "];\n        dr[0] = tr; di[0] = ti;\n";
        for (int k2 = 0; k2 < nu; k2++)
          o << "        for (int j = 0; j < " << (1 << k2) << "; j++) { dr[j + " << (1 << k2) << "] = dr[j]; di[j + " << (1 << k2)
            << "] = di[j]; qj::cmul(dr[j + " << (1 << k2) << "], di[j + " << (1 << k2) << "], " << uname(used[k2], 1, 'r') << ", "
            << uname(used[k2], 1, 'i') << "); qj::cmul(dr[j], di[j], " << uname(used[k2], 0, 'r') << ", " << uname(used[k2], 0, 'i')
            << "); }\n";
      }
      for (int idx = 0; idx < (1 << nu); idx++) {
        std::string flip;   // register-thread CZs whose register bit is set in this entry
        for (auto& zc : czrt)
          if ((idx >> zc.first) & 1) flip += std::string(flip.empty() ? "" : " ^ ") + "((tb >> " + std::to_string(zc.second) + ") & 1u)";
        const bool plain = !has_t && flip.empty();
        const int e0 = dr.off + dr.es * idx;
        o << "        {";
        if (!tab) {
          o << " const T fr = dr[" << idx << "], fi = di[" << idx << "];";
          if (pk) o << " const float2 fr2 = qj::f2(fr), fi2 = qj::f2(fi), fn2 = qj::f2(-fi);";
          o << "\n";
        } else if (pk && plain) {
          o << " const float4 f = *reinterpret_cast<const float4*>(c.tab + " << e0 << ");"
            << " const float2 fr2 = make_float2(f.x, f.y), fi2 = make_float2(f.z, f.w), fn2 = make_float2(-f.z, -f.w);\n";
        } else {
          o << " T fr, fi; qj::ldtab(c.tab + " << e0 << ", " << (dr.es == 4 ? 2 : 1) << ", fr, fi);";
          if (has_t) o << " qj::cmul(fr, fi, tr, ti);";
          if (!flip.empty()) o << " if (" << flip << ") { fr = -fr; fi = -fi; }";
          if (pk) o << " const float2 fr2 = qj::f2(fr), fi2 = qj::f2(fi), fn2 = qj::f2(-fi);";
          o << "\n";
        }
        for (int i = 0; i < N; i++) {
          int ci = 0;
          for (int k2 = 0; k2 < nu; k2++)
            if ((i >> used[k2]) & 1) ci |= 1 << k2;
          if (ci != idx) continue;
          if (!bwd) {
            o << "          qj::cmul(re[" << i << "], im[" << i << "], fr, fi);\n";
          } else if (pk) {
            o << "          { const float2 x = X[" << i << "], y = Y[" << i << "]; X[" << i << "] = qj::pfma(fn2, y, __fmul2_rn(fr2, x)); Y["
              << i << "] = qj::pfma(fi2, x, __fmul2_rn(fr2, y)); }\n";
          } else {
            o << "          qj::cmul(pr[" << i << "], pq[" << i << "], fr, fi); qj::cmul(lr[" << i << "], lq[" << i << "], fr, fi);\n";
          }
        }
        o << "        }\n";
      }
      for (const DevOp* op : czrr) {
        const std::string t = std::to_string(N) + ", " + std::to_string(1 << op->a) + ", " + std::to_string(1 << op->b);
        if (!bwd) o << "        qj::cz<" << t << ">(re, im);\n";
        else if (pk) o << "        qj::cz_p<" << t << ">(X, Y);\n";
        else o << "        qj::cz<" << t << ">(pr, pq); qj::cz<" << t << ">(lr, lq);\n";
      }
      o << "      }\n";
    };
    {
      const std::vector<std::pair<size_t, size_t>> rng = diag_ranges(s, order, bwd);
      size_t x = 0;
      for (auto& xy : rng) {
        for (; x < xy.first; x++) emit_op(order[x]);
        const DiagRun& dr = druns[run_i++];
        if (dr.ops != std::vector<int>(order.begin() + xy.first, order.begin() + xy.second)) {
          fprintf(stderr, "qsim: diagonal run tables out of step with the generated code\n");
          abort();
        }
        emit_diag_run(dr);
        x = xy.second;
      }
      for (; x < order.size(); x++) emit_op(order[x]);
    }
    // ---- prefix partials (backward of the first pass of a product-prefix plan; a.ppart set only there)
    if (bwd && last && prefix) {
      const int NT = Ph.n_tbits, NS = 2 * K + 1;
      o << "      if (a.ppart != nullptr) {\n"
        << "        const T* ph = reinterpret_cast<const T*>(a.phi) + c.b * a.n * 4;\n"
        << "        T wr[" << N << "], wi[" << N << "], fr[" << R << "][2], fi[" << R << "][2], Sr, Si, nr[" << R << "][2], ni["
        << R << "][2];\n";
      for (int i = 0; i < N; i++) o << "        wr[" << i << "] = " << LR(i) << "; wi[" << i << "] = -" << LQ(i) << ";\n";
      // a folded CNOT's target register holds the element with that bit flipped where the control is set:
      // its factor swaps its two values there (for the other qubits' contractions), and its own two
      // partials swap slots (swr)
      o << "        qj::u32 swr[" << R << "];\n";
      for (int r = 0; r < R; r++)
        o << "        { const qj::u32 sw = " << fold_swap(r) << "; swr[" << r << "] = sw; const T* f = ph + 4 * a.Q["
          << (int)Ph.rbit[r] << "]; fr[" << r << "][0] = f[2 * sw]; fi[" << r << "][0] = f[2 * sw + 1]; fr[" << r
          << "][1] = f[2 - 2 * sw]; fi[" << r << "][1] = f[3 - 2 * sw]; }\n";
      o << "        qj::prefix_contract<T, " << N << ", " << R << ">(wr, wi, fr, fi, Sr, Si, nr, ni);\n";
      o << "        T gr[" << std::max(NT, 1) << "], gi[" << std::max(NT, 1) << "], Ftr = T(1), Fti = T(0);\n";
      for (int jb = 0; jb < NT; jb++)
        o << "        { const T* f = ph + 4 * a.Q[" << (int)Ph.tbit[jb] << "] + 2 * ((tid >> " << jb << ") & 1u); gr[" << jb
          << "] = f[0]; gi[" << jb << "] = f[1]; qj::cmul(Ftr, Fti, f[0], f[1]); }\n";
      o << "        T* ws = reinterpret_cast<T*>(c.tile);\n        __syncthreads();\n";
      for (int r = 0; r < R; r++)
        for (int b = 0; b < 2; b++)
          o << "        { T vr = Ftr, vi = Fti; qj::cmul(vr, vi, qj::sel(swr[" << r << "], nr[" << r << "][" << (b ^ 1) << "], nr["
            << r << "][" << b << "]), qj::sel(swr[" << r << "], ni[" << r << "][" << (b ^ 1) << "], ni[" << r << "][" << b
            << "])); qj::prefix_put<T, " << NTHR << ", S_SELF::CTA>(vr, vi, "
            << 2 * (int)Ph.rbit[r] + b << ", ws, " << NS << ", tid); }\n";
      for (int jb = 0; jb < NT; jb++) {
        o << "        { T er = Sr, ei = Si;";
        for (int j2 = 0; j2 < NT; j2++)
          if (j2 != jb) o << " qj::cmul(er, ei, gr[" << j2 << "], gi[" << j2 << "]);";
        o << "\n          const bool hi = ((tid >> " << jb << ") & 1u) != 0u;\n"
          << "          qj::prefix_put<T, " << NTHR << ", S_SELF::CTA>(hi ? T(0) : er, hi ? T(0) : ei, " << 2 * (int)Ph.tbit[jb]
          << ", ws, " << NS << ", tid);\n"
          << "          qj::prefix_put<T, " << NTHR << ", S_SELF::CTA>(hi ? er : T(0), hi ? ei : T(0), " << 2 * (int)Ph.tbit[jb] + 1
          << ", ws, " << NS << ", tid); }\n";
      }
      o << "        { T vr = Ftr, vi = Fti; qj::cmul(vr, vi, Sr, Si); qj::prefix_put<T, " << NTHR << ", S_SELF::CTA>(vr, vi, "
        << 2 * K << ", ws, " << NS << ", tid); }\n"
        << "        __syncthreads();\n        qj::prefix_store<T, " << NTHR << ">(c, ws, " << NS << ", c.cf[" << d.n_ops << "]);\n"
        << "      }\n";
    }
    // ---- store
    if (last) {
      o << "      const T sc = c.cf[" << d.n_ops << "];\n";
      if (!bwd) {
        o << "      qj::scal<" << N << ">(re, im, sc);\n"
          << "      if (c.valid) {\n        T* out = reinterpret_cast<T*>(a.out);\n";
        for (int i = 0; i < N; i += 2)
          o << "        qj::stg_pair(out + 2 * " << goff("gs", "gs", i) << ", re[" << i << "], im[" << i << "], re[" << i + 1
            << "], im[" << i + 1 << "]);\n";
        o << "      }\n      if (a.zpart != nullptr) {\n        typedef typename qj::Acc<T>::t A;\n        A zt = 0, zs[" << R << "];\n";
        for (int r = 0; r < R; r++) o << "        zs[" << r << "] = 0;\n";
        for (int i = 0; i < N; i++) {
          o << "        { const A p = (A)re[" << i << "] * (A)re[" << i << "] + (A)im[" << i << "] * (A)im[" << i << "]; zt += p;";
          for (int r = 0; r < R; r++) o << " zs[" << r << "] " << (((i >> r) & 1) ? "-=" : "+=") << " p;";
          o << " }\n";
        }
        o << "        qj::z_reduce_regs<T, " << K << ", " << R << ", " << NTHR
          << ", S_SELF>(c.tile, zt, zs, a.zpart + (c.b * a.tps + c.t) * " << K + 1 << ", tid, c.valid);\n      }\n";
      } else if (prefix) {
        // the first pass's backward runs last and stores neither psi nor lambda (api: out = lam_out = nullptr)
        o << "      (void)sc;\n";
      } else {
        // psi is not stored when the previous pass restarts from a checkpoint (a.out == nullptr)
        o << fold_glob("gf", "gs");
        if (pk) o << "      qj::scal_p<" << N << ">(X, Y, sc);\n";
        o << "      if (a.out != nullptr && c.valid) {\n";
        if (!pk) o << "        qj::scal<" << N << ">(pr, pq, sc);\n";
        o << "        T* po = reinterpret_cast<T*>(a.out);\n";
        for (int i = 0; i < N; i += 2)
          o << "        qj::stg_pair(po + 2 * " << goff("gf", "gs", i) << ", " << PR(i) << ", " << PQ(i) << ", " << PR(i + 1)
            << ", " << PQ(i + 1) << ");\n";
        o << "      }\n      if (a.lam_out != nullptr && c.valid) {\n";
        if (!pk) o << "        qj::scal<" << N << ">(lr, lq, sc);\n";
        o << "        T* lo = reinterpret_cast<T*>(a.lam_out);\n";
        for (int i = 0; i < N; i += 2)
          o << "        qj::stg_pair(lo + 2 * " << goff("gf", "gs", i) << ", " << LR(i) << ", " << LQ(i) << ", " << LR(i + 1)
            << ", " << LQ(i + 1) << ");\n";
        o << "      }\n";
      }
    } else {
      const std::string fs = bwd ? fold_smem(Lo) : std::string();
      const char* ad = fs.empty() && disjoint(Lo, Ph) ? "true" : "false";
      o << "      __syncthreads();\n      const qj::u32 so = L" << lout << "(tb)" << fs << ";\n";
      for (int i = 0; i < N; i += 2) {
        const uint32_t cc = lay_eval(Lo, K, dep_of(Ph, i));
        if (!bwd) {
          o << "      qj::stpx<" << ad << ">(c.tile, so, " << cc << "u, re[" << i << "], im[" << i << "], re[" << i + 1 << "], im[" << i + 1 << "]);\n";
        } else if (pk) {
          o << "      qj::stppx<" << ad << ">(c.tile, so, " << cc << "u, X[" << i << "], Y[" << i << "], X[" << i + 1 << "], Y[" << i + 1 << "]);\n";
        } else {
          o << "      qj::stpx<" << ad << ">(c.tile, so, " << cc << "u, pr[" << i << "], pq[" << i << "], pr[" << i + 1 << "], pq[" << i + 1 << "]);\n";
          o << "      qj::stpx<" << ad << ">(c.tile2, so, " << cc << "u, lr[" << i << "], lq[" << i << "], lr[" << i + 1 << "], lq[" << i + 1 << "]);\n";
        }
      }
      o << "      __syncthreads();\n";
    }
    o << "    }\n";
  }
  o << "  }\n";
  return o.str();
}

// Default register bits per phase when a caller gives none: complex64 forward 5 (32 amplitudes per
// thread), backward 4 (psi and lambda); complex128 one less each. Threads per CTA = 2^(k - R) <= 256.
int fwd_R_for(int k, int dtype) { const int r = dtype == QSIM_C128 ? 4 : 5; return k < r ? k : r; }
int bwd_R_for(int k, int dtype) { const int r = dtype == QSIM_C128 ? 3 : 4; return k < r ? k : r; }
// Largest tile of a single-circuit plan: 2^13 complex64 amplitudes (256 threads of 2^5 each; the
// backward's psi and lambda tiles take 128 KiB of shared memory, one CTA per SM), 2^11 complex128.
// The default is one less for complex64 (the autotuner measures 11, 12 and 13); multi-circuit queue
// kernels take at most 2^11 / 2^10 (every pass structure of a direction shares their CTA size).
int max_k_for(int dtype) { return dtype == QSIM_C128 ? 11 : 13; }
int default_k_for(int dtype) { return dtype == QSIM_C128 ? 11 : 12; }
int multi_max_k_for(int dtype) { return dtype == QSIM_C128 ? 10 : 11; }

// Shared-memory bytes of one tile group; mirrors FwdGroupSmem / BwdGroupSmem in jit_device.cuh.
int single_cta(const DevPass& d) { return d.k - d.R < 5 ? 32 : 0; }

size_t single_smem_bytes(const Schedule& s, const DevPass& d, bool bwd) {
  const int cta = single_cta(d);
  const size_t groups = cta > 0 ? (size_t)cta >> (d.k - d.R) : 1;
  return groups * jit_smem_bytes(s, d, bwd, cta);
}

size_t jit_smem_bytes(const Schedule& s, const DevPass& d, bool bwd, int cta) {
  const int dtype = s.dtype;
  const size_t sc = dtype == QSIM_C128 ? 8 : 4, tile = (2 * sc) << d.k;
  const size_t no = (size_t)d.n_ops + 1;   // op coefficients + the pass scale
  const size_t tab = (size_t)diag_table_units(s, d, bwd) * sc;
  if (!bwd) return (tile + tab + no * sc + no + 15) & ~(size_t)15;
  const size_t nthr = (size_t)1 << (d.k - d.R);
  const size_t ng = d.n_gslots > 0 ? d.n_gslots : 1;
  const size_t red = 2 * tile;
  const size_t parts = ng * (nthr >> grad_level(d, dtype, cta, s.max_regs, tab));
  const size_t gq = (red + parts * sc + 15) & ~(size_t)15;
  const size_t tb = (gq + (d.k + 2) * 8 + 15) & ~(size_t)15;
  const size_t cf = tb + tab;
  const size_t fm = cf + no * sc;
  return (fm + no + 15) & ~(size_t)15;
}

// One NVRTC unit per distinct kernel: name -> source (device header + Spec + entry point).
static void jit_units(const Schedule& s, std::vector<std::string>& fnames, std::vector<std::string>& bnames,
                      std::map<std::string, std::string>& units) {
  const char* T = s.dtype == QSIM_C128 ? "double" : "float";
  fnames.clear();
  bnames.clear();
  for (auto& pp : s.passes) {
    for (int dir = 0; dir < 2; dir++) {
      const DevPass& d = dir == 0 ? pp.dev : pp.devb;
      const bool bwd = dir == 1;
      const int K = d.k, R = d.R, NTHR = 1 << (K - R);
      const int cta = single_cta(d), CTA = cta > 0 ? cta : NTHR;
      std::string body = gen_spec_body(s, d, bwd, cta, s.has_prefix && &pp == &s.passes[0]);
      // register cap: at least this many CTAs per SM (65536 registers each)
      const int minb = s.max_regs > 0 ? std::max(1, 65536 / (CTA * s.max_regs)) : 0;
      std::string key = std::string(T) + "|" + std::to_string(K) + "|" + std::to_string(R) + "|" +
                        std::to_string(minb) + "|" + body;
      std::string name = std::string(bwd ? "qb_" : "qf_") + hex64(fnv1a(key));
      if (!units.count(name)) {
        std::ostringstream u;
        std::string b2 = body;
        for (size_t p; (p = b2.find("S_SELF")) != std::string::npos;) b2.replace(p, 6, "S_" + name);
        u << "struct S_" << name << " {\n" << b2 << "};\n";
        u << "extern \"C\" __global__ void __launch_bounds__(" << CTA;
        if (minb > 0) u << ", " << minb;
        u << ") " << name << "(const qj::Args a) {";
        if (cta == 0) {
          u << " qj::" << (bwd ? "bwd_pass" : "fwd_pass") << "<" << T << ", " << K << ", " << R << ", " << NTHR << ", S_"
            << name << ">(a); }\n";
        } else {   // CTA / NTHR tiles per CTA, each group of NTHR threads on its own tile and shared memory
          u << "\n  extern __shared__ __align__(16) unsigned char smem[];\n"
            << "  constexpr int NTHR = " << NTHR << ", G = " << CTA / NTHR << ";\n"
            << "  const unsigned g = threadIdx.x / NTHR, tid = threadIdx.x % NTHR;\n"
            << "  const long long t0 = (long long)blockIdx.x * G, ti = t0 + g;\n"
            << "  const bool valid = ti < a.ntiles;\n";
          if (!bwd)
            u << "  constexpr int GB = qj::FwdGroupSmem<" << T << ", " << K << ", S_" << name << "::NOPS, S_" << name
              << "::NTAB>::BYTES;\n  qj::fwd_tile<" << T << ", " << K << ", " << R << ", NTHR, S_" << name
              << ">(a, valid ? ti : t0, valid, tid, smem + (size_t)g * GB);\n}\n";
          else
            u << "  constexpr int GB = qj::BwdGroupSmem<" << T << ", " << K << ", " << R << ", NTHR, S_" << name << "::NOPS, S_"
              << name << "::NGS, S_" << name << "::GS, S_" << name << "::NTAB>::BYTES;\n  qj::bwd_tile<" << T << ", " << K << ", "
              << R << ", NTHR, S_" << name << ">(a, valid ? ti : t0, valid, tid, smem + (size_t)g * GB);\n}\n";
        }
        units[name] = u.str();
      }
      (bwd ? bnames : fnames).push_back(name);
    }
  }
}

std::string jit_generate(const Schedule& s, std::vector<std::string>& fnames, std::vector<std::string>& bnames) {
  std::map<std::string, std::string> units;
  jit_units(s, fnames, bnames, units);
  std::ostringstream prog;
  prog << kJitDeviceSource << "\n";
  for (auto& kv : units) prog << "// ---- " << kv.first << "\n" << kv.second;
  return prog.str();
}

static int nvrtc_compile_unit(const std::string& src, std::string& cubin, std::string& err, bool rdc = false) {
  Nvrtc& nv = nvrtc();
  if (!nv.h) {
    err = nv.error;
    return QSIM_ERR_UNSUPPORTED;
  }
  nvrtcProgram_t prog = nullptr;
  if (nv.create(&prog, src.c_str(), "qsim_pass.cu", 0, nullptr, nullptr) != 0) {
    err = "nvrtcCreateProgram failed";
    return QSIM_ERR_UNSUPPORTED;
  }
  // relocatable pass functions are linked into one queue kernel whose register count is the maximum
  // over them: cap them so that four 128-thread CTAs fit on an SM
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--fmad=true", "-rdc=true",
                        "--maxrregcount=128"};
  const int rc = nv.compile(prog, rdc ? 6 : 4, opts);
  size_t ls = 0;
  nv.log_size(prog, &ls);
  std::string log(ls, '\0');
  if (ls) nv.log(prog, &log[0]);
  if (rc != 0) {
    nv.destroy(&prog);
    err = "NVRTC compilation of a pass kernel failed:\n" + log.substr(0, 6000);
    return QSIM_ERR_UNSUPPORTED;
  }
  size_t cs = 0;
  nv.cubin_size(prog, &cs);
  cubin.resize(cs);
  nv.cubin(prog, &cubin[0]);
  nv.destroy(&prog);
  return QSIM_OK;
}

int jit_compile(const Schedule& s, std::map<std::string, std::string>& cubins, std::vector<std::string>& fn,
                std::vector<std::string>& bn, std::string& err) {
  std::map<std::string, std::string> units;
  jit_units(s, fn, bn, units);
  Nvrtc& nv = nvrtc();
  int maj = 0, min = 0;
  if (nv.h) nv.version(&maj, &min);
  const std::string tag = "_sm103a_" + std::to_string(maj) + "." + std::to_string(min) + "_" +
                          hex64(fnv1a(kJitDeviceSource)).substr(0, 8);
  const std::string dir = cache_dir();
  std::vector<std::string> todo;
  for (auto& kv : units) {
    std::string bin;
    if (read_file(dir + "/" + kv.first + tag + ".cubin", bin)) cubins[kv.first] = bin;
    else todo.push_back(kv.first);
  }
  if (todo.empty()) return QSIM_OK;
  std::vector<std::string> bins(todo.size()), errs(todo.size());
  std::vector<int> rcs(todo.size(), 0);
  std::atomic<size_t> next{0};
  auto worker = [&]() {
    for (size_t i = next++; i < todo.size(); i = next++) {
      const std::string src = std::string(kJitDeviceSource) + "\n" + units[todo[i]];
      rcs[i] = nvrtc_compile_unit(src, bins[i], errs[i]);
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 4;
  nt = std::min<unsigned>(nt, (unsigned)todo.size());
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; t++) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (size_t i = 0; i < todo.size(); i++) {
    if (rcs[i]) {
      err = errs[i];
      return rcs[i];
    }
    cubins[todo[i]] = bins[i];
    write_file_atomic(dir, dir + "/" + todo[i] + tag + ".cubin", bins[i]);
  }
  return QSIM_OK;
}

int jit_build(const Schedule& s, JitPlan& jp, std::string& err) {
  std::vector<std::string> fn, bn;
  std::map<std::string, std::string> cubins;
  int rc = jit_compile(s, cubins, fn, bn, err);
  if (rc) return rc;
  std::map<std::string, cudaKernel_t> loaded;
  for (auto& kv : cubins) {
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, kv.second.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
      err = std::string("loading the pass kernels: ") + cudaGetErrorString(e);
      return QSIM_ERR_CUDA;
    }
    jp.libs.push_back(lib);
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, lib, kv.first.c_str());
    if (e != cudaSuccess) {
      err = "kernel " + kv.first + " missing: " + cudaGetErrorString(e);
      return QSIM_ERR_CUDA;
    }
    loaded[kv.first] = k;
  }
  jp.fwd.resize(fn.size());
  jp.bwd.resize(bn.size());
  for (int dir = 0; dir < 2; dir++) {
    auto& names = dir == 0 ? fn : bn;
    auto& ks = dir == 0 ? jp.fwd : jp.bwd;
    for (size_t p = 0; p < names.size(); p++) {
      const DevPass& d = dir == 0 ? s.passes[p].dev : s.passes[p].devb;
      cudaKernel_t k = loaded[names[p]];
      ks[p].fn = reinterpret_cast<void*>(k);
      ks[p].smem = single_smem_bytes(s, d, dir == 1);
      ks[p].nthr = single_cta(d) > 0 ? single_cta(d) : 1 << (d.k - d.R);
      ks[p].groups = single_cta(d) > 0 ? single_cta(d) >> (d.k - d.R) : 1;
      if (ks[p].smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks[p].smem);
        if (e != cudaSuccess) {
          err = std::string("shared memory attribute: ") + cudaGetErrorString(e);
          return QSIM_ERR_CUDA;
        }
      }
    }
  }
  return QSIM_OK;
}

// ------------------------------------------------------------------ multi-circuit queue kernels
static std::string multi_unit(const Schedule& s, const DevPass& d, bool bwd, int cta, std::string& name) {
  const char* T = s.dtype == QSIM_C128 ? "double" : "float";
  const int K = d.k, R = d.R, NTHR = 1 << (K - R);
  std::string body = gen_spec_body(s, d, bwd, cta);
  std::string key = std::string(T) + "|" + std::to_string(K) + "|" + std::to_string(R) + "|" + body;
  name = std::string(bwd ? "qsb_" : "qsf_") + hex64(fnv1a(key));
  std::ostringstream u;
  for (size_t p; (p = body.find("S_SELF")) != std::string::npos;) body.replace(p, 6, "S_" + name);
  u << "struct S_" << name << " {\n" << body << "};\n";
  u << "extern \"C\" __device__ void " << name
    << "(const qj::Args* a, long long tile0, long long ntiles, unsigned char* smem) {\n"
    << "  constexpr int NTHR = " << NTHR << ";\n"
    << "  const unsigned g = threadIdx.x / NTHR, tid = threadIdx.x % NTHR;\n"
    << "  const long long ti = tile0 + g;\n"
    << "  const bool valid = ti < ntiles;\n";
  if (!bwd)
    u << "  constexpr int GB = qj::FwdGroupSmem<" << T << ", " << K << ", S_" << name << "::NOPS, S_" << name << "::NTAB>::BYTES;\n"
      << "  qj::fwd_tile<" << T << ", " << K << ", " << R << ", NTHR, S_" << name
      << ">(*a, valid ? ti : tile0, valid, tid, smem + (size_t)g * GB);\n";
  else
    u << "  constexpr int GB = qj::BwdGroupSmem<" << T << ", " << K << ", " << R << ", NTHR, S_" << name << "::NOPS, S_"
      << name << "::NGS, S_" << name << "::GS, S_" << name << "::NTAB>::BYTES;\n"
      << "  qj::bwd_tile<" << T << ", " << K << ", " << R << ", NTHR, S_" << name
      << ">(*a, valid ? ti : tile0, valid, tid, smem + (size_t)g * GB);\n";
  u << "}\n";
  return u.str();
}

static std::string queue_kernel_unit(const std::vector<std::string>& kinds, bool bwd, int cta, std::string& kname) {
  std::ostringstream u;
  std::string all;
  for (auto& k : kinds) all += k + ",";
  kname = std::string(bwd ? "qsim_queue_bwd_" : "qsim_queue_fwd_") + hex64(fnv1a(all + std::to_string(cta)));
  for (auto& k : kinds)
    u << "extern \"C\" __device__ void " << k << "(const qj::Args*, long long, long long, unsigned char*);\n";
  u << "extern \"C\" __global__ void __launch_bounds__(" << cta << ") " << kname << "(const qj::MultiArgs m) {\n"
    << "  extern __shared__ __align__(16) unsigned char smem[];\n"
    << "  __shared__ long long s_item;\n"
    << "  __shared__ int s_run;\n"
    << "  for (;;) {\n"
    << "    __syncthreads();\n"
    << "    if (threadIdx.x == 0) s_item = (long long)atomicAdd(m.head, 1ull);\n"
    << "    __syncthreads();\n"
    << "    const long long it = s_item;\n"
    << "    if (it >= m.n_items) break;\n"
    << "    const qj::Item item = m.items[it];\n"
    << "    if (threadIdx.x == 0) s_run = qj::wait_dependency(m, item) ? 1 : 0;\n"
    << "    __syncthreads();\n"
    << "    if (s_run) {\n"
    << "      switch (item.kind) {\n";
  for (size_t i = 0; i < kinds.size(); i++)
    u << "        case " << i << ": " << kinds[i] << "(m.args + item.arg, item.tile0, item.ntiles, smem); break;\n";
  u << "        default: break;\n"
    << "      }\n"
    << "    }\n"
    << "    __syncthreads();\n"
    << "    if (threadIdx.x == 0) {\n"
    << "      __threadfence();\n"
    << "      if (it != m.withhold) atomicAdd(m.counters + item.done, 1);\n"
    << "    }\n"
    << "  }\n"
    << "}\n";
  return u.str();
}

int jit_build_multi(const std::vector<const Schedule*>& scheds, int cta_f, int cta_b, JitMulti& jm,
                    std::string& err) {
  JitLinker& jl = jitlink();
  Nvrtc& nv = nvrtc();
  if (!jl.h) {
    err = jl.error;
    return QSIM_ERR_UNSUPPORTED;
  }
  int maj = 0, min = 0;
  if (nv.h) nv.version(&maj, &min);
  const std::string tag = "_rdc_r128_sm103a_" + std::to_string(maj) + "." + std::to_string(min) + "_" +
                          hex64(fnv1a(kJitDeviceSource)).substr(0, 8);
  const std::string dir = cache_dir();
  std::map<std::string, std::string> units[2];   // name -> source (per direction)
  std::vector<std::string> kinds[2];
  std::map<std::string, int> kind_id[2];
  jm.kind.assign(scheds.size(), {});
  jm.smem_group[0].clear();
  jm.smem_group[1].clear();
  size_t max_smem[2] = {0, 0};
  for (size_t c = 0; c < scheds.size(); c++) {
    if (!scheds[c]) continue;   // a circuit the queue does not run
    const Schedule& s = *scheds[c];
    jm.kind[c].resize(2 * s.passes.size());
    for (size_t p = 0; p < s.passes.size(); p++) {
      for (int dir = 0; dir < 2; dir++) {
        const DevPass& d = dir == 0 ? s.passes[p].dev : s.passes[p].devb;
        const int cta = dir == 0 ? cta_f : cta_b;
        std::string name;
        std::string src = multi_unit(s, d, dir == 1, cta, name);
        if (!kind_id[dir].count(name)) {
          kind_id[dir][name] = (int)kinds[dir].size();
          kinds[dir].push_back(name);
          units[dir][name] = src;
        }
        jm.kind[c][2 * p + dir] = kind_id[dir][name];
        const int nthr = 1 << (d.k - d.R);
        const size_t groups = (size_t)cta / nthr;
        max_smem[dir] = std::max(max_smem[dir], groups * jit_smem_bytes(s, d, dir == 1, cta));
      }
    }
  }
  // one queue kernel links every distinct pass structure of its direction; keep that link to a size
  // known to work (a few hundred functions of straight-line code make a very large program)
  constexpr size_t kMaxKinds = 192;
  for (int dir = 0; dir < 2; dir++)
    if (kinds[dir].size() > kMaxKinds) {
      err = "multi-circuit plan has " + std::to_string(kinds[dir].size()) +
            " distinct pass structures in one direction (at most " + std::to_string(kMaxKinds) +
            " per queue kernel): split the circuit list into several plans";
      return QSIM_ERR_UNSUPPORTED;
    }
  // compile every unit (relocatable) in parallel, cached
  std::vector<std::pair<std::string, std::string>> todo;   // name, source
  std::map<std::string, std::string> bins;
  std::string qnames[2];
  for (int dir = 0; dir < 2; dir++) {
    for (auto& kv : units[dir]) todo.push_back(kv);
    std::string qn;
    std::string qsrc = queue_kernel_unit(kinds[dir], dir == 1, dir == 0 ? cta_f : cta_b, qn);
    qnames[dir] = qn;
    todo.push_back({qn, qsrc});
  }
  std::vector<std::string> need;
  for (auto& t : todo) {
    std::string b;
    if (read_file(dir + "/" + t.first + tag + ".cubin", b)) bins[t.first] = b;
    else need.push_back(t.first);
  }
  std::map<std::string, std::string> srcs(todo.begin(), todo.end());
  if (!need.empty()) {
    std::vector<std::string> out(need.size()), errs(need.size());
    std::vector<int> rcs(need.size(), 0);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      for (size_t i = next++; i < need.size(); i = next++)
        rcs[i] = nvrtc_compile_unit(std::string(kJitDeviceSource) + "\n" + srcs[need[i]], out[i], errs[i], true);
    };
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 4;
    nt = std::min<unsigned>(nt, (unsigned)need.size());
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; t++) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    for (size_t i = 0; i < need.size(); i++) {
      if (rcs[i]) {
        err = errs[i];
        return rcs[i];
      }
      bins[need[i]] = out[i];
      write_file_atomic(dir, dir + "/" + need[i] + tag + ".cubin", out[i]);
    }
  }
  // link each direction's queue kernel with its pass functions
  for (int dir = 0; dir < 2; dir++) {
    nvJitLinkHandle_t h = nullptr;
    const char* lopts[] = {"-arch=sm_103a"};
    if (jl.create(&h, 1, lopts) != 0) {
      err = "nvJitLinkCreate failed";
      return QSIM_ERR_UNSUPPORTED;
    }
    bool ok = true;
    for (auto& k : kinds[dir]) ok = ok && jl.add_data(h, 1 /*CUBIN*/, bins[k].data(), bins[k].size(), k.c_str()) == 0;
    ok = ok && jl.add_data(h, 1, bins[qnames[dir]].data(), bins[qnames[dir]].size(), qnames[dir].c_str()) == 0;
    ok = ok && jl.complete(h) == 0;
    if (!ok) {
      size_t es = 0;
      jl.err_size(h, &es);
      std::string log(es, '\0');
      if (es) jl.err_log(h, &log[0]);
      jl.destroy(&h);
      err = "nvJitLink failed: " + log.substr(0, 4000);
      return QSIM_ERR_UNSUPPORTED;
    }
    size_t cs = 0;
    jl.cubin_size(h, &cs);
    std::string linked(cs, '\0');
    jl.cubin(h, &linked[0]);
    jl.destroy(&h);
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, linked.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
      err = std::string("loading the queue kernel: ") + cudaGetErrorString(e);
      return QSIM_ERR_CUDA;
    }
    jm.libs.push_back(lib);
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, lib, qnames[dir].c_str());
    if (e != cudaSuccess) {
      err = std::string("queue kernel missing: ") + cudaGetErrorString(e);
      return QSIM_ERR_CUDA;
    }
    JitKernel& jk = dir == 0 ? jm.fwd : jm.bwd;
    jk.fn = reinterpret_cast<void*>(k);
    jk.nthr = dir == 0 ? cta_f : cta_b;
    jk.smem = max_smem[dir];
    if (jk.smem > 48 * 1024) {
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)jk.smem);
      if (e != cudaSuccess) {
        err = std::string("queue kernel shared memory (") + std::to_string(jk.smem) + " B): " + cudaGetErrorString(e);
        return QSIM_ERR_UNSUPPORTED;
      }
    }
    int per_sm = 0, devi = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(k), jk.nthr, jk.smem);
    if (e != cudaSuccess || per_sm < 1) {
      err = "queue kernel cannot be resident";
      return QSIM_ERR_UNSUPPORTED;
    }
    cudaGetDevice(&devi);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devi);
    jk.max_blocks = (int64_t)per_sm * sms;   // persistent grid: every block resident at once
    jk.per_sm = per_sm;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k)) == cudaSuccess) jk.regs = fa.numRegs;
  }
  jm.n_kinds[0] = (int)kinds[0].size();
  jm.n_kinds[1] = (int)kinds[1].size();
  return QSIM_OK;
}

void jit_free_multi(JitMulti& jm) {
  for (auto l : jm.libs) cudaLibraryUnload(l);
  jm.libs.clear();
}

void jit_free(JitPlan& jp) {
  for (auto l : jp.libs) cudaLibraryUnload(l);
  jp.libs.clear();
  jp.fwd.clear();
  jp.bwd.clear();
}

cudaError_t jit_launch(const JitKernel& k, int64_t blocks, const JitArgs& a, cudaStream_t st) {
  if (blocks <= 0 || blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  JitArgs la = a;
  la.ntiles = blocks;   // tiles; a CTA takes k.groups of them
  const int64_t grid = (blocks + k.groups - 1) / k.groups;
  void* args[] = {&la};
  cudaError_t e = cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3((unsigned)k.nthr), args, k.smem, st);
  if (e == cudaSuccess) g_kernel_launches++;
  return e;
}

}  // namespace qsim
