// C ABI: plan objects, workspace management and the launch sequences of forward / backward.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "jit.hpp"
#include "launch.hpp"
#include "planner.hpp"

using namespace qsim;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return QSIM_ERR_CUDA;
}

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& v) {
  *dptr = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dptr), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}
}  // namespace

namespace qsim {
void set_last_error(const std::string& s) { g_err = s; }
}  // namespace qsim

struct qsim_plan_s {
  Schedule s;
  qsim_plan_opts opts{};
  int el = 8, sc = 4;
  // device copy of the schedule
  bool uploaded = false;
  int32_t* d_exec_gates_b = nullptr;
  int32_t* d_exec_begin_b = nullptr;
  std::vector<int32_t> h_exec_begin, h_exec_begin_b;   // first op of every pass in the packed coefficients
  JitPlan jit;
  int32_t* d_gate_type = nullptr;
  int32_t* d_gate_param = nullptr;
  int32_t* d_gate_q0 = nullptr;   // target qubit of every gate (Pauli frame walk)
  int32_t* d_gate_q1 = nullptr;   // control qubit (-1 for single-qubit gates)
  int32_t* d_exec_gates = nullptr;
  int32_t* d_exec_begin = nullptr;
  int32_t* d_occ_gate = nullptr;
  int64_t* d_occ_slot = nullptr;
  int32_t *d_p_ptr = nullptr, *d_p_occ = nullptr, *d_i_ptr = nullptr, *d_i_occ = nullptr;
  uint8_t* d_Qnl_last = nullptr;
  int n_occ = 0;
  // product-state prefix: CSR over qubits of the prefix gates, their gradient occurrences, and the first
  // pass's tile / tile-index qubits
  int32_t *d_pfx_begin = nullptr, *d_pfx_gate = nullptr, *d_pfx_occ = nullptr;
  uint8_t* d_Qnl_first = nullptr;
  void* phi = nullptr;         // [B][n][4] prefix states (state precision)
  double* ppart = nullptr;     // [B][tps of pass 0][2k + 1][2] backward partials of the first pass
  // a prefix plan given an initial state runs this plan (same gates and options, no prefix) instead
  qsim_plan_s* alt = nullptr;
  bool via_alt = false;
  // batch workspace
  int B_cap = -1;
  int n_segments = 1;
  std::vector<int> seg_begin;   // pass index where each checkpoint segment starts (+ end sentinel)
  void* coef = nullptr;
  uint8_t* form = nullptr;
  void* cfp_f = nullptr;     // packed per-pass op coefficients [exec_begin[p] * B + b * n_ops + i] (forward)
  uint8_t* fmp_f = nullptr;
  void* cfp_b = nullptr;     // the same for the backward op lists, coefficients negated
  uint8_t* fmp_b = nullptr;
  void* scale_f = nullptr;
  void* scale_b = nullptr;
  double* gm = nullptr;
  double* zpart = nullptr;
  double* gpart = nullptr;
  double* G = nullptr;
  void* W = nullptr;
  void* Lam = nullptr;
  // Pauli frame (pauli_frame plans): the last pass's output in the stored representation F^dag (true
  // state), the frame signs and final frames, and the loss weights with the frame's signs
  void* S_end = nullptr;
  int8_t* sigma = nullptr;
  uint64_t* frame_x = nullptr;
  uint64_t* frame_z = nullptr;
  int32_t* frame_k = nullptr;
  double* gsign = nullptr;
  std::vector<void*> ckpt;
  int64_t ws_bytes = 0;
  // saved forward context
  bool has_fwd = false;
  const void* params = nullptr;
  const void* inputs = nullptr;
  void* states = nullptr;
  int B = 0;
  cudaStream_t last_stream = nullptr;
  // optional per-launch event timing (a log of launches; read_profile sums them per pass)
  int prof_depth = 0;            // 0 = off; else number of forward + backward calls to log
  bool profiling = false;
  struct ProfRec {
    int dir, pass;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_log;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  int64_t n_fwd_calls = 0, n_bwd_calls = 0;

  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
  bool calls_left(int dir) const {
    return profiling && (dir == 0 ? n_fwd_calls : n_bwd_calls) < prof_depth;
  }
  // record an event before a launch; returns the log index (or -1)
  int prof_begin(int dir, int pass, cudaStream_t st) {
    if (!calls_left(dir)) return -1;
    cudaEvent_t a = next_event(), b = next_event();
    if (!a || !b) return -1;
    cudaEventRecord(a, st);
    prof_log.push_back({dir, pass, a, b});
    return (int)prof_log.size() - 1;
  }
  void prof_end(int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(prof_log[idx].b, st);
  }
  void destroy_events() {
    for (auto e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    prof_log.clear();
    ev_used = 0;
  }

  int P() const { return (int)s.passes.size(); }
  // samples per launch group (all passes run over one group before the next); 0 = whole batch
  int group_size(int B_) const {
    if (opts.sample_block > 0 && s.mode == QSIM_FUSED) return std::min(opts.sample_block, B_);
    return B_ > 0 ? B_ : 1;
  }
  int64_t tps() const {
    return s.mode == QSIM_PER_GATE ? pg_blocks_per_sample(s.n) : s.passes.empty() ? 1 : s.passes[0].dev.tiles_per_sample;
  }
  int64_t state_bytes(int B_) const { return (int64_t)B_ * ((int64_t)1 << s.n) * el; }

  void free_ws() {
    void* ptrs[] = {coef, form, cfp_f, fmp_f, cfp_b, fmp_b, scale_f, scale_b, gm, zpart, gpart, G, W, Lam,
                    S_end, sigma, frame_x, frame_z, frame_k, gsign, phi, ppart};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    S_end = nullptr;
    phi = nullptr;
    ppart = nullptr;
    sigma = nullptr;
    frame_x = frame_z = nullptr;
    frame_k = nullptr;
    gsign = nullptr;
    for (void* p : ckpt)
      if (p) cudaFree(p);
    coef = cfp_f = cfp_b = nullptr;
    form = fmp_f = fmp_b = nullptr;
    scale_f = scale_b = nullptr;
    gm = zpart = gpart = G = nullptr;
    W = Lam = nullptr;
    ckpt.clear();
    ws_bytes = 0;
    B_cap = -1;
  }
  void free_all() {
    free_ws();
    destroy_events();
    void* ptrs[] = {d_gate_type, d_gate_param, d_gate_q0, d_gate_q1, d_exec_gates, d_exec_begin, d_exec_gates_b,
                    d_exec_begin_b, d_occ_gate, d_occ_slot, d_p_ptr, d_p_occ, d_i_ptr, d_i_occ, d_Qnl_last,
                    d_pfx_begin, d_pfx_gate, d_pfx_occ, d_Qnl_first};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    jit_free(jit);
    uploaded = false;
  }

  int upload_schedule() {
    if (uploaded) return QSIM_OK;
    cudaError_t e = cudaSuccess;
    std::vector<int32_t> gtype, gparam, gq0, gq1, exec, exec_begin, exec_b, exec_begin_b;
    for (auto& g : s.gates) {
      gtype.push_back(g.type);
      gparam.push_back(g.param);
      gq0.push_back(g.t0);
      gq1.push_back(g.c0);
    }
    for (auto& pp : s.passes) {
      exec_begin.push_back((int32_t)exec.size());
      exec_begin_b.push_back((int32_t)exec_b.size());
      if (s.mode == QSIM_PER_GATE) {
        exec.push_back(pp.gates[0]);
        exec_b.push_back(pp.gates[0]);
      } else {
        for (int i = 0; i < pp.dev.n_ops; i++) exec.push_back(s.ops[pp.dev.op0 + i].gate);
        for (int i = 0; i < pp.devb.n_ops; i++) exec_b.push_back(s.ops[pp.devb.op0 + i].gate);
      }
    }
    exec_begin.push_back((int32_t)exec.size());
    exec_begin_b.push_back((int32_t)exec_b.size());
    h_exec_begin = exec_begin;
    h_exec_begin_b = exec_begin_b;
    n_occ = (int)s.grad_gate.size();
    std::vector<int32_t> occ_gate(s.grad_gate.begin(), s.grad_gate.end());
    std::vector<int64_t> occ_slot(n_occ);
    for (int j = 0; j < n_occ; j++)
      occ_slot[j] = s.grad_pass[j] < 0 ? -1 : s.passes[s.grad_pass[j]].devb.gpart_offset + s.grad_slot[j];
    std::vector<int32_t> p_ptr(s.n_params + 1, 0), i_ptr(s.n_inputs + 1, 0), p_occ, i_occ;
    for (int p = 0; p < s.n_params; p++) {
      for (int j = 0; j < n_occ; j++)
        if (s.gates[occ_gate[j]].param == p) p_occ.push_back(j);
      p_ptr[p + 1] = (int32_t)p_occ.size();
    }
    for (int c = 0; c < s.n_inputs; c++) {
      for (int j = 0; j < n_occ; j++)
        if (s.gates[occ_gate[j]].param == -2 - c) i_occ.push_back(j);
      i_ptr[c + 1] = (int32_t)i_occ.size();
    }
    std::vector<uint8_t> lnl;
    if (s.mode == QSIM_FUSED && !s.passes.empty()) {
      const DevPass& d = s.passes.back().dev;   // logical qubits of its tile and tile-index bits
      for (int j = 0; j < d.k; j++) lnl.push_back(d.Q[j]);
      for (int j = 0; j < d.n_nonlocal; j++) lnl.push_back(d.QN[j]);
      lnl.push_back(0);
    }
    std::vector<int32_t> pfx_begin, pfx_gate, pfx_occ;
    std::vector<uint8_t> lnf;
    if (s.has_prefix) {
      pfx_begin.push_back(0);
      for (int q = 0; q < s.n; q++) {
        for (int gi : s.prefix[q]) {
          int occ = -1;
          for (int j = 0; j < n_occ; j++)
            if (s.grad_pass[j] < 0 && s.grad_gate[j] == gi) occ = j;
          pfx_gate.push_back(gi);
          pfx_occ.push_back(occ);
        }
        pfx_begin.push_back((int32_t)pfx_gate.size());
      }
      const DevPass& d = s.passes.front().dev;
      for (int j = 0; j < d.k; j++) lnf.push_back(d.Q[j]);
      for (int j = 0; j < d.n_nonlocal; j++) lnf.push_back(d.QN[j]);
      lnf.push_back(0);
    }
#define QSIM_UP(PTR, VEC) \
  if (e == cudaSuccess) e = upload(&PTR, VEC);
    QSIM_UP(d_exec_gates_b, exec_b)
    QSIM_UP(d_exec_begin_b, exec_begin_b)
    QSIM_UP(d_gate_type, gtype)
    QSIM_UP(d_gate_param, gparam)
    QSIM_UP(d_gate_q0, gq0)
    QSIM_UP(d_gate_q1, gq1)
    QSIM_UP(d_exec_gates, exec)
    QSIM_UP(d_exec_begin, exec_begin)
    QSIM_UP(d_occ_gate, occ_gate)
    QSIM_UP(d_occ_slot, occ_slot)
    QSIM_UP(d_p_ptr, p_ptr)
    QSIM_UP(d_p_occ, p_occ)
    QSIM_UP(d_i_ptr, i_ptr)
    QSIM_UP(d_i_occ, i_occ)
    QSIM_UP(d_Qnl_last, lnl)
    QSIM_UP(d_pfx_begin, pfx_begin)
    QSIM_UP(d_pfx_gate, pfx_gate)
    QSIM_UP(d_pfx_occ, pfx_occ)
    QSIM_UP(d_Qnl_first, lnf)
#undef QSIM_UP
    if (e != cudaSuccess) return cuda_fail(e, "uploading the plan");
    if (s.mode == QSIM_FUSED) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      for (auto& pp : s.passes)
        if ((int64_t)single_smem_bytes(s, pp.dev, false) > optin || (int64_t)single_smem_bytes(s, pp.devb, true) > optin)
          return fail(QSIM_ERR_UNSUPPORTED, "tile does not fit in shared memory: lower k");
      std::string err;
      int rc = jit_build(s, jit, err);
      if (rc) return fail(rc, err);
    }
    uploaded = true;
    return QSIM_OK;
  }

  int ensure_ws(int B_) {
    if (B_ == B_cap) return QSIM_OK;
    free_ws();
    const int64_t G_ = (int64_t)s.gates.size(), P_ = P();
    const int64_t sb = state_bytes(B_);
    int64_t zcount = s.mode == QSIM_PER_GATE ? z_partials_count(s.n, B_)
                                             : (int64_t)B_ * tps() * (s.k + 1);
    struct Item {
      void** p;
      int64_t bytes;
    } items[] = {
        {&coef, G_ * B_ * sc}, {reinterpret_cast<void**>(&form), G_ * B_},
        {&cfp_f, (int64_t)h_exec_begin.back() * B_ * sc}, {reinterpret_cast<void**>(&fmp_f), (int64_t)h_exec_begin.back() * B_},
        {&cfp_b, (int64_t)h_exec_begin_b.back() * B_ * sc}, {reinterpret_cast<void**>(&fmp_b), (int64_t)h_exec_begin_b.back() * B_},
        {&scale_f, P_ * B_ * sc}, {&scale_b, P_ * B_ * sc},
        {reinterpret_cast<void**>(&gm), G_ * B_ * 8}, {reinterpret_cast<void**>(&zpart), zcount * 8},
        {reinterpret_cast<void**>(&gpart), s.total_gslots * B_ * tps() * 8},
        {reinterpret_cast<void**>(&G), (int64_t)n_occ * B_ * 8},
        {&W, sb}, {&Lam, sb},
        {&S_end, s.pauli_frame ? sb : 0}, {reinterpret_cast<void**>(&sigma), s.pauli_frame ? G_ * B_ : 0},
        {reinterpret_cast<void**>(&frame_x), s.pauli_frame ? (int64_t)B_ * 8 : 0},
        {reinterpret_cast<void**>(&frame_z), s.pauli_frame ? (int64_t)B_ * 8 : 0},
        {reinterpret_cast<void**>(&frame_k), s.pauli_frame ? (int64_t)B_ * 4 : 0},
        {reinterpret_cast<void**>(&gsign), s.pauli_frame ? (int64_t)B_ * s.n * 8 : 0},
        {&phi, s.has_prefix ? (int64_t)B_ * s.n * 4 * sc : 0},
        {reinterpret_cast<void**>(&ppart),
         s.has_prefix ? (int64_t)B_ * s.passes.front().devb.tiles_per_sample * (2 * s.k + 1) * 2 * 8 : 0},
    };
    for (auto& it : items) {
      if (it.bytes <= 0) continue;
      cudaError_t e = cudaMalloc(it.p, (size_t)it.bytes);
      if (e != cudaSuccess) {
        free_ws();
        return fail(QSIM_ERR_OOM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
      }
      ws_bytes += it.bytes;
    }
    // checkpoint segments (fused path only)
    n_segments = 1;
    if (s.mode == QSIM_FUSED && P_ > 1) {
      int m = 0;
      if (opts.checkpoint_passes > 0) {
        m = opts.checkpoint_passes;
      } else if (opts.checkpoint_passes < 0 && opts.mem_budget_bytes > 0 && sb > 0) {
        const int64_t avail = opts.mem_budget_bytes - ws_bytes;
        const int64_t nck = std::max<int64_t>(0, std::min<int64_t>(avail / sb, P_ - 1));
        if (nck > 0) m = (int)((P_ + nck) / (nck + 1));
      }
      if (m > 0 && m < P_) n_segments = (int)((P_ + m - 1) / m);
      seg_begin.clear();
      for (int j = 0; j < n_segments; j++) seg_begin.push_back(j * (m > 0 ? m : (int)P_));
      seg_begin.push_back((int)P_);
      for (int j = 0; j + 1 < n_segments; j++) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)sb);
        if (e != cudaSuccess) {
          free_ws();
          return fail(QSIM_ERR_OOM, std::string("checkpoint allocation failed: ") + cudaGetErrorString(e));
        }
        ckpt.push_back(p);
        ws_bytes += sb;
      }
    } else {
      seg_begin = {0, (int)P_};
    }
    B_cap = B_;
    return QSIM_OK;
  }

  int seg_of(int p) const {
    for (int j = 0; j < n_segments; j++)
      if (p < seg_begin[j + 1]) return j;
    return n_segments - 1;
  }

  JitArgs jit_args(int p, bool bwd, const void* scale) const {
    JitArgs a{};
    const DevPass& d = bwd ? s.passes[p].devb : s.passes[p].dev;
    const int64_t e0 = (int64_t)(bwd ? h_exec_begin_b[p] : h_exec_begin[p]) * B;
    a.cfp = static_cast<const char*>(bwd ? cfp_b : cfp_f) + e0 * sc;
    a.fmp = (bwd ? fmp_b : fmp_f) + e0;
    a.scale = scale;
    set_bits(a, d, bwd);
    a.tps = d.tiles_per_sample;
    a.gpart_offset = d.gpart_offset;
    a.n_nonlocal = d.n_nonlocal;
    a.n = s.n;
    a.B = B;
    return a;
  }

  PrefixArgs prefix_args(const void* params_, const void* inputs_) const {
    PrefixArgs a{};
    const DevPass& d = s.passes.front().devb;
    a.gate_type = d_gate_type;
    a.gate_param = d_gate_param;
    a.pfx_begin = d_pfx_begin;
    a.pfx_gate = d_pfx_gate;
    a.pfx_occ = d_pfx_occ;
    a.params = params_;
    a.inputs = inputs_;
    a.n_inputs = s.n_inputs;
    a.weight_remap = opts.weight_remap;
    a.n = s.n;
    a.B = B;
    a.phi = phi;
    a.ppart = ppart;
    a.Qnl = d_Qnl_first;
    a.K = d.k;
    a.n_nonlocal = d.n_nonlocal;
    a.tps = d.tiles_per_sample;
    a.G = G;
    return a;
  }

  PerGateArgs pg_args(int g, const void* scale) const {
    PerGateArgs a{};
    const Gate& x = s.gates[g];
    a.n = s.n;
    a.B = B;
    a.dtype = s.dtype;
    a.type = x.type;
    a.pos_t = s.n - 1 - x.t0;
    a.pos_c = x.c0 >= 0 ? s.n - 1 - x.c0 : 0;
    a.gate = g;
    a.coef = coef;
    a.form = form;
    a.scale = scale;
    return a;
  }
};

extern "C" {

void qsim_default_opts(qsim_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->k = 12;
  o->dtype = QSIM_C64;
  o->mode = QSIM_FUSED;
  o->contiguous_bits = 4;
  o->checkpoint_passes = 0;
  o->mem_budget_bytes = 0;
}

const char* qsim_last_error(void) { return g_err.c_str(); }

int qsim_plan(const qsim_gate* gates, int32_t n_gates, int32_t n_qubits, const qsim_plan_opts* opts,
              qsim_plan_t* out) {
  g_err.clear();
  if (!out) return fail(QSIM_ERR_ARG, "out is NULL");
  *out = nullptr;
  qsim_plan_opts o;
  qsim_default_opts(&o);
  if (opts) o = *opts;
  if (o.dtype != QSIM_C64 && o.dtype != QSIM_C128) return fail(QSIM_ERR_ARG, "dtype must be QSIM_C64 or QSIM_C128");
  if (o.mode != QSIM_FUSED && o.mode != QSIM_PER_GATE) return fail(QSIM_ERR_ARG, "mode must be QSIM_FUSED or QSIM_PER_GATE");
  if (o.k < 0 || o.contiguous_bits < 0 || o.checkpoint_passes < -1 || o.mem_budget_bytes < 0)
    return fail(QSIM_ERR_ARG, "negative option value");
  std::vector<Gate> gv;
  int np = 0, ni = 0;
  std::string err;
  int rc = validate_gates(gates, n_gates, n_qubits, gv, np, ni, err);
  if (rc) return fail(rc, err);
  auto* p = new qsim_plan_s();
  p->opts = o;
  p->el = o.dtype == QSIM_C128 ? 16 : 8;
  p->sc = o.dtype == QSIM_C128 ? 8 : 4;
  if (o.mode == QSIM_FUSED) {
    if (o.k == 0) o.k = default_k_for(o.dtype);
    if (o.k > max_k_for(o.dtype)) o.k = max_k_for(o.dtype);
  }
  p->opts = o;
  if (o.bwd_reg_bits < 0 || o.bwd_reg_bits > kMaxR || o.fwd_reg_bits < 0 || o.fwd_reg_bits > kMaxR ||
      o.sample_block < 0 || o.weight_remap < 0 || o.weight_remap > 2 || o.max_regs < 0 ||
      (o.max_regs > 0 && o.max_regs < 32) || (o.rotate_low_bits != 0 && o.rotate_low_bits != 1) ||
      (o.pauli_frame != 0 && o.pauli_frame != 1) || (o.pauli_frame == 1 && o.mode != QSIM_FUSED) ||
      (o.scalar_bwd != 0 && o.scalar_bwd != 1) || (o.product_prefix != 0 && o.product_prefix != 1) ||
      (o.product_prefix == 1 && o.mode != QSIM_FUSED) || (o.split_diagonal != 0 && o.split_diagonal != 1) ||
      o.reserved != 0) {
    delete p;
    return fail(QSIM_ERR_ARG, "fwd_reg_bits/bwd_reg_bits must be in [0, 5], sample_block >= 0, weight_remap 0..2, "
                              "max_regs 0 or >= 32, rotate_low_bits 0 or 1, pauli_frame 0 or 1 (fused mode), "
                              "scalar_bwd 0 or 1, product_prefix 0 or 1 (fused mode), split_diagonal 0 or 1, reserved 0");
  }
  const int Rf = o.fwd_reg_bits > 0 ? o.fwd_reg_bits : fwd_R_for(16, o.dtype);
  // single-circuit complex64 backward kernels hold 2^5 amplitudes of psi and lambda per thread: fewer
  // shared-memory exchanges per pass than 2^4, with 2 CTAs of 128 threads per SM instead of 2 of 256
  // (measured faster on the 20-qubit workload); the multi-circuit queue kernels, capped at 128
  // registers, keep 2^4
  const int Rb = o.bwd_reg_bits > 0 ? o.bwd_reg_bits : (o.dtype == QSIM_C64 ? 5 : bwd_R_for(16, o.dtype));
  // at most 256 threads per tile in either direction: a larger k with fewer amplitudes per thread is cut
  if (o.mode == QSIM_FUSED)
    while (o.k > 1 && (o.k - std::min(Rf, o.k) > 8 || o.k - std::min(Rb, o.k) > 8)) o.k--;
  p->opts = o;
  rc = build_schedule(gv, n_qubits, o, Rf, Rb, p->s, err, o.rotate_low_bits == 1);
  if (rc) {
    delete p;
    return fail(rc, err);
  }
  p->s.n_params = np;
  p->s.n_inputs = ni;
  *out = p;
  return QSIM_OK;
}

int qsim_plan_info_get(qsim_plan_t p, qsim_plan_info* info) {
  if (!p || !info) return fail(QSIM_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof *info);
  info->n_qubits = p->s.n;
  info->n_gates = (int32_t)p->s.gates.size();
  info->n_params = p->s.n_params;
  info->n_inputs = p->s.n_inputs;
  info->n_passes = p->P();
  info->k = p->s.k;
  info->dtype = p->s.dtype;
  info->mode = p->s.mode;
  info->n_checkpoints = (int32_t)p->ckpt.size();
  info->workspace_bytes = p->ws_bytes;
  return QSIM_OK;
}

int qsim_plan_describe(qsim_plan_t p, char* buf, size_t cap, size_t* needed) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  std::string d = describe_schedule(p->s);
  if (needed) *needed = d.size() + 1;
  if (buf && cap > 0) {
    size_t m = std::min(cap - 1, d.size());
    std::memcpy(buf, d.data(), m);
    buf[m] = 0;
  }
  return QSIM_OK;
}

int qsim_plan_kernel_source(qsim_plan_t p, char* buf, size_t cap, size_t* needed) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  std::string src;
  if (p->s.mode == QSIM_FUSED) {
    std::vector<std::string> fn, bn;
    src = jit_generate(p->s, fn, bn);
  }
  if (needed) *needed = src.size() + 1;
  if (buf && cap > 0) {
    size_t m = std::min(cap - 1, src.size());
    std::memcpy(buf, src.data(), m);
    buf[m] = 0;
  }
  return QSIM_OK;
}

int qsim_plan_compile_kernels(qsim_plan_t p) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  if (p->s.mode != QSIM_FUSED) return QSIM_OK;
  std::string err;
  std::map<std::string, std::string> cubins;
  std::vector<std::string> fn, bn;
  int rc = jit_compile(p->s, cubins, fn, bn, err);
  if (rc) return fail(rc, err);
  return QSIM_OK;
}

int qsim_tile_index_map(qsim_plan_t p, int32_t pass, int64_t tile, int64_t* out) {
  if (!p || !out) return fail(QSIM_ERR_ARG, "NULL argument");
  if (p->s.mode != QSIM_FUSED) return fail(QSIM_ERR_ARG, "index maps exist only for fused plans");
  if (pass < 0 || pass >= p->P()) return fail(QSIM_ERR_ARG, "pass out of range");
  const DevPass& d = p->s.passes[pass].dev;
  if (tile < 0 || tile >= d.tiles_per_sample) return fail(QSIM_ERR_ARG, "tile out of range");
  for (int64_t e = 0; e < ((int64_t)1 << d.k); e++) out[e] = tile_element_index(d, tile, e);
  return QSIM_OK;
}

int qsim_forward(qsim_plan_t p, const void* d_params, const void* d_inputs, int32_t batch, const void* d_init,
                 void* d_states, double* d_z, void* stream) {
  g_err.clear();
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  if (batch < 0) return fail(QSIM_ERR_ARG, "batch < 0");
  if (batch > (kMaxAmplitudes >> p->s.n)) return fail(QSIM_ERR_UNSUPPORTED, "batch x 2^n_qubits above 2^40 amplitudes");
  if (batch > 0 && (!d_states || !d_z)) return fail(QSIM_ERR_ARG, "d_states and d_z are required");
  if (p->s.n_params > 0 && !d_params) return fail(QSIM_ERR_ARG, "d_params is NULL but the circuit has parameters");
  if (p->s.n_inputs > 0 && batch > 0 && !d_inputs) return fail(QSIM_ERR_ARG, "d_inputs is NULL but the circuit has inputs");
  if (((uintptr_t)d_states & 15) || ((uintptr_t)d_init & 15)) return fail(QSIM_ERR_ARG, "state buffers must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  p->has_fwd = false;
  p->via_alt = false;
  if (p->s.has_prefix && d_init != nullptr) {
    // the prefix assumes the |0...0> start: an initial state runs the same circuit planned without it
    if (!p->alt) {
      std::vector<qsim_gate> gl;
      for (const Gate& g : p->s.gates) gl.push_back(qsim_gate{g.type, {g.t0, g.t1}, {g.c0, g.c1}, g.param});
      qsim_plan_opts o = p->opts;
      o.product_prefix = 0;
      qsim_plan_t a = nullptr;
      const int rc0 = qsim_plan(gl.data(), (int32_t)gl.size(), p->s.n, &o, &a);
      if (rc0) return rc0;
      p->alt = a;
    }
    p->via_alt = true;
    return qsim_forward(p->alt, d_params, d_inputs, batch, d_init, d_states, d_z, stream);
  }
  int rc = p->upload_schedule();
  if (rc) return rc;
  if (batch == 0) return QSIM_OK;
  rc = p->ensure_ws(batch);
  if (rc) return rc;
  p->B = batch;
  p->params = d_params;
  p->inputs = d_inputs;
  p->states = d_states;
  p->last_stream = st;
  const Schedule& s = p->s;
  cudaError_t e;
  CoefArgs ca{};
  ca.gate_type = p->d_gate_type;
  ca.gate_param = p->d_gate_param;
  ca.exec_gates = p->d_exec_gates;
  ca.exec_begin = p->d_exec_begin;
  ca.exec_gates_b = p->d_exec_gates_b;
  ca.exec_begin_b = p->d_exec_begin_b;
  ca.params = d_params;
  ca.inputs = d_inputs;
  ca.n_inputs = s.n_inputs;
  ca.B = batch;
  ca.P = p->P();
  ca.G = (int)s.gates.size();
  ca.weight_remap = p->opts.weight_remap;
  ca.coef = p->coef;
  ca.form = p->form;
  ca.cfp_f = p->cfp_f;
  ca.fmp_f = p->fmp_f;
  ca.cfp_b = p->cfp_b;
  ca.fmp_b = p->fmp_b;
  ca.scale_f = p->scale_f;
  ca.scale_b = p->scale_b;
  ca.gm = p->gm;
  if (s.pauli_frame) {
    ca.gate_q0 = p->d_gate_q0;
    ca.gate_q1 = p->d_gate_q1;
    ca.sigma = p->sigma;
    ca.frame_x = p->frame_x;
    ca.frame_z = p->frame_z;
    ca.frame_k = p->frame_k;
  }
  // every pass reads its per-sample scale (and, with a Pauli frame, the frame) from the packing kernel,
  // so it runs even for a gate list without rotations or an empty one (scales 1, identity frame)
  if (ca.P > 0) {
    e = launch_coef(ca, s.dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "coefficient kernel");
  }
  if (s.has_prefix) {   // phi_q of every sample and qubit: the first pass starts from their product
    e = launch_prefix_phi(p->prefix_args(d_params, d_inputs), s.dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "prefix state kernel");
  }
  const char* sf = reinterpret_cast<const char*>(p->scale_f);
  if (s.mode == QSIM_PER_GATE) {
    e = launch_pg_init(d_states, d_init, s.n, batch, s.dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    for (int g = 0; g < (int)s.gates.size(); g++) {
      const int rec = p->prof_begin(0, g, st);
      e = launch_pg_gate(p->pg_args(g, sf + (size_t)g * batch * p->sc), d_states, false, st);
      if (e != cudaSuccess) return cuda_fail(e, "per-gate kernel");
      p->prof_end(rec, st);
    }
    e = launch_expval_z(d_states, s.n, batch, s.dtype, p->zpart, d_z, st);
    if (e != cudaSuccess) return cuda_fail(e, "<Z> kernel");
  } else {
    const int P_ = p->P();
    const int G = p->group_size(batch);
    for (int b0 = 0; b0 < batch; b0 += G) {
      const int nb = std::min(G, batch - b0);
      for (int q = 0; q < P_; q++) {
        // Passes update their segment's buffer in place (a pass reads and writes the same addresses of
        // every tile: the layout changes between passes only permute qubits of its tile). The last
        // pass also restores the canonical qubit order, which moves qubits outside its tile, so it
        // writes out of place: the last segment runs in the workspace W and only its last pass writes
        // the caller's buffer.
        const int seg = p->seg_of(q);
        void* sbuf = (seg == p->n_segments - 1) ? (P_ > 1 ? p->W : d_states) : p->ckpt[seg];
        void* out = (q == P_ - 1) ? (s.pauli_frame ? p->S_end : d_states) : sbuf;
        const void* in;
        if (q == p->seg_begin[seg]) in = (seg == 0) ? d_init : p->ckpt[seg - 1];
        else in = sbuf;
        JitArgs ja = p->jit_args(q, false, sf + (size_t)q * batch * p->sc);
        ja.in = in;
        ja.out = out;
        ja.zpart = (q == P_ - 1) ? p->zpart : nullptr;
        ja.phi = (q == 0 && s.has_prefix) ? p->phi : nullptr;
        ja.b0 = b0;
        const int rec = p->prof_begin(0, q, st);
        e = jit_launch(p->jit.fwd[q], s.passes[q].dev.tiles_per_sample * nb, ja, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused forward pass");
        p->prof_end(rec, st);
      }
    }
    const DevPass& last = s.passes.back().dev;
    e = launch_z_final(p->zpart, last.k, p->d_Qnl_last, last.n_nonlocal, last.tiles_per_sample, s.n, batch, d_z, st,
                       s.pauli_frame ? p->frame_x : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "<Z> reduction");
    if (s.pauli_frame) {   // the returned states: F applied to the stored representation
      e = launch_frame_fixup(p->S_end, d_states, p->frame_x, p->frame_z, p->frame_k, s.n, batch, s.dtype, st);
      if (e != cudaSuccess) return cuda_fail(e, "frame fix-up");
    }
  }
  p->has_fwd = true;
  if (p->calls_left(0)) p->n_fwd_calls++;
  return QSIM_OK;
}

int qsim_backward(qsim_plan_t p, const double* d_grad_out, double* d_dparams, double* d_dinputs, void* stream) {
  g_err.clear();
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  if (p->via_alt) return qsim_backward(p->alt, d_grad_out, d_dparams, d_dinputs, stream);
  if (!p->has_fwd) return fail(QSIM_ERR_NO_FORWARD, "backward called without a preceding forward on this plan");
  const int B = p->B;
  if (!d_grad_out) return fail(QSIM_ERR_ARG, "d_grad_out is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  p->last_stream = st;
  const Schedule& s = p->s;
  cudaError_t e;
  const char* sbk = reinterpret_cast<const char*>(p->scale_b);
  if (s.mode == QSIM_PER_GATE) {
    e = launch_pg_lambda_init(p->states, p->W, p->Lam, d_grad_out, s.n, B, s.dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "lambda init");
    const int bps = pg_blocks_per_sample(s.n);
    for (int g = (int)s.gates.size() - 1; g >= 0; g--) {
      double* gp = p->gpart + s.passes[g].dev.gpart_offset * (int64_t)B * bps;
      const int rec = p->prof_begin(1, g, st);
      e = launch_pg_bwd_gate(p->pg_args(g, sbk + (size_t)g * B * p->sc), p->W, p->Lam, gp, bps, st);
      if (e != cudaSuccess) return cuda_fail(e, "per-gate backward kernel");
      p->prof_end(rec, st);
    }
  } else {
    const int P_ = p->P();
    if (s.pauli_frame) {   // lambda starts from g_{b,q} with the sign the final frame gives Z_q
      e = launch_frame_gsign(d_grad_out, p->frame_x, s.n, B, p->gsign, st);
      if (e != cudaSuccess) return cuda_fail(e, "frame signs");
    }
    const int G = p->group_size(B);
    for (int b0 = 0; b0 < B; b0 += G) {
      const int nb = std::min(G, B - b0);
      for (int q = P_ - 1; q >= 0; q--) {
        const int seg = p->seg_of(q);
        const bool seg_last = (q == p->seg_begin[seg + 1] - 1);
        const void* pend = s.pauli_frame ? p->S_end : p->states;   // the stored representation
        const void* pin = seg_last ? ((seg == p->n_segments - 1) ? pend : p->ckpt[seg]) : p->W;
        const void* lin = (q == P_ - 1) ? nullptr : p->Lam;
        // the previous pass restarts from its checkpoint when this pass begins a segment: psi not stored
        void* pout = (q == 0 || q == p->seg_begin[seg]) ? nullptr : p->W;
        void* lout = q == 0 ? nullptr : p->Lam;
        JitArgs ja = p->jit_args(q, true, sbk + (size_t)q * B * p->sc);
        ja.in = pin;
        ja.out = pout;
        ja.lam_in = lin;
        ja.lam_out = lout;
        ja.grad_out = s.pauli_frame ? p->gsign : d_grad_out;
        if (q == 0 && s.has_prefix) {   // the first pass also contracts lambda with the prefix states
          ja.phi = p->phi;
          ja.ppart = p->ppart;
        }
        ja.gpart = p->gpart;
        ja.b0 = b0;
        const int rec = p->prof_begin(1, q, st);
        e = jit_launch(p->jit.bwd[q], s.passes[q].devb.tiles_per_sample * nb, ja, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused backward pass");
        p->prof_end(rec, st);
      }
    }
  }
  GradReduceArgs ga{};
  ga.gpart = p->gpart;
  ga.tiles_per_sample = p->tps();
  ga.n_occ = p->n_occ;
  ga.occ_gate = p->d_occ_gate;
  ga.occ_slot = p->d_occ_slot;
  ga.gm = p->gm;
  ga.G = p->G;
  ga.B = B;
  ga.n_params = s.n_params;
  ga.n_inputs = s.n_inputs;
  ga.p_ptr = p->d_p_ptr;
  ga.p_occ = p->d_p_occ;
  ga.i_ptr = p->d_i_ptr;
  ga.i_occ = p->d_i_occ;
  ga.dparams = d_dparams;
  ga.dinputs = d_dinputs;
  ga.params = p->params;
  ga.inputs = p->inputs;
  ga.weight_remap = p->opts.weight_remap;
  ga.dtype = s.dtype;
  e = launch_grad_gather(ga, st);
  if (e == cudaSuccess && s.has_prefix) e = launch_prefix_grad(p->prefix_args(p->params, p->inputs), s.dtype, st);
  if (e == cudaSuccess) e = launch_grad_scatter(ga, st);
  if (e != cudaSuccess) return cuda_fail(e, "gradient reduction");
  if (p->calls_left(1)) p->n_bwd_calls++;
  return QSIM_OK;
}

int qsim_set_profiling(qsim_plan_t p, int32_t depth) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  if (depth < 0) return fail(QSIM_ERR_ARG, "depth < 0");
  if (p->uploaded) cudaStreamSynchronize(p->last_stream);
  p->prof_log.clear();
  p->ev_used = 0;
  p->n_fwd_calls = p->n_bwd_calls = 0;
  p->prof_depth = depth;
  p->profiling = depth > 0;
  return QSIM_OK;
}

int qsim_read_profile(qsim_plan_t p, float* fwd, float* bwd, int32_t cap, int32_t* n_passes, int32_t* n_calls) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  const int P_ = p->P();
  if (n_passes) *n_passes = P_;
  if (n_calls) {
    n_calls[0] = (int32_t)std::min<int64_t>(p->n_fwd_calls, p->prof_depth);
    n_calls[1] = (int32_t)std::min<int64_t>(p->n_bwd_calls, p->prof_depth);
  }
  for (int q = 0; q < P_ && q < cap; q++) {
    if (fwd) fwd[q] = 0.f;
    if (bwd) bwd[q] = 0.f;
  }
  for (auto& r : p->prof_log) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "reading profiling events");
    if (r.pass < cap) {
      float* dst = r.dir == 0 ? fwd : bwd;
      if (dst) dst[r.pass] += ms;
    }
  }
  return QSIM_OK;
}

int64_t qsim_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

int qsim_sync_status(qsim_plan_t p) {
  if (!p) return fail(QSIM_ERR_ARG, "plan is NULL");
  if (p->via_alt) return qsim_sync_status(p->alt);
  cudaError_t e = cudaStreamSynchronize(p->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return QSIM_OK;
}

int qsim_expval_z(const void* d_states, int32_t batch, int32_t n, int32_t dtype, double* d_z, void* stream) {
  g_err.clear();
  if (n < 1 || n > kMaxQubits) return fail(QSIM_ERR_UNSUPPORTED, "n_qubits outside [1, 34]");
  if (batch < 0) return fail(QSIM_ERR_ARG, "batch < 0");
  if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(QSIM_ERR_ARG, "bad dtype");
  if (batch > (kMaxAmplitudes >> n)) return fail(QSIM_ERR_UNSUPPORTED, "batch x 2^n_qubits above 2^40 amplitudes");
  if (batch == 0) return QSIM_OK;
  if (!d_states || !d_z) return fail(QSIM_ERR_ARG, "NULL buffer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), (size_t)z_partials_count(n, batch) * 8, st);
  if (e != cudaSuccess) return fail(QSIM_ERR_OOM, std::string("scratch allocation: ") + cudaGetErrorString(e));
  e = launch_expval_z(d_states, n, batch, dtype, scratch, d_z, st);
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_fail(e, "<Z> kernels");
  if (e2 != cudaSuccess) return cuda_fail(e2, "scratch free");
  return QSIM_OK;
}

int qsim_expval_z_noalloc(const void* d_states, int32_t batch, int32_t n, int32_t dtype, double* d_z,
                          void* stream) {
  g_err.clear();
  if (n < 1 || n > kMaxQubits) return fail(QSIM_ERR_UNSUPPORTED, "n_qubits outside [1, 34]");
  if (batch < 0) return fail(QSIM_ERR_ARG, "batch < 0");
  if (dtype != QSIM_C64 && dtype != QSIM_C128) return fail(QSIM_ERR_ARG, "bad dtype");
  if (batch == 0) return QSIM_OK;
  if (!d_states || !d_z) return fail(QSIM_ERR_ARG, "NULL buffer");
  const int64_t need = z_partials_count(n, batch);
  if (need > kNoAllocZPartials) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "batch %d x %d qubits needs %lld partial sums; the fixed scratch holds %lld "
             "(at 12+ qubits: batch * 2^(n-12) <= 40329); use qsim_expval_z",
             batch, n, (long long)need, (long long)kNoAllocZPartials);
    return fail(QSIM_ERR_UNSUPPORTED, buf);
  }
  cudaError_t e = launch_expval_z_noalloc(d_states, n, batch, dtype, d_z, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "<Z> kernels (no-allocation variant)");
  return QSIM_OK;
}

void qsim_plan_destroy(qsim_plan_t p) {
  if (!p) return;
  qsim_plan_destroy(p->alt);
  p->alt = nullptr;
  if (p->uploaded || p->B_cap >= 0) {
    cudaStreamSynchronize(p->last_stream);
    p->free_all();
  }
  delete p;
}

}  // extern "C"
