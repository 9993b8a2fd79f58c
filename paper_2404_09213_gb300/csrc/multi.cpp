// Several circuits of uneven size in one persistent launch per direction.
//
// Every circuit is planned as usual (its own k-local passes). A device work queue lists tile jobs in
// rounds (pass 0 of every circuit, then pass 1, ...); one persistent kernel per direction claims
// jobs with an atomic counter, waits (bounded) until the previous pass of the same circuit is
// complete, runs the job's specialised pass code, and signals completion. Small circuits run several
// samples' tiles per CTA. Coefficients, <Z> and gradient reductions are one launch each for all
// circuits; with opts.graph the whole launch sequence is captured once into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "jit.hpp"
#include "launch.hpp"
#include "planner.hpp"

using namespace qsim;

namespace {
thread_local std::string m_err;
int mfail(int code, const std::string& msg);

// Queue kernel CTAs of 128 threads in both directions; with tiles of at most 11 qubits (10 for
// complex128; 2^(k - R) <= 128 threads per tile) and at most 128 registers per thread (link option) four
// CTAs fit on an SM. Every pass structure of a direction lives in one kernel, so its registers and
// shared memory are the maxima over them: larger tiles would cost every circuit occupancy.
constexpr int kCtaF = 128, kCtaB = 128;
static int multi_max_k(int dtype) { return multi_max_k_for(dtype); }

struct QItem {   // mirrors qj::Item
  int32_t kind, arg;
  int64_t tile0, ntiles;
  int32_t wait, wait_target, done, pad;
};
struct QMultiArgs {   // mirrors qj::MultiArgs
  const QItem* items;
  int64_t n_items;
  unsigned long long* head;
  int* counters;
  int* status;
  const JitArgs* args;
  int64_t timeout_ns;
  int64_t withhold;
};

template <typename T>
cudaError_t up(T** d, const std::vector<T>& v) {
  *d = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}
}  // namespace

// error text shared with the single-circuit API (qsim_last_error)
namespace qsim {
void set_last_error(const std::string& s);
}

namespace {
int mfail(int code, const std::string& msg) {
  qsim::set_last_error(msg);
  return code;
}
int mcuda(cudaError_t e, const char* what) {
  qsim::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return QSIM_ERR_CUDA;
}
// exec-list entry of an op: its gate in the concatenated gate list, or -1 for a rescale op
int32_t op_gate(const DevOp& op, int64_t goff) { return op.gate < 0 ? -1 : (int32_t)(goff + op.gate); }
}  // namespace

struct qsim_multi_s {
  std::vector<Schedule> sch;
  // circuits run by their own single-circuit plan (at least large_circuit_qubits qubits): no queue
  // items, no queue-kernel code, no queue gradient occurrences, no <Z> rows
  std::vector<char> ext;
  std::vector<qsim_plan_t> ext_plan;
  qsim_plan_opts opts{};
  int C = 0, el = 8, sc = 4, dtype = QSIM_C64;
  const void* params = nullptr;   // of the last forward (weight remapping needs them in the backward)
  // global numbering
  std::vector<int64_t> goff, poff, param_off, col_off, amp_off, zq_off;
  int64_t G_tot = 0, P_tot = 0, n_params = 0, n_cols = 0;
  // static device data
  bool uploaded = false;
  JitMulti jm;
  int32_t *d_gtype = nullptr, *d_gparam = nullptr, *d_exf = nullptr, *d_exbf = nullptr, *d_exb = nullptr,
          *d_exbb = nullptr, *d_gate_circ = nullptr, *d_ninp = nullptr;
  int64_t *d_circ_param_off = nullptr, *d_circ_col_off = nullptr, *d_zq_off = nullptr;
  uint8_t* d_bits = nullptr;
  std::vector<int64_t> off_bits;                     // per global pass
  std::vector<int32_t> h_exbf, h_exbb;               // first op of every global pass in the packed coefficients
  int n_occ = 0;
  int32_t *d_occ_gate = nullptr, *d_p_ptr = nullptr, *d_p_occ = nullptr, *d_i_ptr = nullptr, *d_i_occ = nullptr,
          *d_col_stride = nullptr, *d_col_index = nullptr;
  int64_t* d_col_circ_off = nullptr;
  std::vector<int32_t> occ_circ, occ_slot;   // host: circuit, slot within its circuit's gradient slots
  // batch workspace
  int B = -1;
  void *coef = nullptr, *scale_f = nullptr, *scale_b = nullptr, *W = nullptr, *Lam = nullptr;
  uint8_t* form = nullptr;
  void *cfp_f = nullptr, *cfp_b = nullptr;           // packed per-pass op coefficients (backward: negated)
  uint8_t *fmp_f = nullptr, *fmp_b = nullptr;
  double *gm = nullptr, *zpart = nullptr, *gpart = nullptr, *G = nullptr;
  int64_t *d_occ_base = nullptr, *d_occ_tps = nullptr;
  ZCirc* d_zcirc = nullptr;
  QItem *d_items_f = nullptr, *d_items_b = nullptr;
  int64_t n_items_f = 0, n_items_b = 0;
  int* d_counters = nullptr;
  unsigned long long* d_heads = nullptr;   // [0] forward, [1] backward
  int* d_status = nullptr;
  JitArgs *d_args_f = nullptr, *d_args_b = nullptr;
  std::vector<int64_t> zp_off, gp_off;   // per circuit (elements)
  int64_t timeout_ns = 4000000000LL;
  int64_t withhold = -1;
  // saved forward
  bool has_fwd = false;
  void* states = nullptr;
  cudaStream_t last = nullptr;
  // CUDA graphs of the two launch sequences (keyed by the pointers they were captured with)
  cudaGraphExec_t gx_f = nullptr, gx_b = nullptr;
  long long graph_kernels_f = 0, graph_kernels_b = 0;   // kernel nodes of each captured graph
  std::vector<const void*> key_f, key_b;
  std::vector<JitArgs> host_args_f, host_args_b;   // last uploaded argument blocks
  cudaStream_t cap = nullptr;   // plan-owned stream the graphs are captured on (the caller's may be the legacy stream)

  cudaError_t capture_stream() {
    if (cap) return cudaSuccess;
    return cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  }

  int64_t tps(int c) const { return sch[c].passes[0].dev.tiles_per_sample; }
  int P(int c) const { return (int)sch[c].passes.size(); }

  void free_ws() {
    void* ps[] = {coef, cfp_f, cfp_b, fmp_f, fmp_b, scale_f, scale_b, W, Lam, form, gm, zpart, gpart, G, d_occ_base, d_occ_tps, d_zcirc,
                  d_items_f, d_items_b, d_counters, d_heads, d_status, d_args_f, d_args_b};
    for (void* p : ps)
      if (p) cudaFree(p);
    coef = cfp_f = cfp_b = scale_f = scale_b = W = Lam = nullptr;
    form = fmp_f = fmp_b = nullptr;
    gm = zpart = gpart = G = nullptr;
    d_occ_base = d_occ_tps = nullptr;
    d_zcirc = nullptr;
    d_items_f = d_items_b = nullptr;
    d_counters = nullptr;
    d_heads = nullptr;
    d_status = nullptr;
    d_args_f = d_args_b = nullptr;
    host_args_f.clear();
    host_args_b.clear();
    if (gx_f) cudaGraphExecDestroy(gx_f);
    if (gx_b) cudaGraphExecDestroy(gx_b);
    gx_f = gx_b = nullptr;
    key_f.clear();
    key_b.clear();
    B = -1;
  }
  void free_all() {
    free_ws();
    void* ps[] = {d_gtype, d_gparam, d_exf, d_exbf, d_exb, d_exbb, d_gate_circ, d_ninp, d_circ_param_off,
                  d_circ_col_off, d_zq_off, d_bits, d_occ_gate, d_p_ptr, d_p_occ, d_i_ptr, d_i_occ,
                  d_col_stride, d_col_index, d_col_circ_off};
    for (void* p : ps)
      if (p) cudaFree(p);
    jit_free_multi(jm);
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
    uploaded = false;
  }

  int upload() {
    if (uploaded) return QSIM_OK;
    std::vector<int32_t> gtype, gparam, exf, exbf, exb, exbb, gate_circ, ninp, p_ptr, p_occ, i_ptr, i_occ,
        col_stride, col_index, occ_gate;
    std::vector<int64_t> cpo, cco, zqo, col_circ_off;
    std::vector<uint8_t> bits;
    occ_circ.clear();
    occ_slot.clear();
    std::vector<std::vector<int>> p_list(n_params), i_list(n_cols);
    for (int c = 0; c < C; c++) {
      const Schedule& s = sch[c];
      for (auto& g : s.gates) {
        gtype.push_back(g.type);
        gparam.push_back(g.param);
        gate_circ.push_back(c);
      }
      cpo.push_back(param_off[c]);
      cco.push_back(col_off[c]);
      ninp.push_back(s.n_inputs);
      for (int p = 0; p < P(c); p++) {
        const auto& pp = s.passes[p];
        exbf.push_back((int32_t)exf.size());
        for (int i = 0; i < pp.dev.n_ops; i++) exf.push_back(op_gate(s.ops[pp.dev.op0 + i], goff[c]));
        exbb.push_back((int32_t)exb.size());
        for (int i = 0; i < pp.devb.n_ops; i++) exb.push_back(op_gate(s.ops[pp.devb.op0 + i], goff[c]));
        off_bits.push_back((int64_t)bits.size());
        for (int j = 0; j < pp.dev.k; j++) bits.push_back(pp.dev.Q[j]);   // logical qubits (<Z> reduction)
        for (int j = 0; j < pp.dev.n_nonlocal; j++) bits.push_back(pp.dev.QN[j]);
        bits.push_back(0);
      }
      for (size_t j = 0; j < (ext[c] ? 0 : s.grad_gate.size()); j++) {
        const int g = s.grad_gate[j];
        const int occ = (int)occ_gate.size();
        occ_gate.push_back((int32_t)(goff[c] + g));
        occ_circ.push_back(c);
        occ_slot.push_back((int32_t)(s.passes[s.grad_pass[j]].devb.gpart_offset + s.grad_slot[j]));
        const int pr = s.gates[g].param;
        if (pr >= 0) p_list[param_off[c] + pr].push_back(occ);
        else i_list[col_off[c] + (-2 - pr)].push_back(occ);
      }
      for (int col = 0; col < s.n_inputs; col++) {
        col_circ_off.push_back(col_off[c]);
        col_stride.push_back(s.n_inputs);
        col_index.push_back(col);
      }
    }
    exbf.push_back((int32_t)exf.size());
    exbb.push_back((int32_t)exb.size());
    h_exbf = exbf;
    h_exbb = exbb;
    for (int c = 0; c <= C; c++) zqo.push_back(zq_off[c]);
    p_ptr.push_back(0);
    for (auto& l : p_list) {
      for (int o : l) p_occ.push_back(o);
      p_ptr.push_back((int32_t)p_occ.size());
    }
    i_ptr.push_back(0);
    for (auto& l : i_list) {
      for (int o : l) i_occ.push_back(o);
      i_ptr.push_back((int32_t)i_occ.size());
    }
    n_occ = (int)occ_gate.size();
    cudaError_t e = cudaSuccess;
#define QSIM_UP(P, V) \
  if (e == cudaSuccess) e = up(&P, V);
    QSIM_UP(d_gtype, gtype) QSIM_UP(d_gparam, gparam) QSIM_UP(d_exf, exf) QSIM_UP(d_exbf, exbf)
    QSIM_UP(d_exb, exb) QSIM_UP(d_exbb, exbb) QSIM_UP(d_gate_circ, gate_circ) QSIM_UP(d_ninp, ninp)
    QSIM_UP(d_circ_param_off, cpo) QSIM_UP(d_circ_col_off, cco) QSIM_UP(d_zq_off, zqo) QSIM_UP(d_bits, bits)
    QSIM_UP(d_occ_gate, occ_gate) QSIM_UP(d_p_ptr, p_ptr) QSIM_UP(d_p_occ, p_occ)
    QSIM_UP(d_i_ptr, i_ptr) QSIM_UP(d_i_occ, i_occ) QSIM_UP(d_col_stride, col_stride)
    QSIM_UP(d_col_index, col_index) QSIM_UP(d_col_circ_off, col_circ_off)
#undef QSIM_UP
    if (e != cudaSuccess) return mcuda(e, "uploading the multi-circuit plan");
    std::vector<const Schedule*> ptrs;
    for (int c = 0; c < C; c++) ptrs.push_back(ext[c] ? nullptr : &sch[c]);
    std::string err;
    int rc = jit_build_multi(ptrs, kCtaF, kCtaB, jm, err);
    if (rc) return mfail(rc, err);
    uploaded = true;
    return QSIM_OK;
  }

  int ensure_ws(int B_) {
    if (B_ == B) return QSIM_OK;
    free_ws();
    std::vector<int64_t> occ_base(n_occ), occ_tps(n_occ);
    zp_off.assign(C + 1, 0);
    gp_off.assign(C + 1, 0);
    for (int c = 0; c < C; c++) {
      zp_off[c + 1] = zp_off[c] + (int64_t)B_ * tps(c) * (sch[c].k + 1);
      gp_off[c + 1] = gp_off[c] + sch[c].total_gslots * B_ * tps(c);
    }
    for (int j = 0; j < n_occ; j++) {
      const int c = occ_circ[j];
      occ_tps[j] = tps(c);
      occ_base[j] = gp_off[c] + (int64_t)occ_slot[j] * B_ * tps(c);
    }
    std::vector<ZCirc> zc(C);
    for (int c = 0; c < C; c++) {
      const DevPass& last = sch[c].passes.back().dev;
      zc[c] = {zp_off[c], tps(c), off_bits[poff[c] + P(c) - 1], ext[c] ? -1 : last.k, sch[c].n, last.n_nonlocal, 0};
    }
    // work queues: rounds of passes, items of up to CTA / NTHR tiles
    std::vector<QItem> itf, itb;
    std::vector<int> n_items_pass(2 * P_tot, 0);
    int maxP = 0;
    for (int c = 0; c < C; c++) maxP = std::max(maxP, P(c));
    for (int dir = 0; dir < 2; dir++) {
      auto& items = dir == 0 ? itf : itb;
      const int cta = dir == 0 ? kCtaF : kCtaB;
      for (int r = 0; r < maxP; r++) {
        for (int c = 0; c < C; c++) {
          if (r >= P(c) || ext[c]) continue;
          const int p = dir == 0 ? r : P(c) - 1 - r;
          const DevPass& d = dir == 0 ? sch[c].passes[p].dev : sch[c].passes[p].devb;
          const int nthr = 1 << (d.k - d.R);
          const int per = std::max(1, cta / nthr);
          const int64_t nt = (int64_t)B_ * tps(c);
          const int64_t gp = poff[c] + p;
          const int ctr = (int)(dir * P_tot + gp);
          int wait = -1, target = 0;
          if (r > 0) {
            const int prev = dir == 0 ? p - 1 : p + 1;
            wait = (int)(dir * P_tot + poff[c] + prev);
            target = n_items_pass[wait];
          }
          for (int64_t t0 = 0; t0 < nt; t0 += per) {
            items.push_back({jm.kind[c][2 * p + dir], (int32_t)gp, t0, nt, wait, target, ctr, 0});
            n_items_pass[ctr]++;
          }
        }
      }
    }
    n_items_f = (int64_t)itf.size();
    n_items_b = (int64_t)itb.size();
    const int64_t amps = amp_off[C] * B_;
    struct Alloc {
      void** p;
      int64_t bytes;
    } al[] = {{&coef, G_tot * B_ * sc}, {reinterpret_cast<void**>(&form), G_tot * B_},
              {&cfp_f, (int64_t)h_exbf.back() * B_ * sc}, {reinterpret_cast<void**>(&fmp_f), (int64_t)h_exbf.back() * B_},
              {&cfp_b, (int64_t)h_exbb.back() * B_ * sc}, {reinterpret_cast<void**>(&fmp_b), (int64_t)h_exbb.back() * B_},
              {&scale_f, P_tot * B_ * sc}, {&scale_b, P_tot * B_ * sc},
              {reinterpret_cast<void**>(&gm), G_tot * B_ * 8}, {reinterpret_cast<void**>(&zpart), zp_off[C] * 8},
              {reinterpret_cast<void**>(&gpart), gp_off[C] * 8}, {reinterpret_cast<void**>(&G), (int64_t)n_occ * B_ * 8},
              {&W, amps * el}, {&Lam, amps * el},
              {reinterpret_cast<void**>(&d_counters), 2 * P_tot * 4}, {reinterpret_cast<void**>(&d_heads), 16},
              {reinterpret_cast<void**>(&d_status), 16},
              {reinterpret_cast<void**>(&d_args_f), P_tot * (int64_t)sizeof(JitArgs)},
              {reinterpret_cast<void**>(&d_args_b), P_tot * (int64_t)sizeof(JitArgs)}};
    for (auto& a : al) {
      if (a.bytes <= 0) continue;
      cudaError_t e = cudaMalloc(a.p, (size_t)a.bytes);
      if (e != cudaSuccess) {
        free_ws();
        return mfail(QSIM_ERR_OOM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
      }
    }
    cudaError_t e = up(&d_occ_base, occ_base);
    if (e == cudaSuccess) e = up(&d_occ_tps, occ_tps);
    if (e == cudaSuccess) e = up(&d_zcirc, zc);
    if (e == cudaSuccess) e = up(&d_items_f, itf);
    if (e == cudaSuccess) e = up(&d_items_b, itb);
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, 16);
    if (e != cudaSuccess) {
      free_ws();
      return mcuda(e, "uploading the work queues");
    }
    B = B_;
    return QSIM_OK;
  }

  JitArgs pass_args(int c, int p, bool bwd, const void* states_c, const double* gout) const {
    JitArgs a{};
    const DevPass& d = bwd ? sch[c].passes[p].devb : sch[c].passes[p].dev;
    const int64_t gp = poff[c] + p;
    const int64_t amp0 = amp_off[c] * B;
    const int64_t e0 = (int64_t)(bwd ? h_exbb[gp] : h_exbf[gp]) * B;
    a.cfp = static_cast<const char*>(bwd ? cfp_b : cfp_f) + e0 * sc;
    a.fmp = (bwd ? fmp_b : fmp_f) + e0;
    a.scale = reinterpret_cast<const char*>(bwd ? scale_b : scale_f) + (size_t)gp * B * sc;
    set_bits(a, d, bwd);
    a.tps = d.tiles_per_sample;
    a.gpart_offset = d.gpart_offset;
    a.n_nonlocal = d.n_nonlocal;
    a.n = sch[c].n;
    a.B = B;
    a.b0 = 0;
    char* st = reinterpret_cast<char*>(const_cast<void*>(states_c));
    if (!bwd) {
      // intermediate states in the workspace W (updated in place); the last pass, which restores the
      // canonical qubit order and so does not write the addresses it reads, writes the state block
      char* w = reinterpret_cast<char*>(W) + amp0 * el;
      a.in = p == 0 ? nullptr : w;
      a.out = p == P(c) - 1 ? st : w;
      a.zpart = p == P(c) - 1 ? zpart + zp_off[c] : nullptr;
    } else {
      char* w = reinterpret_cast<char*>(W) + amp0 * el;
      char* l = reinterpret_cast<char*>(Lam) + amp0 * el;
      const bool first = p == P(c) - 1;
      a.in = first ? st : w;
      a.out = p == 0 ? nullptr : w;
      a.lam_in = first ? nullptr : l;
      a.lam_out = p == 0 ? nullptr : l;
      a.grad_out = gout + zq_off[c] * B;
      a.gpart = gpart + gp_off[c];
    }
    return a;
  }
};

extern "C" {

int qsim_multi_plan(const qsim_gate* const* lists, const int32_t* n_gates, const int32_t* n_qubits, int32_t n_circ,
                    const qsim_plan_opts* opts, const int32_t* h_k, qsim_multi_t* out) {
  qsim::set_last_error("");
  if (!out) return mfail(QSIM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_circ < 1 || !lists || !n_gates || !n_qubits) return mfail(QSIM_ERR_ARG, "empty circuit list");
  qsim_plan_opts o;
  qsim_default_opts(&o);
  if (opts) o = *opts;
  if (o.mode != QSIM_FUSED) return mfail(QSIM_ERR_ARG, "multi-circuit plans use the fused mode");
  if (o.dtype != QSIM_C64 && o.dtype != QSIM_C128) return mfail(QSIM_ERR_ARG, "bad dtype");
  if (o.bwd_reg_bits < 0 || o.bwd_reg_bits > kMaxR || o.fwd_reg_bits < 0 || o.fwd_reg_bits > kMaxR ||
      (o.weight_remap != 0 && o.weight_remap != 1) || o.max_regs != 0 || o.pauli_frame != 0 || o.scalar_bwd != 0 ||
      o.product_prefix != 0 || o.split_diagonal != 0 || o.reserved != 0)
    return mfail(QSIM_ERR_ARG, "fwd_reg_bits/bwd_reg_bits must be in [0, 5], weight_remap 0 or 1, max_regs 0 "
                               "(multi-circuit kernels size their own CTAs), pauli_frame 0, scalar_bwd 0, product_prefix 0, split_diagonal 0, reserved 0");
  if (o.k == 0 || o.k > multi_max_k(o.dtype)) o.k = multi_max_k(o.dtype);
  auto* m = new qsim_multi_s();
  m->opts = o;
  m->C = n_circ;
  m->dtype = o.dtype;
  m->el = o.dtype == QSIM_C128 ? 16 : 8;
  m->sc = o.dtype == QSIM_C128 ? 8 : 4;
  m->goff.assign(1, 0);
  m->poff.assign(1, 0);
  m->param_off.assign(1, 0);
  m->col_off.assign(1, 0);
  m->amp_off.assign(1, 0);
  m->zq_off.assign(1, 0);
  for (int c = 0; c < n_circ; c++) {
    std::vector<Gate> gv;
    int np = 0, ni = 0;
    std::string err;
    int rc = validate_gates(lists[c], n_gates[c], n_qubits[c], gv, np, ni, err);
    if (!rc && n_qubits[c] > 30) {
      rc = QSIM_ERR_UNSUPPORTED;
      err = "multi-circuit plans support up to 30 qubits per circuit";
    }
    Schedule s;
    if (!rc) {
      const int Rf = o.fwd_reg_bits > 0 ? o.fwd_reg_bits : fwd_R_for(16, o.dtype);
      const int Rb = o.bwd_reg_bits > 0 ? o.bwd_reg_bits : bwd_R_for(16, o.dtype);
      qsim_plan_opts oc = o;
      if (h_k) {
        if (h_k[c] < 1 || h_k[c] > multi_max_k(o.dtype)) {
          delete m;
          return mfail(QSIM_ERR_ARG, "circuit " + std::to_string(c) + ": per-circuit k outside [1, " +
                                         std::to_string(multi_max_k(o.dtype)) + "]");
        }
        oc.k = h_k[c];
      }
      rc = build_schedule(gv, n_qubits[c], oc, Rf, Rb, s, err, false);
    }
    if (rc) {
      delete m;
      return mfail(rc, "circuit " + std::to_string(c) + ": " + err);
    }
    s.n_params = np;
    s.n_inputs = ni;
    m->goff.push_back(m->goff.back() + (int64_t)s.gates.size());
    m->poff.push_back(m->poff.back() + (int64_t)s.passes.size());
    m->param_off.push_back(m->param_off.back() + np);
    m->col_off.push_back(m->col_off.back() + ni);
    m->amp_off.push_back(m->amp_off.back() + ((int64_t)1 << n_qubits[c]));
    m->zq_off.push_back(m->zq_off.back() + n_qubits[c]);
    m->sch.push_back(std::move(s));
  }
  // circuits large enough to fill the GPU on their own run as single-circuit plans (the queue's kernels
  // hold every pass structure at once and so run with smaller tiles and fewer registers than theirs)
  // default 18: measured on the 256-circuit workload (8..22 qubits, batch 4), 16 / 17 / 18 / 20 / 22 /
  // none gave 6155 / 6429 / 6604 / 6284 / 4833 / 3588 samples/s
  const int large = o.large_circuit_qubits > 0 ? o.large_circuit_qubits : o.large_circuit_qubits == 0 ? 18 : 1 << 30;
  m->ext.assign(n_circ, 0);
  m->ext_plan.assign(n_circ, nullptr);
  for (int c = 0; c < n_circ; c++) {
    if (n_qubits[c] < large) continue;
    qsim_plan_opts so;
    qsim_default_opts(&so);
    so.dtype = o.dtype;
    so.weight_remap = o.weight_remap;
    so.pauli_frame = 1;
    so.product_prefix = 1;
    const int rc = qsim_plan(lists[c], n_gates[c], n_qubits[c], &so, &m->ext_plan[c]);
    if (rc) {
      const std::string why = qsim_last_error();
      qsim_multi_destroy(m);
      return mfail(rc, "circuit " + std::to_string(c) + " (own plan): " + why);
    }
    m->ext[c] = 1;
  }
  m->G_tot = m->goff.back();
  m->P_tot = m->poff.back();
  m->n_params = m->param_off.back();
  m->n_cols = m->col_off.back();
  *out = m;
  return QSIM_OK;
}

int qsim_multi_offsets(qsim_multi_t m, int32_t batch, int64_t* po, int64_t* io, int64_t* so, int64_t* zo) {
  if (!m || batch < 0) return mfail(QSIM_ERR_ARG, "bad arguments");
  for (int c = 0; c <= m->C; c++) {
    if (po) po[c] = m->param_off[c];
    if (io) io[c] = (int64_t)batch * m->col_off[c];
    if (so) so[c] = (int64_t)batch * m->amp_off[c];
    if (zo) zo[c] = (int64_t)batch * m->zq_off[c];
  }
  return QSIM_OK;
}

int qsim_multi_set_test_hooks(qsim_multi_t m, int64_t withhold_item, int64_t timeout_ns) {
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  // captured graphs hold the old values in their kernel parameters: drop them (the next call with
  // graphs on captures again), after any replay still in flight has finished
  if (m->gx_f || m->gx_b) {
    cudaError_t e = cudaStreamSynchronize(m->last);
    if (e != cudaSuccess) return mcuda(e, "stream synchronize");
    if (m->gx_f) cudaGraphExecDestroy(m->gx_f);
    if (m->gx_b) cudaGraphExecDestroy(m->gx_b);
    m->gx_f = m->gx_b = nullptr;
    m->key_f.clear();
    m->key_b.clear();
  }
  m->withhold = withhold_item;
  m->timeout_ns = timeout_ns > 0 ? timeout_ns : 4000000000LL;
  return QSIM_OK;
}

static cudaError_t multi_enqueue_fwd(qsim_multi_t m, const void* d_params, const void* d_inputs, void* d_states,
                                     double* d_z, cudaStream_t st) {
  CoefArgs ca{};
  ca.gate_type = m->d_gtype;
  ca.gate_param = m->d_gparam;
  ca.exec_gates = m->d_exf;
  ca.exec_begin = m->d_exbf;
  ca.exec_gates_b = m->d_exb;
  ca.exec_begin_b = m->d_exbb;
  ca.params = d_params;
  ca.inputs = d_inputs;
  ca.n_inputs = 0;
  ca.B = m->B;
  ca.P = (int)m->P_tot;
  ca.G = (int)m->G_tot;
  ca.weight_remap = m->opts.weight_remap;
  ca.coef = m->coef;
  ca.form = m->form;
  ca.cfp_f = m->cfp_f;
  ca.fmp_f = m->fmp_f;
  ca.cfp_b = m->cfp_b;
  ca.fmp_b = m->fmp_b;
  ca.scale_f = m->scale_f;
  ca.scale_b = m->scale_b;
  ca.gm = m->gm;
  ca.gate_circ = m->d_gate_circ;
  ca.circ_param_off = m->d_circ_param_off;
  ca.circ_col_off = m->d_circ_col_off;
  ca.circ_ninputs = m->d_ninp;
  cudaError_t e = launch_coef(ca, m->dtype, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(m->d_counters, 0, (size_t)m->P_tot * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_heads, 0, 8, st);
  if (e != cudaSuccess) return e;
  QMultiArgs qa{m->d_items_f, m->n_items_f, m->d_heads, m->d_counters, m->d_status, m->d_args_f, m->timeout_ns,
                m->withhold};
  void* args[] = {&qa};
  const int64_t blocks = std::min<int64_t>(m->jm.fwd.max_blocks, std::max<int64_t>(1, m->n_items_f));
  e = cudaLaunchKernel(m->jm.fwd.fn, dim3((unsigned)blocks), dim3((unsigned)m->jm.fwd.nthr), args, m->jm.fwd.smem, st);
  if (e != cudaSuccess) return e;
  g_kernel_launches++;
  ZMultiArgs za{m->zpart, m->d_zcirc, m->d_zq_off, m->d_bits, d_z, m->C, m->B};
  return launch_z_final_multi(za, (int64_t)m->B * m->zq_off[m->C], st);
}

int qsim_multi_forward(qsim_multi_t m, const void* d_params, const void* d_inputs, int32_t batch, void* d_states,
                       double* d_z, void* stream) {
  qsim::set_last_error("");
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  if (batch < 1) return mfail(QSIM_ERR_ARG, "batch must be >= 1");
  for (const Schedule& s : m->sch)
    if (batch > (kMaxAmplitudes >> s.n)) return mfail(QSIM_ERR_UNSUPPORTED, "batch x 2^n_qubits above 2^40 amplitudes");
  if (!d_states || !d_z) return mfail(QSIM_ERR_ARG, "d_states and d_z are required");
  if (m->n_params > 0 && !d_params) return mfail(QSIM_ERR_ARG, "d_params is NULL");
  if (m->n_cols > 0 && !d_inputs) return mfail(QSIM_ERR_ARG, "d_inputs is NULL");
  if ((uintptr_t)d_states & 15) return mfail(QSIM_ERR_ARG, "states must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = m->upload();
  if (rc) return rc;
  rc = m->ensure_ws(batch);
  if (rc) return rc;
  m->last = st;
  // argument blocks of every pass (they depend on the caller's buffers)
  std::vector<JitArgs> af(m->P_tot);
  for (int c = 0; c < m->C; c++) {
    void* sc_ = reinterpret_cast<char*>(d_states) + m->amp_off[c] * batch * m->el;
    for (int p = 0; p < m->P(c); p++) af[m->poff[c] + p] = m->pass_args(c, p, false, sc_, nullptr);
  }
  std::vector<const void*> key = {d_params, d_inputs, d_states, d_z};
  const bool same = m->gx_f && key == m->key_f;
  if (af.size() != m->host_args_f.size() ||
      std::memcmp(af.data(), m->host_args_f.data(), af.size() * sizeof(JitArgs)) != 0) {
    // argument blocks changed (new buffers): replace them once the stream has drained
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_args_f, af.data(), af.size() * sizeof(JitArgs), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mcuda(e, "uploading pass arguments");
    m->host_args_f = af;
  }
  cudaError_t e;
  if (m->opts.graph) {
    if (!same) {
      if (m->gx_f) cudaGraphExecDestroy(m->gx_f);
      m->gx_f = nullptr;
      cudaGraph_t g = nullptr;
      e = m->capture_stream();
      if (e == cudaSuccess) e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const long long c0 = g_kernel_launches.load();
        cudaError_t e2 = multi_enqueue_fwd(m, d_params, d_inputs, d_states, d_z, m->cap);
        e = cudaStreamEndCapture(m->cap, &g);
        if (e == cudaSuccess) e = e2;
        m->graph_kernels_f = g_kernel_launches.load() - c0;   // captured, not run: counted per replay
        g_kernel_launches -= m->graph_kernels_f;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&m->gx_f, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return mcuda(e, "capturing the forward graph");
      m->key_f = key;
    }
    e = cudaGraphLaunch(m->gx_f, st);
    if (e == cudaSuccess) g_kernel_launches += m->graph_kernels_f;
  } else {
    e = multi_enqueue_fwd(m, d_params, d_inputs, d_states, d_z, st);
  }
  if (e != cudaSuccess) return mcuda(e, "multi-circuit forward");
  for (int c = 0; c < m->C; c++) {   // the large circuits, each on its slices of the buffers
    if (!m->ext[c]) continue;
    const Schedule& s = m->sch[c];
    const void* pc = s.n_params ? static_cast<const char*>(d_params) + m->param_off[c] * m->sc : nullptr;
    const void* ic = s.n_inputs ? static_cast<const char*>(d_inputs) + (int64_t)batch * m->col_off[c] * m->sc : nullptr;
    void* stc = static_cast<char*>(d_states) + m->amp_off[c] * batch * m->el;
    const int r2 = qsim_forward(m->ext_plan[c], pc, ic, batch, nullptr, stc, d_z + (int64_t)batch * m->zq_off[c], stream);
    if (r2) return r2;
  }
  m->states = d_states;
  m->params = d_params;
  m->has_fwd = true;
  return QSIM_OK;
}

static cudaError_t multi_enqueue_bwd(qsim_multi_t m, double* d_dparams, double* d_dinputs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(m->d_counters + m->P_tot, 0, (size_t)m->P_tot * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_heads + 1, 0, 8, st);
  if (e != cudaSuccess) return e;
  QMultiArgs qa{m->d_items_b, m->n_items_b, m->d_heads + 1, m->d_counters, m->d_status, m->d_args_b, m->timeout_ns,
                m->withhold};
  void* args[] = {&qa};
  const int64_t blocks = std::min<int64_t>(m->jm.bwd.max_blocks, std::max<int64_t>(1, m->n_items_b));
  e = cudaLaunchKernel(m->jm.bwd.fn, dim3((unsigned)blocks), dim3((unsigned)m->jm.bwd.nthr), args, m->jm.bwd.smem, st);
  if (e != cudaSuccess) return e;
  g_kernel_launches++;
  GradMultiArgs ga{};
  ga.gpart = m->gpart;
  ga.n_occ = m->n_occ;
  ga.occ_gate = m->d_occ_gate;
  ga.occ_base = m->d_occ_base;
  ga.occ_tps = m->d_occ_tps;
  ga.gm = m->gm;
  ga.G = m->G;
  ga.B = m->B;
  ga.n_params = m->n_params;
  ga.n_cols = m->n_cols;
  ga.p_ptr = m->d_p_ptr;
  ga.p_occ = m->d_p_occ;
  ga.i_ptr = m->d_i_ptr;
  ga.i_occ = m->d_i_occ;
  ga.col_circ_off = m->d_col_circ_off;
  ga.col_stride = m->d_col_stride;
  ga.col_index = m->d_col_index;
  ga.dparams = d_dparams;
  ga.dinputs = d_dinputs;
  ga.params = m->params;
  ga.weight_remap = m->opts.weight_remap;
  ga.dtype = m->dtype;
  return launch_grad_reduce_multi(ga, st);
}

int qsim_multi_backward(qsim_multi_t m, const double* d_grad_out, double* d_dparams, double* d_dinputs,
                        void* stream) {
  qsim::set_last_error("");
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  if (!m->has_fwd) return mfail(QSIM_ERR_NO_FORWARD, "backward called without a preceding forward on this plan");
  if (!d_grad_out) return mfail(QSIM_ERR_ARG, "d_grad_out is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last = st;
  std::vector<JitArgs> ab(m->P_tot);
  for (int c = 0; c < m->C; c++) {
    void* sc_ = reinterpret_cast<char*>(m->states) + m->amp_off[c] * m->B * m->el;
    for (int p = 0; p < m->P(c); p++) ab[m->poff[c] + p] = m->pass_args(c, p, true, sc_, d_grad_out);
  }
  std::vector<const void*> key = {m->states, d_grad_out, d_dparams, d_dinputs};
  const bool same = m->gx_b && key == m->key_b;
  if (ab.size() != m->host_args_b.size() ||
      std::memcmp(ab.data(), m->host_args_b.data(), ab.size() * sizeof(JitArgs)) != 0) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_args_b, ab.data(), ab.size() * sizeof(JitArgs), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mcuda(e, "uploading pass arguments");
    m->host_args_b = ab;
  }
  cudaError_t e;
  if (m->opts.graph) {
    if (!same) {
      if (m->gx_b) cudaGraphExecDestroy(m->gx_b);
      m->gx_b = nullptr;
      cudaGraph_t g = nullptr;
      e = m->capture_stream();
      if (e == cudaSuccess) e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const long long c0 = g_kernel_launches.load();
        cudaError_t e2 = multi_enqueue_bwd(m, d_dparams, d_dinputs, m->cap);
        e = cudaStreamEndCapture(m->cap, &g);
        if (e == cudaSuccess) e = e2;
        m->graph_kernels_b = g_kernel_launches.load() - c0;   // captured, not run: counted per replay
        g_kernel_launches -= m->graph_kernels_b;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&m->gx_b, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return mcuda(e, "capturing the backward graph");
      m->key_b = key;
    }
    e = cudaGraphLaunch(m->gx_b, st);
    if (e == cudaSuccess) g_kernel_launches += m->graph_kernels_b;
  } else {
    e = multi_enqueue_bwd(m, d_dparams, d_dinputs, st);
  }
  if (e != cudaSuccess) return mcuda(e, "multi-circuit backward");
  // the queue's gradient scatter wrote zeros for the large circuits' entries: their plans come after
  for (int c = 0; c < m->C; c++) {
    if (!m->ext[c]) continue;
    const Schedule& s = m->sch[c];
    double* dp = (d_dparams && s.n_params) ? d_dparams + m->param_off[c] : nullptr;
    double* di = (d_dinputs && s.n_inputs) ? d_dinputs + (int64_t)m->B * m->col_off[c] : nullptr;
    const int r2 = qsim_backward(m->ext_plan[c], d_grad_out + (int64_t)m->B * m->zq_off[c], dp, di, stream);
    if (r2) return r2;
  }
  return QSIM_OK;
}

int qsim_multi_sync_status(qsim_multi_t m) {
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  if (!m->d_status) return QSIM_OK;
  cudaError_t e = cudaStreamSynchronize(m->last);
  if (e != cudaSuccess) return mcuda(e, "stream synchronize");
  int status = 0;
  e = cudaMemcpy(&status, m->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return mcuda(e, "reading the device status");
  if (status != 0) {
    cudaMemset(m->d_status, 0, sizeof(int));
    return mfail(status, "a queue item waited longer than the time limit for the pass before it");
  }
  return QSIM_OK;
}

int qsim_multi_info(qsim_multi_t m, int32_t* n_circuits, int64_t* n_items_fwd, int64_t* n_items_bwd,
                    int32_t* n_kernels_fwd, int32_t* n_kernels_bwd) {
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  if (n_circuits) *n_circuits = m->C;
  if (n_items_fwd) *n_items_fwd = m->n_items_f;
  if (n_items_bwd) *n_items_bwd = m->n_items_b;
  if (n_kernels_fwd) *n_kernels_fwd = m->jm.n_kinds[0];
  if (n_kernels_bwd) *n_kernels_bwd = m->jm.n_kinds[1];
  return QSIM_OK;
}

int qsim_multi_kernel_info(qsim_multi_t m, int32_t* ctas_per_sm, int32_t* regs, int64_t* smem) {
  if (!m) return mfail(QSIM_ERR_ARG, "plan is NULL");
  if (!m->uploaded) return mfail(QSIM_ERR_NO_FORWARD, "the queue kernels are built by the first forward");
  const JitKernel* k[2] = {&m->jm.fwd, &m->jm.bwd};
  for (int d = 0; d < 2; d++) {
    if (ctas_per_sm) ctas_per_sm[d] = k[d]->per_sm;
    if (regs) regs[d] = k[d]->regs;
    if (smem) smem[d] = (int64_t)k[d]->smem;
  }
  return QSIM_OK;
}

void qsim_multi_destroy(qsim_multi_t m) {
  if (!m) return;
  for (qsim_plan_t p : m->ext_plan) qsim_plan_destroy(p);
  m->ext_plan.clear();
  if (m->uploaded || m->B >= 0) {
    cudaStreamSynchronize(m->last);
    m->free_all();
  }
  delete m;
}

}  // extern "C"
