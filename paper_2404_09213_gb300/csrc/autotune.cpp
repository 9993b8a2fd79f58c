// Tile-size autotuner: times the fused path of a circuit for each candidate k on scratch buffers and
// keeps the fastest. Built on the public entry points only (qsim_plan / qsim_forward / qsim_backward).
//
// Candidates are the largest tiles that still fit the register/shared-memory budget of one CTA
// (max_k - 2 .. max_k). A larger k means fewer passes (fewer HBM round trips); a smaller one means
// smaller CTAs with cheaper barriers and more of them resident per SM. Which wins depends on the
// circuit and the batch, so it is measured. Circuits with n <= max_k run in one pass at k = n; for
// them the candidates are the amplitudes per thread of the register phases instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "jit.hpp"

namespace qsim {
void set_last_error(const std::string& s);
}

namespace {

struct Scratch {
  std::vector<void*> bufs;
  ~Scratch() {
    for (void* p : bufs) cudaFree(p);
  }
  void* get(size_t bytes, cudaStream_t st, cudaError_t& e) {
    if (e != cudaSuccess || bytes == 0) return nullptr;
    void* p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return nullptr;
    bufs.push_back(p);
    e = cudaMemsetAsync(p, 0, bytes, st);
    return p;
  }
};

int fail(int code, const std::string& m) {
  qsim::set_last_error(m);
  return code;
}

// Mean milliseconds of one forward (+ backward) call of the circuit planned with `o`; < 0 on error.
int time_candidate(const qsim_gate* g, int32_t ng, int32_t n, int32_t batch, int32_t with_bwd, int32_t reps,
                   const qsim_plan_opts& o, cudaStream_t st, float& ms) {
  qsim_plan_t p = nullptr;
  int rc = qsim_plan(g, ng, n, &o, &p);
  if (rc) return rc;
  qsim_plan_info inf;
  qsim_plan_info_get(p, &inf);
  const size_t sc = o.dtype == QSIM_C128 ? 8 : 4;
  Scratch s;
  cudaError_t e = cudaSuccess;
  void* params = s.get(std::max<size_t>(1, (size_t)inf.n_params) * sc, st, e);
  void* inputs = s.get(std::max<size_t>(1, (size_t)batch * inf.n_inputs) * sc, st, e);
  void* states = s.get((size_t)batch * (2 * sc) << n, st, e);
  double* z = static_cast<double*>(s.get((size_t)batch * n * 8, st, e));
  double* gout = static_cast<double*>(s.get((size_t)batch * n * 8, st, e));
  double* dp = static_cast<double*>(s.get(std::max<size_t>(1, (size_t)inf.n_params) * 8, st, e));
  double* di = static_cast<double*>(s.get(std::max<size_t>(1, (size_t)batch * inf.n_inputs) * 8, st, e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    qsim_plan_destroy(p);
    return fail(QSIM_ERR_OOM, std::string("autotune scratch: ") + cudaGetErrorString(e));
  }
  auto step = [&]() {
    int r = qsim_forward(p, params, inf.n_inputs ? inputs : nullptr, batch, nullptr, states, z, st);
    if (!r && with_bwd) r = qsim_backward(p, gout, dp, inf.n_inputs ? di : nullptr, st);
    return r;
  };
  rc = step();   // untimed: compiles the pass kernels and sizes the workspace
  if (!rc) {
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps && !rc; i++) rc = step();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (!rc && e != cudaSuccess) rc = fail(QSIM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    if (!rc) rc = qsim_sync_status(p);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms = t / (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  qsim_plan_destroy(p);
  return rc;
}

// Candidates kmax - 2 .. kmax; n_qubits <= kmax runs in one pass at k = n_qubits.
int autotune_upto(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, int32_t batch, int32_t with_backward,
                  int32_t reps, qsim_plan_opts* opts, float* h_ms, void* stream, int kmax) {
  if (!opts || batch < 1 || reps < 1) return fail(QSIM_ERR_ARG, "autotune: opts must be set, batch >= 1, reps >= 1");
  if (opts->mode != QSIM_FUSED) return fail(QSIM_ERR_ARG, "autotune: fused mode only");
  if (opts->dtype != QSIM_C64 && opts->dtype != QSIM_C128) return fail(QSIM_ERR_ARG, "autotune: bad dtype");
  if (h_ms)
    for (int i = 0; i < 4; i++) h_ms[i] = -1.f;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n_qubits <= kmax) {
    // One pass holds the whole state, so k is n; what remains to choose is the amplitudes per thread of
    // the register phases and the Pauli frame. Candidates: 2^5 and 2^4 with the frame and without it
    // when it was requested, else 2^5, 2^4 and 2^3 without. Fewer amplitudes mean shorter unrolled code
    // and more resident warps, more mean fewer shared-memory exchanges; the frame halves the code but
    // adds a walk per sample and a fix-up of the returned states, which a single short pass may not
    // repay. Single-circuit plans only.
    opts->k = n_qubits;
    if (kmax != qsim::max_k_for(opts->dtype) || opts->fwd_reg_bits != 0 || opts->bwd_reg_bits != 0) return QSIM_OK;
    const int top = qsim::fwd_R_for(16, opts->dtype);
    const bool frame = opts->pauli_frame == 1;
    const int nc = frame ? 4 : 3;
    const int rb[4] = {top, top - 1, frame ? top : top - 2, top - 1};
    const bool off[4] = {!frame, !frame, true, true};
    float ms[4];
    int best = 0;
    for (int i = 0; i < nc; i++) {
      qsim_plan_opts o = *opts;
      o.fwd_reg_bits = std::min(rb[i], n_qubits);
      if (with_backward) o.bwd_reg_bits = std::min(rb[i], n_qubits);
      if (off[i]) o.pauli_frame = 0;
      const int rc = time_candidate(h_gates, n_gates, n_qubits, batch, with_backward, reps, o, st, ms[i]);
      if (rc) return rc;
      if (h_ms) h_ms[i] = ms[i];
      if (ms[i] < ms[best]) best = i;
    }
    if (off[best]) opts->pauli_frame = 0;
    if (rb[best] != top) {   // keep the library defaults (0) when the largest register count wins
      opts->fwd_reg_bits = std::min(rb[best], n_qubits);
      if (with_backward) opts->bwd_reg_bits = std::min(rb[best], n_qubits);
    }
    return QSIM_OK;
  }
  float ms[3];
  for (int i = 0; i < 3; i++) {
    qsim_plan_opts o = *opts;
    o.k = kmax - 2 + i;
    const int rc = time_candidate(h_gates, n_gates, n_qubits, batch, with_backward, reps, o, st, ms[i]);
    if (rc) return rc;
    if (h_ms) h_ms[i] = ms[i];
  }
  // the largest k within 2 % of the fastest: fewer passes over HBM, and a choice that does not flip
  // with timing noise between near-equal candidates
  const float fastest = std::min(ms[0], std::min(ms[1], ms[2]));
  int best = kmax - 2;
  for (int i = 0; i < 3; i++)
    if (ms[i] <= fastest * 1.02f) best = kmax - 2 + i;
  opts->k = best;
  return QSIM_OK;
}

}  // namespace

extern "C" {

int qsim_autotune(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, int32_t batch, int32_t with_backward,
                  int32_t reps, qsim_plan_opts* opts, float* h_ms, void* stream) {
  if (!opts) return fail(QSIM_ERR_ARG, "autotune: opts must be set");
  return autotune_upto(h_gates, n_gates, n_qubits, batch, with_backward, reps, opts, h_ms, stream,
                       qsim::max_k_for(opts->dtype));
}

int qsim_multi_autotune(const qsim_gate* const* h_gate_lists, const int32_t* h_n_gates, const int32_t* h_n_qubits,
                        int32_t n_circuits, int32_t batch, int32_t with_backward, int32_t reps,
                        const qsim_plan_opts* opts, int32_t* h_k, void* stream) {
  if (!h_gate_lists || !h_n_gates || !h_n_qubits || !h_k || n_circuits < 1)
    return fail(QSIM_ERR_ARG, "multi autotune: NULL argument or no circuits");
  qsim_plan_opts base;
  qsim_default_opts(&base);
  if (opts) base = *opts;
  // time single-circuit plans with the register bits the queue kernels use (their own default differs)
  if (base.bwd_reg_bits == 0) base.bwd_reg_bits = qsim::bwd_R_for(16, base.dtype);
  if (base.fwd_reg_bits == 0) base.fwd_reg_bits = qsim::fwd_R_for(16, base.dtype);
  // one representative (the first circuit) per qubit count
  std::map<int, int> rep_of;
  for (int c = 0; c < n_circuits; c++)
    if (!rep_of.count(h_n_qubits[c])) rep_of[h_n_qubits[c]] = c;
  std::map<int, int> k_of;
  for (auto& kv : rep_of) {
    qsim_plan_opts o = base;
    const int c = kv.second;
    // multi-circuit plans take tiles of at most multi_max_k_for qubits (see multi.cpp)
    const int rc = autotune_upto(h_gate_lists[c], h_n_gates[c], h_n_qubits[c], batch, with_backward, reps, &o,
                                 nullptr, stream, qsim::multi_max_k_for(o.dtype));
    if (rc) return rc;
    k_of[kv.first] = o.k;
  }
  for (int c = 0; c < n_circuits; c++) h_k[c] = k_of[h_n_qubits[c]];
  return QSIM_OK;
}

}  // extern "C"
