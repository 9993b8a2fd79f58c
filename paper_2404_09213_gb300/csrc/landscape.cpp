// Gradient landscape: dL/dtheta_k with theta_k swept over a list of values while the other parameters
// stay at a base point, for every k, in one batched forward + adjoint backward.
//
// The paper maps these landscapes (App. "Barren Plateaus": absolute gradient of every parameter at
// different rotations of that parameter, others constant, with and without weight remapping) to show
// that remapping removes barren plateaus. Here every trainable parameter of the circuit becomes a
// per-sample angle (an input column), so sample k * V + v carries the base vector with entry k set
// to values[v], and its dL/dinputs row holds the whole gradient at that point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qsim.h"
#include "launch.hpp"

namespace qsim {
void set_last_error(const std::string& s);
}

namespace {
int lfail(int code, const std::string& m) {
  qsim::set_last_error(m);
  return code;
}

// Sweeps repeat with the same circuit: the plan (with its compiled kernels and workspace) and the call's
// buffers are kept for the last few circuits, keyed by the remapped gate list, qubits, options and number
// of values. An event recorded after each call orders a later call on another stream behind it.
struct Entry {
  std::string key;
  qsim_plan_t plan = nullptr;
  void* rows = nullptr;
  void* states = nullptr;
  double* z = nullptr;
  double* gout = nullptr;
  double* dinp = nullptr;
  cudaEvent_t done = nullptr;
};
constexpr size_t kCached = 4;
std::mutex g_mu;
std::vector<Entry*>& cache() {   // most recently used last; never destroyed (no CUDA calls at exit)
  static std::vector<Entry*>* c = new std::vector<Entry*>();
  return *c;
}

void release(Entry* e) {
  if (e->done) {
    cudaEventSynchronize(e->done);
    cudaEventDestroy(e->done);
  }
  for (void* p : {e->rows, e->states, (void*)e->z, (void*)e->gout, (void*)e->dinp})
    if (p) cudaFree(p);
  if (e->plan) qsim_plan_destroy(e->plan);
  delete e;
}

std::string make_key(const std::vector<qsim_gate>& g, int n, const qsim_plan_opts& o, int n_values) {
  std::string k(reinterpret_cast<const char*>(g.data()), g.size() * sizeof(qsim_gate));
  k.append(reinterpret_cast<const char*>(&o), sizeof o);
  k.append(reinterpret_cast<const char*>(&n), sizeof n);
  k.append(reinterpret_cast<const char*>(&n_values), sizeof n_values);
  return k;
}
}  // namespace

extern "C" {

int qsim_landscape(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, const qsim_plan_opts* opts,
                   const void* d_base, const void* d_values, int32_t n_values, const double* d_weights,
                   double* d_grid, double* d_z, void* stream) {
  if (!h_gates || n_gates < 1 || !d_base || !d_values || n_values < 1 || !d_weights || !d_grid)
    return lfail(QSIM_ERR_ARG, "qsim_landscape: gates, base, values, weights and grid are required");
  qsim_plan_opts o;
  qsim_default_opts(&o);
  if (opts) o = *opts;
  if (o.mode != QSIM_FUSED || (o.weight_remap != 0 && o.weight_remap != 1))
    return lfail(QSIM_ERR_ARG, "qsim_landscape: fused mode, weight_remap 0 or 1");
  // trainable parameter p -> input column p; the circuit may not have input-encoded gates of its own
  std::vector<qsim_gate> g(h_gates, h_gates + n_gates);
  int P = 0;
  for (auto& x : g) {
    if (x.param <= -2) return lfail(QSIM_ERR_PARAM, "qsim_landscape: the circuit has input-encoded gates");
    if (x.param >= 0) {
      P = std::max(P, x.param + 1);
      x.param = -2 - x.param;
    }
  }
  if (P == 0) return lfail(QSIM_ERR_PARAM, "qsim_landscape: the circuit has no trainable parameter");
  const int64_t B64 = (int64_t)P * n_values;
  if (B64 > (1 << 30)) return lfail(QSIM_ERR_UNSUPPORTED, "qsim_landscape: n_params * n_values too large");
  const int B = (int)B64;
  o.weight_remap = o.weight_remap ? 2 : 0;   // the swept weights now sit in the input columns
  std::lock_guard<std::mutex> lock(g_mu);
  const std::string key = make_key(g, n_qubits, o, n_values);
  auto& c = cache();
  Entry* en = nullptr;
  for (size_t i = 0; i < c.size(); i++)
    if (c[i]->key == key) {
      en = c[i];
      c.erase(c.begin() + (long)i);
      break;
    }
  const size_t sc = o.dtype == QSIM_C128 ? 8 : 4;
  if (!en) {
    en = new Entry();
    en->key = key;
    int rc = qsim_plan(g.data(), n_gates, n_qubits, &o, &en->plan);
    cudaError_t e = rc ? cudaSuccess : cudaMalloc(&en->rows, (size_t)B * P * sc);
    if (!rc && e == cudaSuccess) e = cudaMalloc(&en->states, ((size_t)B * 2 * sc) << n_qubits);
    if (!rc && e == cudaSuccess) e = cudaMalloc((void**)&en->z, (size_t)B * n_qubits * 8);
    if (!rc && e == cudaSuccess) e = cudaMalloc((void**)&en->gout, (size_t)B * n_qubits * 8);
    if (!rc && e == cudaSuccess) e = cudaMalloc((void**)&en->dinp, (size_t)B * P * 8);
    if (!rc && e == cudaSuccess) e = cudaEventCreateWithFlags(&en->done, cudaEventDisableTiming);
    if (rc || e != cudaSuccess) {
      release(en);
      return rc ? rc : lfail(QSIM_ERR_OOM, std::string("qsim_landscape: ") + cudaGetErrorString(e));
    }
    if (c.size() == kCached) {   // the least recently used circuit makes room
      release(c.front());
      c.erase(c.begin());
    }
  }
  c.push_back(en);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamWaitEvent(st, en->done, 0);   // the previous call with these buffers
  int rc = 0;
  if (e == cudaSuccess) e = qsim::launch_landscape_inputs(d_base, d_values, P, n_values, o.dtype, en->rows, d_weights,
                                                    n_qubits, en->gout, st);
  if (e != cudaSuccess) rc = lfail(QSIM_ERR_CUDA, std::string("qsim_landscape: ") + cudaGetErrorString(e));
  if (!rc) rc = qsim_forward(en->plan, nullptr, en->rows, B, nullptr, en->states, en->z, stream);
  if (!rc) rc = qsim_backward(en->plan, en->gout, nullptr, en->dinp, stream);
  if (!rc) {
    e = qsim::launch_landscape_gather(en->dinp, P, n_values, d_grid, st);
    if (e == cudaSuccess && d_z) e = cudaMemcpyAsync(d_z, en->z, (size_t)B * n_qubits * 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) rc = lfail(QSIM_ERR_CUDA, std::string("qsim_landscape: ") + cudaGetErrorString(e));
  }
  cudaEventRecord(en->done, st);
  return rc;
}

void qsim_landscape_clear_cache(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (Entry* en : cache()) release(en);
  cache().clear();
}

}  // extern "C"
