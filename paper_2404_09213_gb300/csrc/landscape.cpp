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
  qsim_plan_t plan = nullptr;
  int rc = qsim_plan(g.data(), n_gates, n_qubits, &o, &plan);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t sc = o.dtype == QSIM_C128 ? 8 : 4;
  void *rows = nullptr, *states = nullptr;
  double *z = nullptr, *gout = nullptr, *dinp = nullptr;
  cudaError_t e = cudaMallocAsync(&rows, (size_t)B * P * sc, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&states, ((size_t)B * 2 * sc) << n_qubits, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&z, (size_t)B * n_qubits * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&gout, (size_t)B * n_qubits * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dinp, (size_t)B * P * 8, st);
  if (e == cudaSuccess) e = qsim::launch_landscape_inputs(d_base, d_values, P, n_values, o.dtype, rows, d_weights,
                                                    n_qubits, gout, st);
  if (e != cudaSuccess) rc = lfail(QSIM_ERR_OOM, std::string("qsim_landscape: ") + cudaGetErrorString(e));
  if (!rc) rc = qsim_forward(plan, nullptr, rows, B, nullptr, states, z, stream);
  if (!rc) rc = qsim_backward(plan, gout, nullptr, dinp, stream);
  if (!rc) {
    e = qsim::launch_landscape_gather(dinp, P, n_values, d_grid, st);
    if (e == cudaSuccess && d_z) e = cudaMemcpyAsync(d_z, z, (size_t)B * n_qubits * 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) rc = lfail(QSIM_ERR_CUDA, std::string("qsim_landscape: ") + cudaGetErrorString(e));
  }
  for (void* ptr : {rows, states, (void*)z, (void*)gout, (void*)dinp})
    if (ptr) cudaFreeAsync(ptr, st);
  qsim_plan_destroy(plan);   // waits for the stream (the plan's workspace is in use until then)
  return rc;
}

}  // extern "C"
