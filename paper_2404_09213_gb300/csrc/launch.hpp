// Host-side launch interfaces of the CUDA kernels (C++ linkage, used by the C ABI layer).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "plan_types.h"
#include "../../include/qsim.h"

namespace qsim {

// Number of kernels this library has launched in the process (for launch accounting).
extern std::atomic<long long> g_kernel_launches;

struct PassLaunch {
  const DevPass* h_pass;     // host copy (for sizes)
  const DevPass* d_pass;     // device copy
  const DevPhase* d_phases;
  const DevOp* d_ops;
  const DevLayout* d_layouts;
  int n, B;
  const void* coef;          // [G * B] scaled-rotation coefficients
  const uint8_t* form;       // [G * B] 0: tangent form, 1: cotangent form
  const void* scale;         // [B] this pass's scale (forward or backward)
};

// Forward pass over all tiles: in == nullptr starts from |0...0>; zpart != nullptr adds the
// <Z> epilogue (per-tile partial sums, (B * tiles) x (k+1) doubles).
cudaError_t launch_fwd_pass(const PassLaunch& L, int dtype, const void* in, void* out, double* zpart,
                            cudaStream_t st);

// Backward pass: psi_in/lam_in -> psi_out/lam_out (out == nullptr: no store); lam_in == nullptr
// initialises lambda = (sum_i g_{b,i} Z_i) psi from grad_out. Gradient partials go to gpart.
cudaError_t launch_bwd_pass(const PassLaunch& L, int dtype, const void* psi_in, void* psi_out,
                            const void* lam_in, void* lam_out, const double* grad_out, double* gpart,
                            cudaStream_t st);

size_t fwd_pass_smem(const DevPass& p, int dtype, int nthr);
size_t bwd_pass_smem(const DevPass& p, int dtype, int nthr);
cudaError_t prepare_pass_kernels(int dtype, size_t max_fwd_smem, size_t max_bwd_smem);
int bwd_R(int k);
int fwd_R_for(int k, int dtype);
int bwd_R_for(int k, int dtype);
int max_k_for(int dtype);

// ---- coefficients: one thread per (pass, sample)
struct CoefArgs {
  const int32_t* gate_type;     // [G]
  const int32_t* gate_param;    // [G]
  const int32_t* exec_gates;    // gate indices of every pass in forward execution order
  const int32_t* exec_begin;    // [P + 1]
  const int32_t* exec_gates_b;  // gate indices of every pass in the backward op order (undone last to first)
  const int32_t* exec_begin_b;  // [P + 1]
  const void* params;
  const void* inputs;
  int n_inputs, B, P;
  void* coef;                   // [G * B]
  uint8_t* form;                // [G * B]
  void* scale_f;                // [P * B]
  void* scale_b;                // [P * B]
  double* gm;                   // [G * B] squared backward scale at each rotation
};
cudaError_t launch_coef(const CoefArgs& a, int dtype, cudaStream_t st);

// ---- <Z> final reduction from per-tile partials: z[b][q]
cudaError_t launch_z_final(const double* zpart, int k, const uint8_t* d_L_and_nonlocal, int n_nonlocal,
                           int64_t tiles_per_sample, int n, int B, double* z, cudaStream_t st);

// ---- gradient reductions
struct GradReduceArgs {
  const double* gpart;
  int64_t tiles_per_sample;
  int n_occ;                    // parametric gate occurrences
  const int32_t* occ_gate;      // [n_occ]
  const int64_t* occ_slot;      // [n_occ] global slot (pass offset + slot)
  const double* gm;             // [G * B]
  double* G;                    // [n_occ * B]
  int B;
  int n_params, n_inputs;
  const int32_t* p_ptr; const int32_t* p_occ;     // CSR: param -> occurrences
  const int32_t* i_ptr; const int32_t* i_occ;     // CSR: input column -> occurrences
  double* dparams;              // may be null
  double* dinputs;              // may be null
};
cudaError_t launch_grad_reduce(const GradReduceArgs& a, cudaStream_t st);

// ---- per-gate (plain) path
struct PerGateArgs {
  int n, B, dtype;
  int type, pos_t, pos_c;       // physical bit positions of target / control
  int gate;                     // gate index (coefficients)
  const void* coef; const uint8_t* form; const void* scale;   // scale: [B] for this gate
};
cudaError_t launch_pg_init(void* states, const void* init, int n, int B, int dtype, cudaStream_t st);
cudaError_t launch_pg_gate(const PerGateArgs& a, void* states, bool inverse, cudaStream_t st);
cudaError_t launch_pg_bwd_gate(const PerGateArgs& a, void* psi, void* lam, double* gpart_slot,
                               int blocks_per_sample, cudaStream_t st);
cudaError_t launch_pg_lambda_init(const void* states, void* psi, void* lam, const double* grad_out, int n,
                                  int B, int dtype, cudaStream_t st);
int pg_blocks_per_sample(int n);

// ---- standalone <Z>: per-block partials + final reduction (scratch given by the caller)
int64_t z_partials_count(int n, int B);   // doubles of scratch needed
cudaError_t launch_expval_z(const void* states, int n, int B, int dtype, double* scratch, double* z,
                            cudaStream_t st);

}  // namespace qsim
