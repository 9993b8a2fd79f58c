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
  int n_inputs, B, P, G;
  int weight_remap;             // 1: trainable angles enter as pi * tanh(param); 2: input angles as well
  void* coef;                   // [G * B]
  uint8_t* form;                // [G * B]
  void* cfp_f;                  // packed forward op coefficients: pass p, sample b, op i at
                                //   exec_begin[p] * B + b * (ops of p) + i (0 for ops without one)
  uint8_t* fmp_f;               // packed forward forms, same index
  void* cfp_b;                  // packed backward op coefficients (negated: the inverse rotation), indexed
                                //   by exec_begin_b like cfp_f
  uint8_t* fmp_b;
  void* scale_f;                // [P * B]
  void* scale_b;                // [P * B]
  double* gm;                   // [G * B] squared backward scale at each rotation
  // several circuits (all null for a single circuit): circuit of every gate and its offsets
  const int32_t* gate_circ;     // [G]
  const int64_t* circ_param_off;   // [C] first parameter of the circuit
  const int64_t* circ_col_off;     // [C] input columns before the circuit (per sample)
  const int32_t* circ_ninputs;     // [C]
  // Pauli frame (all null without one): per gate its target and control qubit, per (gate, sample) the sign
  // the frame gives the rotation's coefficient, per sample the final frame F = i^k X^x Z^z (bit q = qubit q)
  const int32_t* gate_q0;       // [G] target qubit
  const int32_t* gate_q1;       // [G] control qubit (-1 for single-qubit gates)
  int8_t* sigma;                // [G * B]
  uint64_t* frame_x;            // [B]
  uint64_t* frame_z;            // [B]
  int32_t* frame_k;             // [B]
};
cudaError_t launch_coef(const CoefArgs& a, int dtype, cudaStream_t st);

// ---- Pauli frame: the returned states F S from the stored representation S (out of place), and the
// loss weights g_{b,q} with the sign (-1)^x_q the frame gives Z_q (lambda starts from them)
cudaError_t launch_frame_fixup(const void* S, void* out, const uint64_t* fx, const uint64_t* fz, const int32_t* fk,
                               int n, int B, int dtype, cudaStream_t st);
cudaError_t launch_frame_gsign(const double* grad_out, const uint64_t* fx, int n, int B, double* out,
                               cudaStream_t st);

// ---- <Z> final reduction from per-tile partials: z[b][q]
// d_Q_and_nonlocal: logical qubit of every tile bit, then of every tile-index bit, of the last pass
cudaError_t launch_z_final(const double* zpart, int k, const uint8_t* d_Q_and_nonlocal, int n_nonlocal,
                           int64_t tiles_per_sample, int n, int B, double* z, cudaStream_t st,
                           const uint64_t* frame_x = nullptr);

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
  const void* params;           // weight_remap: the raw params (float32 / float64 by dtype) for the chain rule
  const void* inputs;           // weight_remap == 2: the raw inputs (B x n_inputs) likewise
  int weight_remap, dtype;
};
cudaError_t launch_grad_reduce(const GradReduceArgs& a, cudaStream_t st);
// the two halves of launch_grad_reduce: per-occurrence sums (occurrences with occ_slot < 0 are skipped),
// then the sums over occurrences and samples
cudaError_t launch_grad_gather(const GradReduceArgs& a, cudaStream_t st);
cudaError_t launch_grad_scatter(const GradReduceArgs& a, cudaStream_t st);

// ---- product-state prefix (single-circuit fused plans)
struct PrefixArgs {
  const int32_t* gate_type;     // [G]
  const int32_t* gate_param;    // [G]
  const int32_t* pfx_begin;     // [n + 1] CSR over qubits into pfx_gate / pfx_occ
  const int32_t* pfx_gate;      // prefix gates of every qubit, in circuit order
  const int32_t* pfx_occ;       // gradient occurrence of each prefix gate (-1: not a rotation)
  const void* params;
  const void* inputs;
  int n_inputs, weight_remap;
  int n, B;
  void* phi;                    // [B][n][4] phi_q(0), phi_q(1) in the state's precision
  const double* ppart;          // [B][tps][2K + 1][2] backward partials of the first pass
  const uint8_t* Qnl;           // first pass: logical qubit of every tile bit, then of every tile-index bit
  int K, n_nonlocal;
  int64_t tps;
  double* G;                    // [n_occ][B]: dL/dtheta of every occurrence and sample
};
// phi_q = G_m ... G_1 |0> in FP64 for every (sample, qubit), stored in the state's precision
cudaError_t launch_prefix_phi(const PrefixArgs& a, int dtype, cudaStream_t st);
// mu_q from the partials, then dL/dtheta of every prefix rotation into G
cudaError_t launch_prefix_grad(const PrefixArgs& a, int dtype, cudaStream_t st);

// ---- several circuits
struct ZCirc {
  int64_t zp_off, tps, bits_off;
  int32_t k, n, n_nonlocal, pad;
};
struct ZMultiArgs {
  const double* zpart;
  const ZCirc* circ;
  const int64_t* zq_off;        // [C + 1] qubits before each circuit (per sample)
  const uint8_t* bits;
  double* z;
  int C, B;
};
cudaError_t launch_z_final_multi(const ZMultiArgs& a, int64_t total, cudaStream_t st);
struct GradMultiArgs {
  const double* gpart;
  int n_occ;
  const int32_t* occ_gate;      // global gate index
  const int64_t* occ_base;      // offset of the occurrence's partials for sample 0
  const int64_t* occ_tps;       // tiles per sample of its circuit
  const double* gm;
  double* G;
  int B;
  int64_t n_params, n_cols;     // global parameter count, global input columns
  const int32_t* p_ptr; const int32_t* p_occ;
  const int32_t* i_ptr; const int32_t* i_occ;
  const int64_t* col_circ_off;  // per global column: input columns before its circuit (per sample)
  const int32_t* col_stride;    // per global column: its circuit's n_inputs
  const int32_t* col_index;     // per global column: column within its circuit
  double* dparams;
  double* dinputs;
  const void* params;           // weight_remap: the raw concatenated params for the chain rule
  int weight_remap, dtype;
};
cudaError_t launch_grad_reduce_multi(const GradMultiArgs& a, cudaStream_t st);

// ---- gradient landscape (one batched evaluation of n_params x n_values parameter vectors)
// rows[k * V + v][j] = (j == k ? values[v] : base[j]); gout[b][i] = weights[i] for every row b;
// grid[k][v] = dinputs[(k * V + v) * P + k]
cudaError_t launch_landscape_inputs(const void* base, const void* values, int P, int V, int dtype, void* rows,
                                    const double* weights, int n, double* gout, cudaStream_t st);
cudaError_t launch_landscape_gather(const double* dinputs, int P, int V, double* grid, cudaStream_t st);

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

// ---- standalone <Z> with the partials in a fixed device array (no allocation); at most
// kNoAllocZPartials partial sums, i.e. z_partials_count(n, B) <= kNoAllocZPartials
constexpr int64_t kNoAllocZPartials = 524288;   // 4 MiB of doubles
cudaError_t launch_expval_z_noalloc(const void* states, int n, int B, int dtype, double* z, cudaStream_t st);

// ---- standalone <Z>: per-block partials + final reduction (scratch given by the caller)
int64_t z_partials_count(int n, int B);   // doubles of scratch needed
cudaError_t launch_expval_z(const void* states, int n, int B, int dtype, double* scratch, double* z,
                            cudaStream_t st);

}  // namespace qsim
