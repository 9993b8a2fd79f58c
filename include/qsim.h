/*
 * qsim.h — C ABI of the batched state-vector simulator (GB300, sm_103a).
 *
 * What it computes (arXiv 2404.09213, "Qandle"):
 *   - a batch of B states of n qubits, psi_b in C^(2^n), stored (B, 2^n) row-major with interleaved
 *     (re, im) — the batched shape (B, 2^W) of Sec. "Concept of Shapes";
 *   - qubit q is the q-th MOST significant index bit (MSb-0, Sec. "Symbols"): bit (n-1-q) of x;
 *   - a gate list (Sec. "Hybrid Machine Learning": embedding layers, trainable layers) applied in order, each gate one
 *     of RX, RY, RZ (R_P(theta) = exp(-i theta P / 2); RX written as in Eq. 1), H, X, CNOT, CZ;
 *   - the measurement layer <Z_i>_b = sum_x |psi_b[x]|^2 (1 - 2 bit_i(x)) for every qubit i;
 *   - gradients of L = sum_{b,i} g_{b,i} <Z_i>_b by the adjoint method (Sec. "Hybrid Machine Learning": backpropagation
 *     through the simulator); shared parameters sum over the batch, inputs are per sample.
 *
 * Gates are never expanded to 2^n x 2^n matrices (the paper's Eq. 2 caching): the planner groups
 * consecutive gates touching at most k qubits into one pass over the state (the circuit splitting
 * of Sec. "Circuit Splitting"), and each 2x2 is formed on the device from the angle.
 *
 * Conventions for every call below:
 *   - status: 0 = QSIM_OK, negative = error; the message is in qsim_last_error() (thread-local).
 *   - "d_" pointers are DEVICE pointers owned by the caller; host pointers are marked "h_".
 *   - all device work is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream) and is
 *     asynchronous; the status only reports validation and enqueue errors. Device-side failures
 *     (a bounded wait that timed out) are reported by qsim_sync_status().
 *   - scalar type: QSIM_C64 -> state complex64, params/inputs float32; QSIM_C128 -> complex128,
 *     params/inputs float64. <Z>, grad_out and all gradients are float64 in both modes.
 */
#ifndef QSIM_PUBLIC_API_H_
#define QSIM_PUBLIC_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gate types (Sec. "Gate Matrix Caching" names R_x; RY/RZ/H/X/CNOT/CZ follow the textbook definitions). */
enum { QSIM_RX = 0, QSIM_RY = 1, QSIM_RZ = 2, QSIM_H = 3, QSIM_X = 4, QSIM_CNOT = 5, QSIM_CZ = 6 };

/* One gate: {type, targets, controls, param index}.
 *   single-qubit gates: targets[0] = qubit, others -1.
 *   CNOT: controls[0] = control, targets[0] = target.   CZ: controls[0], targets[0] (symmetric).
 *   param >= 0: index into the trainable parameter vector (shared by the batch), below 2^24;
 *   param == -1: no parameter (H, X, CNOT, CZ);
 *   param <= -2: encoded input, column (-2 - param) of the (B, n_inputs) input matrix, below 2^20. */
typedef struct {
  int32_t type;
  int32_t targets[2];
  int32_t controls[2];
  int32_t param;
} qsim_gate;

enum {
  QSIM_OK = 0,
  QSIM_ERR_ARG = -1,        /* null pointer, bad size or option                       */
  QSIM_ERR_QUBIT = -2,      /* qubit index out of range or control == target          */
  QSIM_ERR_PARAM = -3,      /* parameter field inconsistent with the gate type        */
  QSIM_ERR_GATE = -4,       /* unknown gate type                                      */
  QSIM_ERR_NO_FORWARD = -5, /* backward without a preceding forward on this plan      */
  QSIM_ERR_OOM = -6,        /* workspace allocation failed or exceeds the budget      */
  QSIM_ERR_CUDA = -7,       /* a CUDA call failed (message has the CUDA error string) */
  QSIM_ERR_TIMEOUT = -8,    /* a bounded device-side wait gave up                     */
  QSIM_ERR_UNSUPPORTED = -9 /* size outside what the library supports                 */
};

enum { QSIM_C64 = 0, QSIM_C128 = 1 };
enum { QSIM_FUSED = 0, QSIM_PER_GATE = 1 };

typedef struct {
  int32_t k;                 /* max qubits local to one fused pass (tile = 2^k amplitudes); 0 = default
                                (12 complex64, 11 complex128); at most 13 for complex64, 11 for complex128,
                                and at most 8 more than the register bits of either direction (256
                                threads per tile) */
  int32_t dtype;             /* QSIM_C64 or QSIM_C128 */
  int32_t mode;              /* QSIM_FUSED (default) or QSIM_PER_GATE (one kernel per gate: the plain baseline) */
  int32_t contiguous_bits;   /* low index bits local in every pass (runs of 2^c amplitudes); 0 = default (4) */
  int32_t checkpoint_passes; /* >0: backward restarts psi from a stored forward state every this many passes;
                                0: no checkpoints; -1: choose from mem_budget_bytes */
  int32_t sample_block;      /* >0: samples per launch group; every pass runs over one group before the next
                                group starts (keeps a group's states in L2); 0 = the whole batch per launch */
  int32_t bwd_reg_bits;      /* amplitudes per thread in backward phases = 2^bits (0 = default: 5 for complex64
                                single-circuit plans, 4 for complex64 multi-circuit plans, 3 for complex128);
                                more bits mean fewer shared-memory round trips per pass */
  int32_t fwd_reg_bits;      /* amplitudes per thread in forward phases = 2^bits (0 = default: 5 for complex64,
                                4 for complex128); fewer bits mean fewer registers and more resident warps */
  int32_t weight_remap;      /* 1: every trainable angle enters as theta' = pi * tanh(theta) (quantum weight
                                remapping, Sec. "Additional Optimizations"), dparams are dL/dtheta through
                                that map; inputs are used as given. 2: input angles are remapped as well
                                (dinputs likewise; single-circuit plans, used by qsim_landscape).
                                0: angles as given */
  int32_t graph;             /* multi-circuit plans: capture each direction's launch sequence in a CUDA graph and
                                replay it while the caller's buffers are unchanged (0 = plain launches) */
  int32_t max_regs;          /* >0: registers per thread of the pass kernels capped so that at least
                                65536 / (threads per tile * max_regs) CTAs fit on an SM (more resident warps,
                                possibly a few spills); 0: the compiler's choice */
  int32_t rotate_low_bits;   /* 1: index bits 1..contiguous_bits-1 are handed between passes to qubits needed
                                next (a qubit remap folded into each pass's store; fewer passes when
                                k >= 2 * contiguous_bits + 2, but each pass holds more gates and phases);
                                0 (default): the contiguous_bits lowest bits hold the same qubits in every
                                pass. Multi-circuit plans always keep them fixed */
  int32_t pauli_frame;       /* 1: every rotation runs the tangent form only; a cotangent-form rotation equals the
                                tangent form with coefficient -cot(theta/2) followed by -iP, and those Paulis are
                                carried per sample as a Pauli frame F (stored states are F^dag times the true
                                state; the returned states have F applied). Fused single-circuit plans only.
                                0 (default): both forms, chosen per rotation and sample at run time */
  int32_t scalar_bwd;        /* complex64 pauli_frame plans: 0 (default) the backward pass kernels hold psi and lambda
                                as register pairs (Re psi, Re lambda), (Im psi, Im lambda) and update both with one
                                packed FP32x2 FMA; 1: separate scalar FMAs. Other plans ignore it; 0 or 1 */
  int32_t product_prefix;    /* 1: the single-qubit gates that act on a qubit before its first two-qubit gate are
                                merged, per sample, into that qubit's state phi_q = G_m...G_1|0> (FP64); the
                                first fused pass writes the product state of all phi_q instead of starting from
                                |0...0> and applying them, and their gradients come from one contraction of the
                                adjoint state with the other qubits' phi (Sec. "Gate Matrix Caching": the
                                embedding's per-qubit matrices; the paper merges partial matrices, here the
                                merged per-qubit gates act on |0> and collapse to a vector). A forward given an
                                initial state runs an internal plan without it. Fused single-circuit plans only;
                                0 (default): every gate runs inside the fused passes */
  int32_t split_diagonal;    /* pauli_frame plans: 0 (default) a run of consecutive diagonal ops (RZ, CZ) in a register
                                phase is applied as one complex factor per amplitude, built from per-bit factors,
                                and in the backward all of the run's RZ gradients come from one pass over the
                                amplitudes (Im(conj(lambda) psi) is unchanged through diagonal ops up to a known
                                real factor); 1: every op on its own. 0 or 1 */
  int32_t large_circuit_qubits; /* multi-circuit plans: a circuit of at least this many qubits runs as its own
                                single-circuit fused plan (Pauli frame, product prefix, merged diagonal runs) on its
                                slices of the caller's buffers, right after the queue launch; the queue keeps the
                                smaller circuits. 0 = default (18); < 0: every circuit in the queue. Single-circuit
                                plans ignore it */
  int32_t reserved;          /* must be 0 */
  int64_t mem_budget_bytes;  /* workspace limit used when checkpoint_passes == -1 (0 = unlimited) */
} qsim_plan_opts;

typedef struct {
  int32_t n_qubits, n_gates, n_params, n_inputs;
  int32_t n_passes, k, dtype, mode;
  int32_t n_checkpoints;     /* stored forward states the backward restarts from (0 = none) */
  int32_t reserved;
  int64_t workspace_bytes;   /* device bytes held by the plan for the last batch size used */
} qsim_plan_info;

typedef struct qsim_plan_s* qsim_plan_t;

/* Fill `opts` with the defaults (k = 12, complex64, fused, c = 4, no checkpoints). */
void qsim_default_opts(qsim_plan_opts* opts);

/* Build a plan (host only; no device memory is touched until the first forward).
 *   h_gates: n_gates gate records (host memory, copied); n_qubits in [1, 34].
 *   opts: NULL for defaults. On success *out owns the plan (free with qsim_plan_destroy).
 *   Errors: QSIM_ERR_ARG / _QUBIT / _PARAM / _GATE with a message naming the first bad gate. */
int qsim_plan(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits,
              const qsim_plan_opts* opts, qsim_plan_t* out);

/* Sizes and schedule summary of a plan. */
int qsim_plan_info_get(qsim_plan_t plan, qsim_plan_info* info);

/* JSON description of the pass schedule (local qubits, tile-bit positions, register phases and
 * the gate indices of every op), for inspection and tests. Ops of kind "scale" (gate -1) are the
 * range-control rescale ops the planner inserts after every 48 rotations / Hadamards of a pass
 * (which holds at most 256 of them). Writes at most `cap` bytes including
 * the terminating NUL into h_buf (which may be NULL when cap == 0) and the full length + 1 into
 * *needed. */
int qsim_plan_describe(qsim_plan_t plan, char* h_buf, size_t cap, size_t* needed);

/* The fused pass kernels of a plan are specialised per pass structure and compiled with NVRTC for
 * sm_103a the first time a plan is used (compiled binaries are cached on disk, keyed by the source).
 * qsim_plan_kernel_source returns that program text (same buffer convention as qsim_plan_describe);
 * qsim_plan_compile_kernels compiles it (or finds it in the cache) without touching a GPU. */
int qsim_plan_kernel_source(qsim_plan_t plan, char* h_buf, size_t cap, size_t* needed);
int qsim_plan_compile_kernels(qsim_plan_t plan);

/* Physical amplitude indices (within one sample) of the 2^k elements of tile `tile` of pass
 * `pass`, in tile order, in the qubit layout that pass reads (tile bit j <-> physical bit L_j of
 * that layout; pass 0 reads the canonical layout, and a pass writes the layout the next one reads):
 * the gather map of that pass. h_out must hold 2^k int64 values. Host only. */
int qsim_tile_index_map(qsim_plan_t plan, int32_t pass, int64_t tile, int64_t* h_out);

/* Forward pass.
 *   d_params:  (n_params,) float32/float64 trainable angles (may be NULL if n_params == 0)
 *   d_inputs:  (batch, n_inputs) float32/float64 encoded inputs (NULL if n_inputs == 0)
 *   d_init:    (batch, 2^n) complex initial states, or NULL for |0...0> in every sample
 *   d_states:  (batch, 2^n) complex output: the final states, canonical qubit order (may equal d_init)
 *   d_z:       (batch, n) float64 output <Z_i>_b
 * Intermediate states live in the plan's workspace (and checkpoints); only the last pass writes
 * d_states. The plan remembers d_params, d_inputs and d_states for the backward: they must stay
 * unchanged until qsim_backward has been enqueued. Workspace is (re)allocated on `stream` when the
 * batch size changes. Errors: QSIM_ERR_ARG for NULL or misaligned buffers, QSIM_ERR_UNSUPPORTED when
 * batch x 2^n exceeds 2^40 amplitudes (also for qsim_expval_z and qsim_multi_forward), QSIM_ERR_OOM
 * when the workspace does not fit. */
int qsim_forward(qsim_plan_t plan, const void* d_params, const void* d_inputs, int32_t batch,
                 const void* d_init, void* d_states, double* d_z, void* stream);

/* Adjoint backward of the last forward on this plan.
 *   d_grad_out: (batch, n) float64 dL/d<Z_i>_b
 *   d_dparams:  (n_params,) float64 output dL/dparams (summed over the batch), may be NULL
 *   d_dinputs:  (batch, n_inputs) float64 output dL/dinputs, may be NULL
 * Reads the saved final states (not modified); uses the plan's own workspace for psi and lambda. */
int qsim_backward(qsim_plan_t plan, const double* d_grad_out, double* d_dparams, double* d_dinputs,
                  void* stream);

/* Synchronize `plan`'s last stream and return its status: QSIM_OK, or QSIM_ERR_CUDA when the stream
 * reports a CUDA error (single-circuit kernels have no device-side waits; the bounded waits of the
 * multi-circuit queue report QSIM_ERR_TIMEOUT through qsim_multi_sync_status). */
int qsim_sync_status(qsim_plan_t plan);

/* Standalone measurement layer: <Z_i>_b of arbitrary states (the same reduction the fused path
 * runs in its last pass). d_states (batch, 2^n) complex of `dtype`; d_z (batch, n) float64.
 * Allocates its partial-sum scratch on `stream` (stream-ordered) and frees it after use. */
int qsim_expval_z(const void* d_states, int32_t batch, int32_t n_qubits, int32_t dtype, double* d_z,
                  void* stream);

/* Per-pass timing: from now on CUDA events are recorded on the launch stream around every pass of
 * the next `depth` forward and backward calls (a ring of `depth` event sets); depth == 0 turns it
 * off. Synchronizes the plan's last stream and clears earlier records. */
int qsim_set_profiling(qsim_plan_t plan, int32_t depth);

/* Per-pass durations in milliseconds, SUMMED over the recorded calls (at most `depth`): h_fwd_ms and
 * h_bwd_ms hold `cap` floats each, indexed by pass (either may be NULL). h_n_calls[0..1] receives
 * the number of forward and backward calls summed (may be NULL). Waits for the recorded events. */
int qsim_read_profile(qsim_plan_t plan, float* h_fwd_ms, float* h_bwd_ms, int32_t cap, int32_t* n_passes,
                      int32_t* h_n_calls);

/* Number of CUDA kernels this library has launched in the calling process so far. */
int64_t qsim_kernel_launches(void);

/* <Z_i>_b like qsim_expval_z, but allocating nothing: for callers that cannot call cudaMalloc, for
 * example code whose device memory is entirely owned by another allocator (a framework that reserves
 * the GPU's memory up front) or a steady-state loop that must not let a library call allocate, fail
 * for lack of memory, or synchronise the device. The paper has no counterpart; this is an interface
 * convenience of this library.
 *   The partial sums go to one fixed device array inside the library (4 MiB: at most 524288 partial
 *   sums, i.e. batch * 2^(n-12) * 13 <= 524288 for n >= 12, batch * (n+1) <= 524288 below). Larger
 *   requests return QSIM_ERR_UNSUPPORTED and leave d_z untouched; use qsim_expval_z for them.
 *   Every GPU that loads the library holds that array until the process exits.
 *   The first call on each device looks up the array's device address (a set-up with that device
 *   current, cached per device and keyed on the current context, so the first call after the
 *   device's context is re-created, e.g. after cudaDeviceReset, looks it up again); make the first
 *   call on a device, and the first after such a reset, before any stream capture.
 *   All calls share the array and it keeps the last call's contents: calls that can overlap on the
 *   GPU (other streams, other host threads) race and must be ordered by the caller. No entry of the
 *   array has to start at zero (each call writes every partial it reads).
 *   Arguments, layout and errors otherwise as qsim_expval_z. */
int qsim_expval_z_noalloc(const void* d_states, int32_t batch, int32_t n_qubits, int32_t dtype, double* d_z,
                          void* stream);

/* ------------------------------------------------------------------------------------------------
 * Several circuits of uneven size in one persistent launch per direction (the batched training of
 * many hybrid models; Sec. "Hybrid Machine Learning"'s circuits, each planned as above).
 *
 * Every circuit gets its own k-local passes; a device work queue lists tile jobs in rounds (pass 0 of
 * every circuit, then pass 1, ...). One persistent kernel per direction claims jobs with an atomic
 * counter, waits until the previous pass of the same circuit is complete (a bounded wait: it gives
 * up after a time limit and reports QSIM_ERR_TIMEOUT through qsim_multi_sync_status), runs the job's
 * specialised pass code and signals completion. Circuits have up to 30 qubits; every circuit uses
 * the same batch size B; initial states are |0...0>.
 *
 * Buffers are the per-circuit blocks concatenated in circuit order (offsets: qsim_multi_offsets):
 *   params (sum P_c) float32/float64 | inputs: circuit c's (B, n_inputs_c) block | states: circuit c's
 *   (B, 2^n_c) complex block | z, grad_out: circuit c's (B, n_c) float64 block | dparams, dinputs as
 *   params, inputs (float64). */
typedef struct qsim_multi_s* qsim_multi_t;

int qsim_multi_plan(const qsim_gate* const* h_gate_lists, const int32_t* h_n_gates, const int32_t* h_n_qubits,
                    int32_t n_circuits, const qsim_plan_opts* opts, const int32_t* h_k, qsim_multi_t* out);
/*   h_k: NULL (every circuit uses opts->k), or one k per circuit (host, n_circuits entries, each in
 *   [1, 11] for complex64 / [1, 10] for complex128: one below the single-circuit maximum, so that the
 *   queue kernels, which hold every pass structure, stay small enough for four CTAs per SM), e.g. from
 *   qsim_multi_autotune. opts->k is clamped to the same maximum. */

/* Element offsets of every circuit's block for batch size `batch`; each array (n_circuits + 1
 * entries, the last = total) may be NULL. */
int qsim_multi_offsets(qsim_multi_t plan, int32_t batch, int64_t* h_param_off, int64_t* h_input_off,
                       int64_t* h_state_off, int64_t* h_z_off);

int qsim_multi_forward(qsim_multi_t plan, const void* d_params, const void* d_inputs, int32_t batch,
                       void* d_states, double* d_z, void* stream);
int qsim_multi_backward(qsim_multi_t plan, const double* d_grad_out, double* d_dparams, double* d_dinputs,
                        void* stream);

/* Synchronize the last stream; QSIM_OK or QSIM_ERR_TIMEOUT if a queue wait gave up (status cleared).
 * Once one wait has given up, every later queue job that would wait skips its work instead (its
 * results are not valid), in this call and in later calls until this function has read and cleared
 * the status: so a lost dependency costs one time limit, not one per pass. */
int qsim_multi_sync_status(qsim_multi_t plan);

/* Queue statistics: circuits, work items per direction, distinct specialised pass codes per direction. */
int qsim_multi_info(qsim_multi_t plan, int32_t* n_circuits, int64_t* n_items_fwd, int64_t* n_items_bwd,
                    int32_t* n_kernels_fwd, int32_t* n_kernels_bwd);

/* Resources of the two persistent queue kernels (index 0 forward, 1 backward), known after the
 * first forward: resident CTAs per SM, registers per thread, dynamic shared memory per CTA. One
 * queue kernel holds every pass structure of its direction, so these are the maxima over them. */
int qsim_multi_kernel_info(qsim_multi_t plan, int32_t* h_ctas_per_sm, int32_t* h_regs, int64_t* h_smem);

/* Test hook for the bounded waits: the completion of queue item `withhold_item` (-1 = none) is never
 * signalled, and waits give up after timeout_ns (<= 0: the default of 4 s). */
int qsim_multi_set_test_hooks(qsim_multi_t plan, int64_t withhold_item, int64_t timeout_ns);

void qsim_multi_destroy(qsim_multi_t plan);

/* Free the plan and its device workspace (synchronizes the plan's last stream). NULL is a no-op. */
/* OpenQASM 2.0 import (the paper's simulator exchanges circuits through OpenQASM, Sec. "API").
 * `text`: a NUL-terminated program using OPENQASM 2.x; include "qelib1.inc"; qreg / creg
 * declarations (quantum registers are concatenated in declaration order into qubits 0..n-1);
 * barrier and measure (ignored: results are <Z_i>); and the gates h, x, id, rx(a), ry(a), rz(a),
 * cx (CX), cz on qubits reg[i] or whole registers (broadcast). Angles are expressions of decimal
 * literals, pi, + - * / and parentheses. Every rotation gets its own parameter index, in program
 * order, and its angle is written to h_params[index]; no gate is input-encoded.
 * Outputs (host): *n_gates, *n_params, *n_qubits always; h_gates (cap_gates records) and h_params
 * (cap_params doubles) when not NULL (NULL = query the counts only).
 * Errors: QSIM_ERR_ARG with "line L: ..." for anything outside the subset, or arrays too small. */
int qsim_parse_qasm(const char* text, qsim_gate* h_gates, int32_t cap_gates, int32_t* n_gates, double* h_params,
                    int32_t cap_params, int32_t* n_params, int32_t* n_qubits);

/* OpenQASM 2.0 export of a gate list with concrete angles: h_params[param] for trainable rotations,
 * h_inputs[column] (one sample's input row) for input-encoded ones (either may be NULL when unused).
 * Writes one register q[n_qubits] and one statement per gate (angles with 17 significant digits, so
 * qsim_parse_qasm reads back the same doubles). *needed = bytes including the NUL; buf (cap bytes)
 * may be NULL to query. Errors: QSIM_ERR_ARG / QSIM_ERR_QUBIT / QSIM_ERR_PARAM for malformed gates. */
int qsim_export_qasm(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, const double* h_params,
                     const double* h_inputs, char* buf, size_t cap, size_t* needed);

/* Gradient landscape (App. "Barren Plateaus": the absolute gradient of every parameter at different
 * rotations of that parameter, the others constant, with and without weight remapping). For every
 * trainable parameter k and value v: dL/dtheta_k at theta = base with theta_k = values[v], where
 * L = sum_i weights[i] <Z_i>. One batched forward + adjoint backward over n_params * n_values
 * parameter vectors: the circuit's trainable parameters become per-sample angles (input columns),
 * so the batch dimension carries the vectors. The circuit must not have input-encoded gates.
 *   opts: dtype, k, ... as for qsim_plan (fused mode); weight_remap 1 sweeps the raw weights w
 *         (angle = pi * tanh(w)) and returns dL/dw.
 *   d_base (n_params,), d_values (n_values,): float32 (complex64) / float64 (complex128), device.
 *   d_weights (n_qubits,) float64, device.  d_grid (n_params, n_values) float64, device, written.
 *   d_z: NULL, or (n_params * n_values, n_qubits) float64: <Z> of every evaluated vector, row k*V+v.
 * The plan (compiled kernels, workspace) and the buffers for n_params * n_values states are kept for the
 * last 4 distinct circuits (gate list, qubits, options, n_values), so repeated sweeps skip planning,
 * kernel loading and allocation; the work is enqueued on `stream` (asynchronous; a later call on
 * another stream waits for it). qsim_landscape_clear_cache releases them. Errors: those of
 * qsim_plan / qsim_forward / qsim_backward, QSIM_ERR_PARAM (input-encoded gates, no parameters),
 * QSIM_ERR_OOM. */
int qsim_landscape(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, const qsim_plan_opts* opts,
                   const void* d_base, const void* d_values, int32_t n_values, const double* d_weights,
                   double* d_grid, double* d_z, void* stream);

/* Release the plans and buffers qsim_landscape keeps (waits for their last use). */
void qsim_landscape_clear_cache(void);

/* Tile-size autotuner (the fused pass's k). Plans the circuit with *opts for each candidate k in
 * {max_k - 2, max_k - 1, max_k} (max_k = 13 complex64, 11 complex128), runs one untimed forward
 * (+ backward when with_backward != 0; this also compiles the kernels) and then `reps` timed calls
 * on zero-filled scratch buffers of `batch` samples that it allocates and frees itself (run time
 * does not depend on the values), and writes to opts->k the largest candidate whose time is within
 * 2 % of the fastest. n_qubits <= max_k: opts->k = n_qubits (one pass), and when opts leaves
 * fwd_reg_bits and bwd_reg_bits at 0 the candidates are the amplitudes per thread in the register phases
 * and the Pauli frame: 2^5 and 2^4 (2^4 and 2^3 for complex128) with the frame and then without it when
 * opts->pauli_frame is 1, else 2^5, 2^4 and 2^3 without; the backward's phases follow the forward's
 * when with_backward != 0. The fastest is written to opts->fwd_reg_bits (/ bwd_reg_bits; left at 0
 * when the largest count wins) and opts->pauli_frame. h_ms: NULL or 4 floats, mean ms per call of each
 * candidate in that order (-1 when not run; a circuit of several passes has 3 candidates). Synchronises `stream`. Errors: those of qsim_plan / qsim_forward /
 * qsim_backward, QSIM_ERR_OOM for scratch. In the paper the maximum group width is a fixed
 * argument of the greedy splitter (Sec. "Circuit Splitting", typically 3 to 6 qubits); here the
 * width is measured per circuit and batch. */
int qsim_autotune(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, int32_t batch,
                  int32_t with_backward, int32_t reps, qsim_plan_opts* opts, float* h_ms, void* stream);

/* Per-circuit k for qsim_multi_plan: the qsim_autotune measurement (candidates up to the
 * multi-circuit maximum: 11 qubits complex64, 10 complex128) on the first circuit of every distinct
 * qubit count (same batch, opts as the base), the result copied to every circuit of that count.
 * h_k: n_circuits int32 (host, written). */
int qsim_multi_autotune(const qsim_gate* const* h_gate_lists, const int32_t* h_n_gates, const int32_t* h_n_qubits,
                        int32_t n_circuits, int32_t batch, int32_t with_backward, int32_t reps,
                        const qsim_plan_opts* opts, int32_t* h_k, void* stream);

void qsim_plan_destroy(qsim_plan_t plan);

/* Test hook (host only): the Pauli-frame walk of pauli_frame plans over one op list. types / q0 (target)
 * / q1 (control, -1 for single-qubit gates) as in qsim_gate, cot[i] = 1 for a rotation in the cotangent
 * form. Writes sigma[i] = -1 where the frame anticommutes with rotation i's Pauli (else +1) and the final
 * frame F = i^k prod_q X_q^(x bit q) Z_q^(z bit q). QSIM_ERR_ARG on NULL arguments. */
int qsim_frame_walk_host(const int32_t* types, const int32_t* q0, const int32_t* q1, const uint8_t* cot,
                         int32_t n_ops, int8_t* sigma, uint64_t* x, uint64_t* z, int32_t* k);

/* Message of the last failed call on this thread ("" if none). */
const char* qsim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_PUBLIC_API_H_ */
