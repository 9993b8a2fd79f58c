// Host planner: validation, k-local fusion into passes, register phases and smem layouts.
//
// Sec. "Circuit Splitting" of the paper splits a circuit into groups of gates on at most a few qubits and
// runs each group as one operation over the reshaped state. Here the group size is k (a tile of
// 2^k amplitudes in shared memory), groups are chosen greedily in gate order while keeping the
// per-wire order, and each group becomes one pass of a CUDA kernel.
#pragma once
#include <string>
#include <vector>

#include "plan_types.h"
#include "../../include/qsim.h"

namespace qsim {

struct Gate {
  int type, t0, t1, c0, c1, param;
};

struct PassPlan {
  DevPass dev{};                     // forward: register phases with the forward register count
  DevPass devb{};                    // backward: same tile, phases for the backward register count
  std::vector<int> local_qubits;     // qubits held in the tile (by tile bit order)
  std::vector<int> gates;            // gate indices in execution order
};

struct Schedule {
  int n = 0, k = 0, R = 0, Rb = 0, c = 0, dtype = 0, mode = 0;
  int max_regs = 0;                  // register cap of the pass kernels (0: none)
  bool pauli_frame = false;          // rotations run the tangent form only (cotangent Paulis in a frame)
  bool packed_bwd = false;           // backward holds (psi, lambda) register pairs, packed FP32x2 updates
  bool merge_diag = false;           // runs of diagonal ops become one factor per amplitude (tangent form only)
  // product-state prefix: per qubit, the single-qubit gates before its first two-qubit gate (in order),
  // merged into phi_q and taken out of the fused passes
  bool has_prefix = false;
  std::vector<std::vector<int>> prefix;
  int n_params = 0, n_inputs = 0;
  std::vector<Gate> gates;
  std::vector<PassPlan> passes;
  std::vector<DevPhase> phases;
  std::vector<DevOp> ops;
  std::vector<DevLayout> layouts;
  // gradient bookkeeping: every parametric gate occurrence, in gate order
  std::vector<int> grad_gate;        // gate index
  std::vector<int> grad_pass;        // pass holding it
  std::vector<int> grad_slot;        // slot within that pass
  int64_t total_gslots = 0;          // sum over passes of n_gslots
};

// Returns QSIM_OK or an error code with `err` set.
int validate_gates(const qsim_gate* g, int n_gates, int n, std::vector<Gate>& out, int& n_params,
                   int& n_inputs, std::string& err);

// Build the full schedule. R is the register bits per phase (<= kMaxR).
// rotate_low: hand the coalescing bits 1..c-1 between passes (fewer passes; single-circuit plans).
// Multi-circuit plans keep them fixed: every circuit then repeats a few pass structures, and the queue
// kernel links one function per distinct structure.
int build_schedule(const std::vector<Gate>& gates, int n, const qsim_plan_opts& o, int R_fwd, int R_bwd,
                   Schedule& s, std::string& err, bool rotate_low = true);

std::string describe_schedule(const Schedule& s);

// Element index within a sample of tile element e of tile t in pass p.
int64_t tile_element_index(const DevPass& p, int64_t tile, int64_t e);

}  // namespace qsim
