// Plain structs shared by the host planner and the CUDA kernels (no CUDA headers here).
//
// A fused pass works on tiles of 2^k amplitudes of one sample: tile bit j of an element index is
// physical index bit L[j]; the other (n-k) physical bits ("nonlocal", ascending) enumerate the
// tiles of a sample. Inside a CTA the tile sits in shared memory and is processed in register
// phases: in phase p each thread holds 2^R elements that differ in the R tile bits rbit[0..R-1]
// (rbit[0] is always tile bit 0, so pairs of neighbouring amplitudes stay in one 16-byte word),
// and the thread id bits map, in order, onto the remaining tile bits tbit[].
#pragma once
#include <cstdint>

namespace qsim {

constexpr int kMaxTileBits = 16;   // k <= 16
constexpr int kMaxR = 5;           // at most 2^5 amplitudes per thread and array
constexpr int kMaxQubits = 34;
constexpr int kMaxParams = 1 << 24;   // trainable parameter indices per circuit
constexpr int kMaxInputs = 1 << 20;   // encoded input columns per circuit
constexpr long long kMaxAmplitudes = 1LL << 40;   // batch x 2^n of one call (8 TiB of complex64)
// Rotations and Hadamards run unnormalised inside a pass (a tangent or cotangent coefficient, the
// factored cos / sin / 1/sqrt(2) applied later), so each one grows the tile's values by at most
// sqrt(2). A K_SCALE op after every kRescaleEvery of them applies the factors gathered so far: the
// values stay within 2^24 of their true size (2^48 for the backward's lambda-psi products), far
// inside the FP32 range. kMaxScaledOpsPerPass bounds the specialised kernel's length.
constexpr int kRescaleEvery = 48;
constexpr int kMaxScaledOpsPerPass = 256;

// Op kinds understood by the pass kernels. "_R" = operand is a register bit (a/b = register index),
// "_T" = operand is a thread bit (a/b = tile bit index, value taken from the thread's base index).
enum OpKind : uint8_t {
  K_RY_R = 0,   // rotation about Y on register bit a
  K_RX_R,       // rotation about X on register bit a
  K_RZ_R,       // rotation about Z (diagonal) on register bit a
  K_H_R,        // Hadamard on register bit a
  K_X_R,        // Pauli X on register bit a
  K_RZ_T,       // rotation about Z on thread bit a
  K_CNOT_RR,    // CNOT target register a, control register b
  K_CNOT_RT,    // CNOT target register a, control thread bit b
  K_CZ_RR,      // CZ on register bits a, b
  K_CZ_RT,      // CZ on register bit a and thread bit b
  K_CZ_TT,      // CZ on thread bits a, b
  K_SCALE,      // multiply every amplitude of the tile by the op's per-sample value (range control)
  K_NUM_KINDS
};

struct DevOp {
  uint8_t kind;
  uint8_t a;
  uint8_t b;
  uint8_t rot;      // 1: parametric rotation (has a coefficient and a gradient)
  int32_t gate;     // index into the plan's gate list (-1 for K_SCALE)
  int32_t gslot;    // gradient slot within the pass (-1 if none)
};

struct DevPhase {
  uint8_t rbit[kMaxR];          // tile bits held in registers (rbit[0] == 0)
  uint8_t tbit[kMaxTileBits];   // tile bits of thread id bits 0.. (ascending)
  uint8_t n_tbits;
  uint8_t pad[2];
  int32_t op_begin, op_end;     // ops [op_begin, op_end) of the pass-global op array
};

// Shared-memory layout between two phases: element e lives at word e ^ (XOR of m[j] over set
// tile bits j >= 4); m[j] only touches the bank window so the map is a bijection.
struct DevLayout {
  uint8_t m[kMaxTileBits];
};

struct DevPass {
  int32_t k, R, n_phases, phase0;   // phases [phase0, phase0 + n_phases) of the plan phase array
  int32_t n_ops, op0;               // ops [op0, op0 + n_ops)
  int32_t n_gslots, lay0;           // gradient slots; layouts [lay0, lay0 + n_phases + 1)
  int32_t n_nonlocal, pad0;
  int64_t tiles_per_sample;
  int64_t gpart_offset;             // offset of this pass's gradient partials (per batch layout)
  // Layouts: the pass reads its input in layout pi_p and writes its output in pi_{p+1} (logical qubit
  // -> physical index bit; pi_0 and the last output layout are canonical, qubit q at bit n-1-q).
  uint8_t L[kMaxTileBits];          // tile bit j: physical bit in the input layout
  uint8_t nonlocal[40];             // tile-index bit i (a qubit outside the tile): input-layout bit
  uint8_t Lo[kMaxTileBits];         // tile bit j: physical bit in the output layout
  uint8_t nonlocal_o[40];           // tile-index bit i: output-layout bit
  uint8_t Q[kMaxTileBits];          // logical qubit of tile bit j
  uint8_t QN[40];                   // logical qubit of tile-index bit i
};

}  // namespace qsim
