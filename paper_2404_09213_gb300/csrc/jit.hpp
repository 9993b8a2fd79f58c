// Specialised fused-pass kernels compiled at plan time (see jit.cpp).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "planner.hpp"

namespace qsim {

// Host mirror of qj::Args in jit_device.cuh (same field order and types).
struct JitArgs {
  const void* in;
  void* out;
  const void* lam_in;
  void* lam_out;
  const void* cfp;
  const uint8_t* fmp;
  const void* scale;
  double* zpart;
  double* gpart;
  const double* grad_out;
  const void* phi;
  double* ppart;
  int64_t tps;
  int64_t gpart_offset;
  int64_t ntiles;             // tiles of the launch (set by jit_launch)
  int n_nonlocal, n, B, b0;   // b0: first sample of this launch (tiles cover samples b0, b0+1, ...)
  uint8_t L[16];
  uint8_t nonlocal[40];
  uint8_t Lo[16];
  uint8_t nonlocal_o[40];
  uint8_t Q[16];
  uint8_t QN[40];
};
static_assert(sizeof(JitArgs) == 304, "JitArgs must match qj::Args");

// Layouts of a pass into its kernel arguments. The forward reads the pass's input layout and writes
// its output layout; the backward undoes the pass, so it reads the output layout and writes the input.
inline void set_bits(JitArgs& a, const DevPass& d, bool bwd) {
  for (int j = 0; j < d.k; j++) {
    a.L[j] = bwd ? d.Lo[j] : d.L[j];
    a.Lo[j] = bwd ? d.L[j] : d.Lo[j];
    a.Q[j] = d.Q[j];
  }
  for (int j = 0; j < d.n_nonlocal; j++) {
    a.nonlocal[j] = bwd ? d.nonlocal_o[j] : d.nonlocal[j];
    a.nonlocal_o[j] = bwd ? d.nonlocal[j] : d.nonlocal_o[j];
    a.QN[j] = d.QN[j];
  }
}

struct JitKernel {
  void* fn = nullptr;   // cudaKernel_t
  size_t smem = 0;
  int nthr = 0;
  int64_t max_blocks = 0;   // resident blocks (persistent queue kernels only)
  int per_sm = 0, regs = 0; // resident blocks per SM and registers per thread (queue kernels only)
  int groups = 1;           // tiles per CTA (single-circuit kernels of tiles with fewer than 32 threads)
};

struct JitPlan {
  std::vector<JitKernel> fwd, bwd;   // one per pass
  std::vector<cudaLibrary_t> libs;   // one per distinct kernel
};

int fwd_R_for(int k, int dtype);
int bwd_R_for(int k, int dtype);
int max_k_for(int dtype);
int default_k_for(int dtype);
int multi_max_k_for(int dtype);

// Persistent multi-circuit queue kernels (one per direction) linked from relocatable pass functions.
struct JitMulti {
  JitKernel fwd, bwd;                       // max_blocks = resident blocks (persistent grid)
  std::vector<std::vector<int>> kind;       // [circuit][2*pass + dir] -> switch case
  std::vector<size_t> smem_group[2];
  int n_kinds[2] = {0, 0};
  std::vector<cudaLibrary_t> libs;
};
int jit_build_multi(const std::vector<const Schedule*>& scheds, int cta_f, int cta_b, JitMulti& jm, std::string& err);
void jit_free_multi(JitMulti& jm);

// Full NVRTC program text and the kernel name of every pass (forward, backward).
std::string jit_generate(const Schedule& s, std::vector<std::string>& fwd_names, std::vector<std::string>& bwd_names);
// Shared-memory bytes of one tile group; cta: the queue kernel's CTA size (0: single-circuit kernel).
// With a register cap in the plan (s.max_regs) a single-circuit backward sizes its gradient partials so
// that as many CTAs fit in shared memory as in the registers.
size_t jit_smem_bytes(const Schedule& s, const DevPass& d, bool bwd, int cta = 0);
// A single-circuit pass kernel whose tile has fewer than 32 threads runs several tiles per CTA: the
// CTA's threads (0: one tile per CTA), and the shared memory of such a launch's CTA.
int single_cta(const DevPass& d);
size_t single_smem_bytes(const Schedule& s, const DevPass& d, bool bwd);
// NVRTC-compile (or fetch from the on-disk cache) the plan's kernels; host only, no CUDA calls.
int jit_compile(const Schedule& s, std::map<std::string, std::string>& cubins, std::vector<std::string>& fwd_names,
                std::vector<std::string>& bwd_names, std::string& err);
int jit_build(const Schedule& s, JitPlan& jp, std::string& err);
void jit_free(JitPlan& jp);
cudaError_t jit_launch(const JitKernel& k, int64_t blocks, const JitArgs& a, cudaStream_t st);

}  // namespace qsim
