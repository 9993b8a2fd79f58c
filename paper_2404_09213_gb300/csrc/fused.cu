// Fused tile passes (forward and adjoint backward).
//
// One CTA owns one tile: the 2^k amplitudes of one sample whose index bits outside the pass's
// local set are fixed (the paper's Section III-B reshape to (rest, group), with the group axis
// kept in shared memory instead of multiplied by a 2^k x 2^k matrix). The tile is brought in with
// 16-byte cp.async copies (runs of 2^c contiguous amplitudes, c >= 1), the pass's gates are applied
// in register phases (each thread holds 2^R amplitudes), and the tile is written back once.
// The forward's last pass also reduces <Z_i> partial sums; the backward's first pass forms
// lambda = (sum_i g_i Z_i) psi on load (Section II-B measurement layer and its adjoint).
#include <cuda_runtime.h>

#include <type_traits>

#include "launch.hpp"
#include "regops.cuh"

namespace qsim {

template <typename T> struct V2T;
template <> struct V2T<float> { using type = float2; };
template <> struct V2T<double> { using type = double2; };

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Dynamic shared memory carve-up (identical on host and device).
struct FwdSmem {
  size_t tile, lays, coef, form, total;
};
__host__ __device__ inline FwdSmem fwd_smem(int k, int n_phases, int n_ops, int el, int sc, int nthr) {
  FwdSmem m;
  const size_t tile = (size_t)el << k, zred = (size_t)nthr * (kMaxR + 2) * sc;
  m.tile = 0;
  m.lays = align_up(tile > zred ? tile : zred, 16);
  m.coef = align_up(m.lays + (size_t)(n_phases + 1) * sizeof(DevLayout), 16);
  m.form = m.coef + (size_t)n_ops * sc;
  m.total = align_up(m.form + n_ops, 16);
  return m;
}
struct BwdSmem {
  size_t psi, lam, lays, coef, red, gq, form, total;
};
__host__ __device__ inline BwdSmem bwd_smem(int k, int n_phases, int n_ops, int n_gslots, int el, int sc, int nthr) {
  BwdSmem m;
  const size_t tile = (size_t)el << k;
  const size_t n_warps = (nthr + 31) / 32;
  m.psi = 0;
  m.lam = tile;
  m.lays = 2 * tile;
  m.coef = align_up(m.lays + (size_t)(n_phases + 1) * sizeof(DevLayout), 16);
  m.red = align_up(m.coef + (size_t)n_ops * sc, 16);
  m.gq = align_up(m.red + n_warps * (size_t)(n_gslots > 0 ? n_gslots : 1) * sc, 16);
  m.form = m.gq + (kMaxTileBits + 2) * sizeof(double);
  m.total = align_up(m.form + n_ops, 16);
  return m;
}

__device__ __forceinline__ void cp_async16(void* smem_ptr, const void* gptr) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// word index of tile element e under layout m (XOR of the masks of e's set tile bits)
__device__ __forceinline__ uint32_t lay_addr(uint32_t e, const uint8_t* m, int k) {
  uint32_t s = e;
#pragma unroll 4
  for (int j = 0; j < k; j++)
    if ((e >> j) & 1u) s ^= m[j];
  return s;
}

__device__ __forceinline__ int64_t deposit_L(uint32_t e, const uint8_t* L, int k) {
  int64_t x = 0;
#pragma unroll 4
  for (int j = 0; j < k; j++)
    if ((e >> j) & 1u) x |= (int64_t)1 << L[j];
  return x;
}

// ------------------------------------------------------------------ op dispatch
template <int R, template <int, int> class OP, typename T>
__device__ __forceinline__ void dispatch1(int a, T* re, T* im, T c, int form) {
  switch (a) {
    case 0: OP<R, 0>::run(re, im, c, form); break;
    case 1: if constexpr (R > 1) OP<R, 1>::run(re, im, c, form); break;
    case 2: if constexpr (R > 2) OP<R, 2>::run(re, im, c, form); break;
    case 3: if constexpr (R > 3) OP<R, 3>::run(re, im, c, form); break;
    case 4: if constexpr (R > 4) OP<R, 4>::run(re, im, c, form); break;
    default: break;
  }
}

template <int R, int A, typename T>
__device__ __forceinline__ void cnot_rr_b(int b, T* re, T* im) {
  switch (b) {
    case 0: if constexpr (A != 0) reg_cnot_rr_t<R, A, 0>(re, im); break;
    case 1: if constexpr (R > 1 && A != 1) reg_cnot_rr_t<R, A, 1>(re, im); break;
    case 2: if constexpr (R > 2 && A != 2) reg_cnot_rr_t<R, A, 2>(re, im); break;
    case 3: if constexpr (R > 3 && A != 3) reg_cnot_rr_t<R, A, 3>(re, im); break;
    case 4: if constexpr (R > 4 && A != 4) reg_cnot_rr_t<R, A, 4>(re, im); break;
    default: break;
  }
}

template <int R, int A, typename T>
__device__ __forceinline__ void cz_rr_b(int b, T* re, T* im) {
  switch (b) {
    case 0: if constexpr (A != 0) reg_cz_rr<R, A, 0>(re, im); break;
    case 1: if constexpr (R > 1 && A != 1) reg_cz_rr<R, A, 1>(re, im); break;
    case 2: if constexpr (R > 2 && A != 2) reg_cz_rr<R, A, 2>(re, im); break;
    case 3: if constexpr (R > 3 && A != 3) reg_cz_rr<R, A, 3>(re, im); break;
    case 4: if constexpr (R > 4 && A != 4) reg_cz_rr<R, A, 4>(re, im); break;
    default: break;
  }
}

template <int R, typename T>
__device__ __forceinline__ void apply_op(const DevOp& op, T* re, T* im, T c, int form, uint32_t tb) {
  switch (op.kind) {
    case K_RY_R: dispatch1<R, RegRY>(op.a, re, im, c, form); break;
    case K_RX_R: dispatch1<R, RegRX>(op.a, re, im, c, form); break;
    case K_RZ_R: dispatch1<R, RegRZ>(op.a, re, im, c, form); break;
    case K_H_R: dispatch1<R, RegH>(op.a, re, im, c, form); break;
    case K_X_R: dispatch1<R, RegX>(op.a, re, im, c, form); break;
    case K_RZ_T: {
      const T s = ((tb >> op.a) & 1u) ? T(-1) : T(1);
      reg_rz_thread<R>(re, im, c, form, s);
      break;
    }
    case K_CNOT_RR:
      switch (op.a) {
        case 0: cnot_rr_b<R, 0>(op.b, re, im); break;
        case 1: if constexpr (R > 1) cnot_rr_b<R, 1>(op.b, re, im); break;
        case 2: if constexpr (R > 2) cnot_rr_b<R, 2>(op.b, re, im); break;
        case 3: if constexpr (R > 3) cnot_rr_b<R, 3>(op.b, re, im); break;
        case 4: if constexpr (R > 4) cnot_rr_b<R, 4>(op.b, re, im); break;
        default: break;
      }
      break;
    case K_CNOT_RT: {
      const bool ctl = (tb >> op.b) & 1u;
      switch (op.a) {
        case 0: reg_cnot_rt<R, 0>(re, im, ctl); break;
        case 1: if constexpr (R > 1) reg_cnot_rt<R, 1>(re, im, ctl); break;
        case 2: if constexpr (R > 2) reg_cnot_rt<R, 2>(re, im, ctl); break;
        case 3: if constexpr (R > 3) reg_cnot_rt<R, 3>(re, im, ctl); break;
        case 4: if constexpr (R > 4) reg_cnot_rt<R, 4>(re, im, ctl); break;
        default: break;
      }
      break;
    }
    case K_CZ_RR:
      switch (op.a) {
        case 0: cz_rr_b<R, 0>(op.b, re, im); break;
        case 1: if constexpr (R > 1) cz_rr_b<R, 1>(op.b, re, im); break;
        case 2: if constexpr (R > 2) cz_rr_b<R, 2>(op.b, re, im); break;
        case 3: if constexpr (R > 3) cz_rr_b<R, 3>(op.b, re, im); break;
        case 4: if constexpr (R > 4) cz_rr_b<R, 4>(op.b, re, im); break;
        default: break;
      }
      break;
    case K_CZ_RT: {
      const bool o = (tb >> op.b) & 1u;
      switch (op.a) {
        case 0: reg_cz_rt<R, 0>(re, im, o); break;
        case 1: if constexpr (R > 1) reg_cz_rt<R, 1>(re, im, o); break;
        case 2: if constexpr (R > 2) reg_cz_rt<R, 2>(re, im, o); break;
        case 3: if constexpr (R > 3) reg_cz_rt<R, 3>(re, im, o); break;
        case 4: if constexpr (R > 4) reg_cz_rt<R, 4>(re, im, o); break;
        default: break;
      }
      break;
    }
    case K_CZ_TT:
      if (((tb >> op.a) & 1u) && ((tb >> op.b) & 1u)) reg_scale<R>(re, im, T(-1));
      break;
    default: break;
  }
}

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <int R, typename T>
__device__ __forceinline__ typename Acc<T>::type op_grad(const DevOp& op, const T* pr, const T* pi, const T* lr,
                                                         const T* li, uint32_t tb) {
  constexpr bool D = std::is_same<T, double>::value;
  using A = typename Acc<T>::type;
#define QSIM_GRAD_CASE(FN, I)                                                  \
  case I:                                                                      \
    if constexpr (R > I) {                                                     \
      if constexpr (D) return (A)FN##_d<R, I>(pr, pi, lr, li);                 \
      else return (A)FN<R, I>(pr, pi, lr, li);                                 \
    }                                                                          \
    break;
  switch (op.kind) {
    case K_RY_R:
      switch (op.a) { QSIM_GRAD_CASE(grad_ry, 0) QSIM_GRAD_CASE(grad_ry, 1) QSIM_GRAD_CASE(grad_ry, 2)
                      QSIM_GRAD_CASE(grad_ry, 3) QSIM_GRAD_CASE(grad_ry, 4) default: break; }
      break;
    case K_RX_R:
      switch (op.a) { QSIM_GRAD_CASE(grad_rx, 0) QSIM_GRAD_CASE(grad_rx, 1) QSIM_GRAD_CASE(grad_rx, 2)
                      QSIM_GRAD_CASE(grad_rx, 3) QSIM_GRAD_CASE(grad_rx, 4) default: break; }
      break;
    case K_RZ_R:
      switch (op.a) { QSIM_GRAD_CASE(grad_rz, 0) QSIM_GRAD_CASE(grad_rz, 1) QSIM_GRAD_CASE(grad_rz, 2)
                      QSIM_GRAD_CASE(grad_rz, 3) QSIM_GRAD_CASE(grad_rz, 4) default: break; }
      break;
    case K_RZ_T: {
      const A s = ((tb >> op.a) & 1u) ? A(-1) : A(1);
      if constexpr (D) return s * (A)grad_imsum_d<R>(pr, pi, lr, li);
      else return s * (A)grad_imsum<R>(pr, pi, lr, li);
    }
    default: break;
  }
#undef QSIM_GRAD_CASE
  return A(0);
}

// ------------------------------------------------------------------ register <-> smem
// Thread's element i (0 <= i < 2^R) is tile element base | deposit(i over rbit). Pairs (i, i+1)
// differ in tile bit 0 and are adjacent words in every layout.
struct PhaseAddr {
  uint32_t tb;          // thread base element (register bits zero)
  uint32_t s_in, s_out; // its word addresses in the read / write layouts
  uint32_t u_in[kMaxR], u_out[kMaxR];   // address increments of register bits
};

template <int R>
__device__ __forceinline__ void phase_addr(PhaseAddr& pa, const DevPhase& ph, const uint8_t* m_in,
                                           const uint8_t* m_out, int k, uint32_t tid) {
  uint32_t tb = 0;
  for (int j = 0; j < ph.n_tbits; j++)
    if ((tid >> j) & 1u) tb |= 1u << ph.tbit[j];
  pa.tb = tb;
  pa.s_in = lay_addr(tb, m_in, k);
  pa.s_out = lay_addr(tb, m_out, k);
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int j = ph.rbit[r];
    pa.u_in[r] = (1u << j) ^ m_in[j];
    pa.u_out[r] = (1u << j) ^ m_out[j];
  }
}

template <int R>
__device__ __forceinline__ uint32_t reg_word(uint32_t base, const uint32_t* u, int i) {
  uint32_t s = base;
#pragma unroll
  for (int r = 1; r < R; r++)
    if ((i >> r) & 1) s ^= u[r];
  return s;
}

template <int R, typename T>
__device__ __forceinline__ void load_regs(const typename V2T<T>::type* tile, uint32_t base, const uint32_t* u,
                                          T* re, T* im) {
#pragma unroll
  for (int i = 0; i < (1 << R); i += 2) {
    const uint32_t w = reg_word<R>(base, u, i);
    if constexpr (std::is_same<T, float>::value) {
      const float4 v = reinterpret_cast<const float4*>(tile)[w >> 1];
      re[i] = v.x; im[i] = v.y; re[i + 1] = v.z; im[i + 1] = v.w;
    } else {
      const double2 a = tile[w], b = tile[w ^ 1u];
      re[i] = a.x; im[i] = a.y; re[i + 1] = b.x; im[i + 1] = b.y;
    }
  }
}

template <int R, typename T>
__device__ __forceinline__ void store_regs(typename V2T<T>::type* tile, uint32_t base, const uint32_t* u,
                                           const T* re, const T* im) {
#pragma unroll
  for (int i = 0; i < (1 << R); i += 2) {
    const uint32_t w = reg_word<R>(base, u, i);
    if constexpr (std::is_same<T, float>::value) {
      reinterpret_cast<float4*>(tile)[w >> 1] = make_float4(re[i], im[i], re[i + 1], im[i + 1]);
    } else {
      tile[w] = make_double2(re[i], im[i]);
      tile[w ^ 1u] = make_double2(re[i + 1], im[i + 1]);
    }
  }
}

// ------------------------------------------------------------------ chunked global <-> smem
// Chunk ch = tid + i * nthr covers EPC elements starting at EPC * ch (EPC = 16 bytes / element).
// With nthr = 2^(k-R) threads each thread owns 2^NB chunks, NB = R - log2(EPC).
template <typename T, int R>
struct ChunkMap {
  static constexpr int EPC = std::is_same<T, float>::value ? 2 : 1;
  static constexpr int NB = R - (EPC == 2 ? 1 : 0);
  int64_t g_tid;        // global element offset of the thread's chunk 0 (without tile base)
  uint32_t e_tid;       // tile element of chunk 0
  int64_t g_unit[NB > 0 ? NB : 1];
  uint32_t e_unit[NB > 0 ? NB : 1];

  __device__ __forceinline__ void init(const uint8_t* L, int k, uint32_t tid, int nthr_log2) {
    const uint32_t e0 = (uint32_t)EPC * tid;
    e_tid = e0;
    g_tid = deposit_L(e0, L, k);
    const int lo = nthr_log2 + (EPC == 2 ? 1 : 0);
#pragma unroll
    for (int r = 0; r < NB; r++) {
      e_unit[r] = 1u << (lo + r);
      g_unit[r] = (int64_t)1 << L[lo + r];
    }
  }
  __device__ __forceinline__ uint32_t elem(int i) const {
    uint32_t e = e_tid;
#pragma unroll
    for (int r = 0; r < NB; r++)
      if ((i >> r) & 1) e |= e_unit[r];
    return e;
  }
  __device__ __forceinline__ int64_t goff(int i) const {
    int64_t g = g_tid;
#pragma unroll
    for (int r = 0; r < NB; r++)
      if ((i >> r) & 1) g |= g_unit[r];
    return g;
  }
};

// ------------------------------------------------------------------ forward pass
template <typename T, int R>
__global__ void __launch_bounds__(256) fwd_pass_kernel(PassLaunch a, const void* in_, void* out_, double* zpart) {
  using V2 = typename V2T<T>::type;
  constexpr int N = 1 << R;
  constexpr int EPC = ChunkMap<T, R>::EPC;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevPass P;
  const uint32_t tid = threadIdx.x;
  const int nthr = blockDim.x;
  if (tid == 0) P = *a.d_pass;
  __syncthreads();
  const int k = P.k;
  const FwdSmem sm = fwd_smem(k, P.n_phases, P.n_ops, (int)sizeof(V2), (int)sizeof(T), nthr);
  DevLayout* lays = reinterpret_cast<DevLayout*>(smem + sm.lays);
  for (int i = tid; i <= P.n_phases; i += nthr) lays[i] = a.d_layouts[P.lay0 + i];
  const int64_t tps = P.tiles_per_sample;
  const int b = (int)(blockIdx.x / tps);
  const int64_t t = (int64_t)blockIdx.x - (int64_t)b * tps;
  const int64_t dim = (int64_t)1 << a.n;
  int64_t tile_base = (int64_t)b * dim;
  for (int j = 0; j < P.n_nonlocal; j++)
    if ((t >> j) & 1) tile_base += (int64_t)1 << P.nonlocal[j];

  V2* tile = reinterpret_cast<V2*>(smem + sm.tile);
  T* coef_s = reinterpret_cast<T*>(smem + sm.coef);
  uint8_t* form_s = reinterpret_cast<uint8_t*>(smem + sm.form);
  const T* coefg = reinterpret_cast<const T*>(a.coef);
  for (int i = tid; i < P.n_ops; i += nthr) {
    const DevOp op = a.d_ops[P.op0 + i];
    if (op.rot) {
      coef_s[i] = coefg[(int64_t)op.gate * a.B + b];
      form_s[i] = a.form[(int64_t)op.gate * a.B + b];
    } else {
      coef_s[i] = T(0);
      form_s[i] = 0;
    }
  }
  __syncthreads();   // lays[] visible

  int nthr_log2 = 0;
  while ((1 << nthr_log2) < nthr) nthr_log2++;
  using CM = ChunkMap<T, R>;
  CM cm;
  cm.init(P.L, k, tid, nthr_log2);
  constexpr int n_chunks_thr = 1 << CM::NB;
  {
    const uint8_t* m0 = lays[0].m;
    if (in_ == nullptr) {
      // |0...0>: zero tile, amplitude 1 at element 0 of tile 0
#pragma unroll
      for (int i = 0; i < n_chunks_thr; i++) {
        const uint32_t e = cm.elem(i);
        const uint32_t w = lay_addr(e, m0, k);
        if constexpr (EPC == 2) reinterpret_cast<float4*>(tile)[w >> 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        else tile[w] = make_double2(0.0, 0.0);
      }
      __syncthreads();
      if (tid == 0 && t == 0) tile[0].x = T(1);
    } else {
      const V2* in = reinterpret_cast<const V2*>(in_) + tile_base;
#pragma unroll
      for (int i = 0; i < n_chunks_thr; i++) {
        const uint32_t e = cm.elem(i);
        const int64_t g = cm.goff(i);
        const uint32_t w = lay_addr(e, m0, k);
        if constexpr (EPC == 2) cp_async16(&tile[w & ~1u], in + g);
        else cp_async16(&tile[w], in + g);
      }
      cp_async_wait_all();
    }
  }
  __syncthreads();

  T re[N], im[N];
  for (int ph = 0; ph < P.n_phases; ph++) {
    const DevPhase phase = a.d_phases[P.phase0 + ph];
    PhaseAddr pa;
    phase_addr<R>(pa, phase, lays[ph].m, lays[ph + 1].m, k, tid);
    load_regs<R, T>(tile, pa.s_in, pa.u_in, re, im);
    for (int oi = phase.op_begin; oi < phase.op_end; oi++) {
      const DevOp op = a.d_ops[oi];
      const int li = oi - P.op0;
      apply_op<R, T>(op, re, im, coef_s[li], form_s[li], pa.tb);
    }
    __syncthreads();
    store_regs<R, T>(tile, pa.s_out, pa.u_out, re, im);
    __syncthreads();
  }

  // epilogue: scale, optional <Z> partials, store
  cm.init(P.L, k, tid, nthr_log2);
  const T scale = reinterpret_cast<const T*>(a.scale)[b];
  const uint8_t* ml = lays[P.n_phases].m;
  V2* out = reinterpret_cast<V2*>(out_) + tile_base;
  using ZA = typename Acc<T>::type;
  ZA ztot = 0, zs[kMaxR + 1];
#pragma unroll
  for (int r = 0; r <= kMaxR; r++) zs[r] = 0;
#pragma unroll
  for (int i = 0; i < n_chunks_thr; i++) {
    const uint32_t e = cm.elem(i);
    const int64_t g = cm.goff(i);
    const uint32_t w = lay_addr(e, ml, k);
    if constexpr (EPC == 2) {
      float4 v = reinterpret_cast<const float4*>(tile)[w >> 1];
      v.x *= scale; v.y *= scale; v.z *= scale; v.w *= scale;
      *reinterpret_cast<float4*>(out + g) = v;
      if (zpart) {
        const float p0 = fmaf(v.x, v.x, v.y * v.y), p1 = fmaf(v.z, v.z, v.w * v.w);
        ztot += p0 + p1;
        zs[0] += p0 - p1;   // tile bit 0
#pragma unroll
        for (int r = 0; r < CM::NB; r++) zs[1 + r] += ((i >> r) & 1) ? -(p0 + p1) : (p0 + p1);
      }
    } else {
      double2 v = tile[w];
      v.x *= scale; v.y *= scale;
      out[g] = v;
      if (zpart) {
        const double p = v.x * v.x + v.y * v.y;
        ztot += p;
#pragma unroll
        for (int r = 0; r < CM::NB; r++) zs[r] += ((i >> r) & 1) ? -p : p;
      }
    }
  }
  if (zpart) {
    // block reduction: output j < k is sum_e s_j(e) p(e); output k is the tile's total
    __syncthreads();
    constexpr int NZ = kMaxR + 2;
    ZA* red = reinterpret_cast<ZA*>(smem);      // tile no longer needed
    red[tid * NZ + 0] = ztot;
#pragma unroll
    for (int r = 0; r <= kMaxR; r++) red[tid * NZ + 1 + r] = zs[r];
    __syncthreads();
    const int tid_lo = (EPC == 2) ? 1 : 0;    // first tile bit driven by the thread id
    for (int j = tid; j <= k; j += nthr) {
      double acc = 0.0;
      if (j == k) {
        for (int u = 0; u < nthr; u++) acc += (double)red[u * NZ];
      } else if (j >= tid_lo && j < tid_lo + nthr_log2) {
        const int bit = j - tid_lo;
        for (int u = 0; u < nthr; u++) acc += ((u >> bit) & 1) ? -(double)red[u * NZ] : (double)red[u * NZ];
      } else {
        int slot;
        if (EPC == 2 && j == 0) slot = 0;
        else slot = (EPC == 2 ? 1 : 0) + (j - tid_lo - nthr_log2);
        for (int u = 0; u < nthr; u++) acc += (double)red[u * NZ + 1 + slot];
      }
      zpart[((int64_t)b * tps + t) * (k + 1) + j] = acc;
    }
  }
}

// ------------------------------------------------------------------ backward pass
template <typename T, int R>
__global__ void __launch_bounds__(256) bwd_pass_kernel(PassLaunch a, const void* psi_in_, void* psi_out_,
                                                        const void* lam_in_, void* lam_out_, const double* grad_out,
                                                        double* gpart) {
  using V2 = typename V2T<T>::type;
  using GA = typename Acc<T>::type;
  constexpr int N = 1 << R;
  constexpr int EPC = ChunkMap<T, R>::EPC;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevPass P;
  const uint32_t tid = threadIdx.x;
  const int nthr = blockDim.x;
  if (tid == 0) P = *a.d_pass;
  __syncthreads();
  const int k = P.k;
  const BwdSmem sm = bwd_smem(k, P.n_phases, P.n_ops, P.n_gslots, (int)sizeof(V2), (int)sizeof(T), nthr);
  DevLayout* lays = reinterpret_cast<DevLayout*>(smem + sm.lays);
  for (int i = tid; i <= P.n_phases; i += nthr) lays[i] = a.d_layouts[P.lay0 + i];
  const int64_t tps = P.tiles_per_sample;
  const int b = (int)(blockIdx.x / tps);
  const int64_t t = (int64_t)blockIdx.x - (int64_t)b * tps;
  const int64_t dim = (int64_t)1 << a.n;
  int64_t tile_base = (int64_t)b * dim;
  for (int j = 0; j < P.n_nonlocal; j++)
    if ((t >> j) & 1) tile_base += (int64_t)1 << P.nonlocal[j];
  const int n_warps = (nthr + 31) / 32;

  V2* tpsi = reinterpret_cast<V2*>(smem + sm.psi);
  V2* tlam = reinterpret_cast<V2*>(smem + sm.lam);
  T* coef_s = reinterpret_cast<T*>(smem + sm.coef);
  GA* red = reinterpret_cast<GA*>(smem + sm.red);       // [n_warps][n_gslots]
  double* gq = reinterpret_cast<double*>(smem + sm.gq);  // [k + 1]
  uint8_t* form_s = reinterpret_cast<uint8_t*>(smem + sm.form);
  const T* coefg = reinterpret_cast<const T*>(a.coef);
  for (int i = tid; i < P.n_ops; i += nthr) {
    const DevOp op = a.d_ops[P.op0 + i];
    if (op.rot) {
      coef_s[i] = -coefg[(int64_t)op.gate * a.B + b];   // inverse: negated coefficient
      form_s[i] = a.form[(int64_t)op.gate * a.B + b];
    } else {
      coef_s[i] = T(0);
      form_s[i] = 0;
    }
  }
  const bool init_lambda = (lam_in_ == nullptr);
  if (init_lambda && tid == 0) {
    // g of each tile bit, and the contribution of the tile's fixed (nonlocal) bits
    double dconst = 0.0;
    for (int j = 0; j < P.n_nonlocal; j++) {
      const int q = a.n - 1 - P.nonlocal[j];
      const double g = grad_out[(int64_t)b * a.n + q];
      dconst += ((t >> j) & 1) ? -g : g;
    }
    for (int j = 0; j < k; j++) gq[j] = grad_out[(int64_t)b * a.n + (a.n - 1 - P.L[j])];
    gq[k] = dconst;
  }
  __syncthreads();

  int nthr_log2 = 0;
  while ((1 << nthr_log2) < nthr) nthr_log2++;
  using CM = ChunkMap<T, R>;
  CM cm;
  cm.init(P.L, k, tid, nthr_log2);
  constexpr int n_chunks_thr = 1 << CM::NB;
  const uint8_t* mload = lays[P.n_phases].m;
  {
    const V2* pin = reinterpret_cast<const V2*>(psi_in_) + tile_base;
    const V2* lin = init_lambda ? nullptr : reinterpret_cast<const V2*>(lam_in_) + tile_base;
#pragma unroll
    for (int i = 0; i < n_chunks_thr; i++) {
      const uint32_t e = cm.elem(i);
      const int64_t g = cm.goff(i);
      const uint32_t w = lay_addr(e, mload, k) & (EPC == 2 ? ~1u : ~0u);
      cp_async16(&tpsi[w], pin + g);
      if (!init_lambda) cp_async16(&tlam[w], lin + g);
    }
    cp_async_wait_all();
    if (init_lambda) {
      __syncthreads();
      for (int i = 0; i < n_chunks_thr; i++) {
        const uint32_t e = cm.elem(i);
        for (int h = 0; h < EPC; h++) {
          const uint32_t ee = e + h;
          double d = gq[k];
          for (int j = 0; j < k; j++) d += ((ee >> j) & 1u) ? -gq[j] : gq[j];
          const uint32_t w = lay_addr(ee, mload, k);
          V2 v = tpsi[w];
          tlam[w] = V2{(T)(d * v.x), (T)(d * v.y)};
        }
      }
    }
  }
  __syncthreads();

  const unsigned full = nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u);
  const int lane = tid & 31, warp = tid >> 5;
  T pr[N], pi[N], lr[N], li[N];
  for (int ph = P.n_phases - 1; ph >= 0; ph--) {
    const DevPhase phase = a.d_phases[P.phase0 + ph];
    PhaseAddr pa;
    phase_addr<R>(pa, phase, lays[ph + 1].m, lays[ph].m, k, tid);
    load_regs<R, T>(tpsi, pa.s_in, pa.u_in, pr, pi);
    load_regs<R, T>(tlam, pa.s_in, pa.u_in, lr, li);
    for (int oi = phase.op_end - 1; oi >= phase.op_begin; oi--) {
      const DevOp op = a.d_ops[oi];
      const int lo = oi - P.op0;
      if (op.rot) {
        GA g = op_grad<R, T>(op, pr, pi, lr, li, pa.tb);
        for (int off = (nthr >= 32 ? 16 : nthr / 2); off > 0; off >>= 1) g += __shfl_xor_sync(full, g, off);
        if (lane == 0) red[warp * P.n_gslots + op.gslot] = g;
      }
      apply_op<R, T>(op, pr, pi, coef_s[lo], form_s[lo], pa.tb);
      apply_op<R, T>(op, lr, li, coef_s[lo], form_s[lo], pa.tb);
    }
    __syncthreads();
    store_regs<R, T>(tpsi, pa.s_out, pa.u_out, pr, pi);
    store_regs<R, T>(tlam, pa.s_out, pa.u_out, lr, li);
    __syncthreads();
  }

  // gradient partials of this tile: sum over warps in FP64
  for (int sl = tid; sl < P.n_gslots; sl += nthr) {
    double acc = 0.0;
    for (int w = 0; w < n_warps; w++) acc += (double)red[w * P.n_gslots + sl];
    gpart[((P.gpart_offset + sl) * a.B + b) * tps + t] = acc;
  }
  if (psi_out_ == nullptr) return;
  cm.init(P.L, k, tid, nthr_log2);
  const T scale = reinterpret_cast<const T*>(a.scale)[b];
  const uint8_t* ms = lays[0].m;
  V2* pout = reinterpret_cast<V2*>(psi_out_) + tile_base;
  V2* lout = reinterpret_cast<V2*>(lam_out_) + tile_base;
#pragma unroll
  for (int i = 0; i < n_chunks_thr; i++) {
    const uint32_t e = cm.elem(i);
    const int64_t g = cm.goff(i);
    const uint32_t w = lay_addr(e, ms, k);
    if constexpr (EPC == 2) {
      float4 v = reinterpret_cast<const float4*>(tpsi)[w >> 1];
      float4 l = reinterpret_cast<const float4*>(tlam)[w >> 1];
      v.x *= scale; v.y *= scale; v.z *= scale; v.w *= scale;
      l.x *= scale; l.y *= scale; l.z *= scale; l.w *= scale;
      *reinterpret_cast<float4*>(pout + g) = v;
      *reinterpret_cast<float4*>(lout + g) = l;
    } else {
      double2 v = tpsi[w], l = tlam[w];
      v.x *= scale; v.y *= scale; l.x *= scale; l.y *= scale;
      pout[g] = v;
      lout[g] = l;
    }
  }
}

// ------------------------------------------------------------------ host side
// Register bits per phase: complex64 forward 5 (32 amplitudes), backward 4 (psi and lambda);
// complex128 one less each. Threads per CTA = 2^(k - R) <= 256.
int fwd_R_for(int k, int dtype) { const int r = dtype == QSIM_C128 ? 4 : 5; return k < r ? k : r; }
int bwd_R_for(int k, int dtype) { const int r = dtype == QSIM_C128 ? 3 : 4; return k < r ? k : r; }
int max_k_for(int dtype) { return dtype == QSIM_C128 ? 11 : 12; }
int bwd_R(int k) { return bwd_R_for(k, QSIM_C64); }

size_t fwd_pass_smem(const DevPass& p, int dtype, int nthr) {
  const int el = dtype == QSIM_C128 ? 16 : 8, sc = dtype == QSIM_C128 ? 8 : 4;
  return fwd_smem(p.k, p.n_phases, p.n_ops, el, sc, nthr).total;
}

size_t bwd_pass_smem(const DevPass& p, int dtype, int nthr) {
  const int el = dtype == QSIM_C128 ? 16 : 8, sc = dtype == QSIM_C128 ? 8 : 4;
  return bwd_smem(p.k, p.n_phases, p.n_ops, p.n_gslots, el, sc, nthr).total;
}

template <typename T>
static cudaError_t set_attrs(size_t fwd, size_t bwd) {
  cudaError_t e = cudaSuccess;
#define QSIM_ATTR(KERN, BYTES)                                                                      \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BYTES));
  QSIM_ATTR((fwd_pass_kernel<T, 1>), fwd) QSIM_ATTR((fwd_pass_kernel<T, 2>), fwd)
  QSIM_ATTR((fwd_pass_kernel<T, 3>), fwd) QSIM_ATTR((fwd_pass_kernel<T, 4>), fwd)
  QSIM_ATTR((bwd_pass_kernel<T, 1>), bwd) QSIM_ATTR((bwd_pass_kernel<T, 2>), bwd)
  QSIM_ATTR((bwd_pass_kernel<T, 3>), bwd)
  if constexpr (sizeof(T) == 4) {
    QSIM_ATTR((fwd_pass_kernel<T, 5>), fwd)
    QSIM_ATTR((bwd_pass_kernel<T, 4>), bwd)
  }
#undef QSIM_ATTR
  return e;
}

cudaError_t prepare_pass_kernels(int dtype, size_t max_fwd_smem, size_t max_bwd_smem) {
  if (max_fwd_smem < 48 * 1024) max_fwd_smem = 48 * 1024;
  if (max_bwd_smem < 48 * 1024) max_bwd_smem = 48 * 1024;
  return dtype == QSIM_C128 ? set_attrs<double>(max_fwd_smem, max_bwd_smem)
                            : set_attrs<float>(max_fwd_smem, max_bwd_smem);
}

template <typename T>
static cudaError_t fwd_dispatch(const PassLaunch& L, const void* in, void* out, double* zpart, cudaStream_t st) {
  const DevPass& p = *L.h_pass;
  const int R = p.R;
  const int nthr = 1 << (p.k - R);
  const size_t smem = fwd_pass_smem(p, sizeof(T) == 8 ? QSIM_C128 : QSIM_C64, nthr);
  const int64_t blocks = p.tiles_per_sample * L.B;
  if (blocks <= 0 || blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  switch (R) {
    case 1: fwd_pass_kernel<T, 1><<<(unsigned)blocks, nthr, smem, st>>>(L, in, out, zpart); break;
    case 2: fwd_pass_kernel<T, 2><<<(unsigned)blocks, nthr, smem, st>>>(L, in, out, zpart); break;
    case 3: fwd_pass_kernel<T, 3><<<(unsigned)blocks, nthr, smem, st>>>(L, in, out, zpart); break;
    case 4: fwd_pass_kernel<T, 4><<<(unsigned)blocks, nthr, smem, st>>>(L, in, out, zpart); break;
    default:
      if constexpr (sizeof(T) == 4) fwd_pass_kernel<T, 5><<<(unsigned)blocks, nthr, smem, st>>>(L, in, out, zpart);
      break;
  }
  g_kernel_launches++;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t bwd_dispatch(const PassLaunch& L, const void* pin, void* pout, const void* lin, void* lout,
                                const double* g, double* gpart, cudaStream_t st) {
  const DevPass& p = *L.h_pass;
  const int R = p.R;
  const int nthr = 1 << (p.k - R);
  const size_t smem = bwd_pass_smem(p, sizeof(T) == 8 ? QSIM_C128 : QSIM_C64, nthr);
  const int64_t blocks = p.tiles_per_sample * L.B;
  if (blocks <= 0 || blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  switch (R) {
    case 1: bwd_pass_kernel<T, 1><<<(unsigned)blocks, nthr, smem, st>>>(L, pin, pout, lin, lout, g, gpart); break;
    case 2: bwd_pass_kernel<T, 2><<<(unsigned)blocks, nthr, smem, st>>>(L, pin, pout, lin, lout, g, gpart); break;
    case 3: bwd_pass_kernel<T, 3><<<(unsigned)blocks, nthr, smem, st>>>(L, pin, pout, lin, lout, g, gpart); break;
    default:
      if constexpr (sizeof(T) == 4) bwd_pass_kernel<T, 4><<<(unsigned)blocks, nthr, smem, st>>>(L, pin, pout, lin, lout, g, gpart);
      break;
  }
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_fwd_pass(const PassLaunch& L, int dtype, const void* in, void* out, double* zpart,
                            cudaStream_t st) {
  return dtype == QSIM_C128 ? fwd_dispatch<double>(L, in, out, zpart, st) : fwd_dispatch<float>(L, in, out, zpart, st);
}

cudaError_t launch_bwd_pass(const PassLaunch& L, int dtype, const void* psi_in, void* psi_out, const void* lam_in,
                            void* lam_out, const double* grad_out, double* gpart, cudaStream_t st) {
  return dtype == QSIM_C128 ? bwd_dispatch<double>(L, psi_in, psi_out, lam_in, lam_out, grad_out, gpart, st)
                            : bwd_dispatch<float>(L, psi_in, psi_out, lam_in, lam_out, grad_out, gpart, st);
}

}  // namespace qsim
