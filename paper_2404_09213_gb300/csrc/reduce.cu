// Angle -> coefficient formation, and the deterministic FP64 reductions (<Z>, gradients).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "launch.hpp"

namespace qsim {

std::atomic<long long> g_kernel_launches{0};

// ------------------------------------------------------------------ coefficients
// Gate-matrix caching (Sec. "Gate Matrix Caching", Eq. 1) writes R_x(theta) = cos(theta/2) R_xa + (-i sin(theta/2)) R_xb
// with fixed partial matrices and two angle-dependent scalars. Here the scalars are formed once per
// forward for every (gate, sample) and stored as one coefficient per rotation (tan or cot of theta/2,
// whichever is at most 1 in magnitude) plus the factored-out cos / sin, accumulated per pass.
constexpr double kPi = 3.14159265358979323846;

// Angle of a trainable parameter: as given, or remapped into (-pi, pi) by pi * tanh (quantum weight
// remapping, Sec. "Additional Optimizations"); d(angle)/d(param) is remap_slope.
template <typename T>
__device__ __forceinline__ double weight(T p, int remap) {
  return remap ? kPi * tanh((double)p) : (double)p;
}
__device__ __forceinline__ double remap_slope(const void* params, int64_t i, int dtype) {
  const double p = dtype == QSIM_C128 ? reinterpret_cast<const double*>(params)[i]
                                      : (double)reinterpret_cast<const float*>(params)[i];
  const double t = tanh(p);
  return kPi * (1.0 - t * t);
}

// Stage 1, one thread per (gate, sample): the angle's sine and cosine (FP64), the coefficient and its
// form, and the factored-out value (cos for the tangent form, sin for the cotangent form), parked in
// gm until stage 2 turns it into the squared backward scale.
template <typename T>
__global__ void coef_gate_kernel(CoefArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)a.G * a.B) return;
  const int g = (int)(id / a.B), b = (int)(id - (int64_t)g * a.B);
  if (a.gate_type[g] > QSIM_RZ) return;
  const T* params = reinterpret_cast<const T*>(a.params);
  const T* inputs = reinterpret_cast<const T*>(a.inputs);
  int n_inputs = a.n_inputs;
  if (a.gate_circ) {   // several circuits: parameters and inputs of this gate's circuit
    const int c = a.gate_circ[g];
    if (params) params += a.circ_param_off[c];
    if (inputs) inputs += (int64_t)a.B * a.circ_col_off[c];
    n_inputs = a.circ_ninputs[c];
  }
  const int pr = a.gate_param[g];
  const double th = pr >= 0 ? weight(params[pr], a.weight_remap)
                            : weight(inputs[(int64_t)b * n_inputs + (-2 - pr)], a.weight_remap == 2);
  double s, c;
  sincos(0.5 * th, &s, &c);
  const bool cot = fabs(s) > fabs(c);
  reinterpret_cast<T*>(a.coef)[id] = (T)(cot ? c / s : s / c);
  a.form[id] = cot ? 1 : 0;
  a.gm[id] = cot ? s : c;
}

// Stage 2, one warp per (pass, sample): packs the pass's coefficients in op order and multiplies the
// factored-out values into the per-pass scales, 32 ops at a time (no trigonometry). R is the running
// product of the factors in processing order (an inclusive warp scan plus the previous chunks'
// carry); the scale gathered since the last rescale op is R divided by R at that op. The factors lie
// in [1/sqrt(2), 1] and a pass holds at most 256 of them, so R stays far inside the FP64 range.
struct ScanState {
  double carry = 1.0;   // product of the factors of all earlier chunks
  double rlast = 1.0;   // running product at the latest rescale op so far
};

// Returns the inclusive running product at this lane's op; rprev = the running product at the
// latest rescale op before it (in processing order).
__device__ __forceinline__ double scan_chunk(double fac, bool is_scale, ScanState& st, double& rprev) {
  const unsigned full = 0xffffffffu, lane = threadIdx.x & 31u;
  double r = fac;
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(full, r, o);
    if ((int)lane >= o) r *= t;
  }
  r *= st.carry;
  const unsigned m = __ballot_sync(full, is_scale);
  const unsigned below = m & ((1u << lane) - 1u);
  const double rs = __shfl_sync(full, r, below ? 31 - __clz(below) : (int)lane);
  rprev = below ? rs : st.rlast;
  const double rl = __shfl_sync(full, r, m ? 31 - __clz(m) : 0);
  if (m) st.rlast = rl;
  st.carry = __shfl_sync(full, r, 31);
  return r;
}

template <typename T>
__global__ void coef_pass_kernel(CoefArgs a) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= (int64_t)a.P * a.B) return;   // whole warps leave together
  const int lane = (int)(threadIdx.x & 31u);
  const int p = (int)(w / a.B), b = (int)(w - (int64_t)p * a.B);
  const T* coef = reinterpret_cast<const T*>(a.coef);
  constexpr double kH = 0.70710678118654752440;
  // forward: op order
  const int e0 = a.exec_begin[p], e1 = a.exec_begin[p + 1];
  T* cfp = reinterpret_cast<T*>(a.cfp_f) + (int64_t)e0 * a.B + (int64_t)b * (e1 - e0) - e0;
  uint8_t* fmp = a.fmp_f + (int64_t)e0 * a.B + (int64_t)b * (e1 - e0) - e0;
  ScanState sf;
  for (int base = e0; base < e1; base += 32) {
    const int e = base + lane;
    const int g = e < e1 ? a.exec_gates[e] : -2;   // -1: rescale op, -2: past the end
    double fac = 1.0;
    T v = 0;
    uint8_t f = 0;
    if (g >= 0) {
      const int ty = a.gate_type[g];
      if (ty <= QSIM_RZ) {
        const int64_t gi = (int64_t)g * a.B + b;
        v = coef[gi];
        f = a.form[gi];
        fac = a.gm[gi];
        if (a.sigma) {   // Pauli frame: tangent form, coefficient sigma * tan or -sigma * cot
          const T sg = (T)a.sigma[gi];
          v = f ? -sg * v : sg * v;
          f = 0;
        }
      } else if (ty == QSIM_H) {
        fac = kH;
      }
    }
    double rprev;
    const double r = scan_chunk(fac, g == -1, sf, rprev);
    if (g == -1) v = (T)(r / rprev);   // a rescale op applies the factors since the previous one
    if (g >= -1) {
      cfp[e] = v;
      fmp[e] = f;
    }
  }
  if (lane == 0) reinterpret_cast<T*>(a.scale_f)[(int64_t)p * a.B + b] = (T)(sf.carry / sf.rlast);
  __syncwarp();   // every lane's forward reads of gm come before any lane overwrites it below
  // backward: ops undone from the end of the backward op list; gm = (product of the signed inverse
  // scales since the last rescale op, before this op)^2. Every gate sits in exactly one pass, so the
  // factors read and overwritten here are this warp's alone.
  const int b0 = a.exec_begin_b[p], b1 = a.exec_begin_b[p + 1];
  T* cfpb = reinterpret_cast<T*>(a.cfp_b) + (int64_t)b0 * a.B + (int64_t)b * (b1 - b0) - b0;
  uint8_t* fmpb = a.fmp_b + (int64_t)b0 * a.B + (int64_t)b * (b1 - b0) - b0;
  ScanState sb;
  for (int base = 0; base < b1 - b0; base += 32) {
    const int e = b1 - 1 - base - lane;
    const int g = e >= b0 ? a.exec_gates_b[e] : -2;
    double fac = 1.0;
    T v = 0;
    uint8_t f = 0;
    int64_t gi = -1;
    if (g >= 0) {
      const int ty = a.gate_type[g];
      if (ty <= QSIM_RZ) {
        gi = (int64_t)g * a.B + b;
        f = a.form[gi];
        v = -coef[gi];   // the inverse rotation
        fac = f ? -a.gm[gi] : a.gm[gi];
        if (a.sigma) {   // Pauli frame: the negated tangent-form coefficient; cos or sin as it is
          const T sg = (T)a.sigma[gi];
          v = f ? sg * coef[gi] : -sg * coef[gi];
          fac = a.gm[gi];
          f = 0;
        }
      } else if (ty == QSIM_H) {
        fac = kH;
      }
    }
    double rprev;
    const double r = scan_chunk(fac, g == -1, sb, rprev);
    if (gi >= 0) {
      const double bs = (r / fac) / rprev;   // before this op: exclude its own factor
      a.gm[gi] = a.sigma ? (double)a.sigma[gi] * bs * bs : bs * bs;   // the frame's sign of P
    }
    if (g == -1) v = (T)(r / rprev);
    if (g >= -1) {
      cfpb[e] = v;
      fmpb[e] = f;
    }
  }
  if (lane == 0) reinterpret_cast<T*>(a.scale_b)[(int64_t)p * a.B + b] = (T)(sb.carry / sb.rlast);
}

// Pauli frame F = i^k X^x Z^z (per qubit X^x_q Z^z_q, bit q = qubit q), one op at a time in execution
// order. A rotation returns the sign of its Pauli under F (-1 where they anticommute), and a
// cotangent-form rotation then left-multiplies F by -iP; H, X, CNOT and CZ conjugate F. Compiled for the
// device (frame_walk_kernel) and the host (qsim_frame_walk_host, a test hook).
struct Frame {
  uint64_t x = 0, z = 0;
  int k = 0;
};

__host__ __device__ inline int frame_step(Frame& f, int ty, int q, int c, int cot) {
  const uint64_t bq = 1ull << q;
  const int xq = (int)((f.x >> q) & 1u), zq = (int)((f.z >> q) & 1u);
  int sigma = 1;
  if (ty <= QSIM_RZ) {
    const int anti = ty == QSIM_RX ? zq : ty == QSIM_RZ ? xq : (xq ^ zq);
    sigma = anti ? -1 : 1;
    if (cot) {
      if (ty == QSIM_RZ) {
        f.z ^= bq;
        f.k += 2 * xq;
      } else if (ty == QSIM_RX) {
        f.x ^= bq;
      } else {
        f.x ^= bq;
        f.z ^= bq;
        f.k += 1 + 2 * xq;
      }
      f.k += 3;   // the factor -i
    }
  } else if (ty == QSIM_H) {   // X <-> Z, XZ -> -XZ
    if (xq & zq) f.k += 2;
    if (xq != zq) {
      f.x ^= bq;
      f.z ^= bq;
    }
  } else if (ty == QSIM_X) {   // Z -> -Z
    if (zq) f.k += 2;
  } else if (ty == QSIM_CNOT) {   // control c, target q: X_c -> X_c X_q, Z_q -> Z_c Z_q
    if ((f.x >> c) & 1u) f.x ^= bq;
    if (zq) f.z ^= 1ull << c;
  } else if (ty == QSIM_CZ) {   // X_q -> X_q Z_c, X_c -> Z_q X_c
    const int xc = (int)((f.x >> c) & 1u);
    if (xq & xc) f.k += 2;
    if (xq) f.z ^= 1ull << c;
    if (xc) f.z ^= bq;
  }
  f.k &= 3;
  return sigma;
}

// One thread per sample over every op of every pass in execution order, one warp per block. The ops'
// gate, kind and qubits are the same for every sample, and each sample's form bytes of a chunk of ops
// are independent of the walk: both are staged in shared memory first (the form loads pipeline, 32
// consecutive samples per op), so the serial walk itself reads shared memory only.
__global__ void frame_walk_kernel(CoefArgs a) {
  constexpr int CH = 256;
  __shared__ int s_g[CH];
  __shared__ int s_meta[CH];   // kind | q0 << 8 | (q1 + 1) << 16
  __shared__ uint8_t s_form[CH][32];
  const int lane = (int)threadIdx.x;
  const int b = blockIdx.x * 32 + lane;
  Frame f;
  const int e0 = a.exec_begin[0], e1 = a.exec_begin[a.P];
  for (int base = e0; base < e1; base += CH) {
    const int m = min(CH, e1 - base);
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      const int g = a.exec_gates[base + i];
      s_g[i] = g;
      s_meta[i] = g < 0 ? 0 : (a.gate_type[g] | (a.gate_q0[g] << 8) | ((a.gate_q1[g] + 1) << 16));
    }
    __syncwarp();
    for (int i0 = 0; i0 < m; i0 += 64) {   // 64 independent loads in flight, then their stores
      uint8_t v[64];
#pragma unroll
      for (int u = 0; u < 64; u++) {
        const int i = i0 + u;
        const int g = i < m ? s_g[i] : -1;
        v[u] = (g >= 0 && (s_meta[i] & 255) <= QSIM_RZ && b < a.B) ? a.form[(int64_t)g * a.B + b] : 0;
      }
#pragma unroll
      for (int u = 0; u < 64; u++)
        if (i0 + u < m) s_form[i0 + u][lane] = v[u];
    }
    __syncwarp();
    if (b < a.B)
      for (int i = 0; i < m; i++) {
        const int g = s_g[i];
        if (g < 0) continue;   // rescale op
        const int meta = s_meta[i], ty = meta & 255;
        const int sg = frame_step(f, ty, (meta >> 8) & 255, ((meta >> 16) & 255) - 1, s_form[i][lane]);
        if (ty <= QSIM_RZ) a.sigma[(int64_t)g * a.B + b] = (int8_t)sg;
      }
  }
  if (b < a.B) {
    a.frame_x[b] = f.x;
    a.frame_z[b] = f.z;
    a.frame_k[b] = f.k;
  }
}

cudaError_t launch_coef(const CoefArgs& a, int dtype, cudaStream_t st) {
  const int64_t ng = (int64_t)a.G * a.B, np = (int64_t)a.P * a.B;
  if (np == 0) return cudaSuccess;
  const int tg = 128, tp = 128;   // stage 2: one warp per (pass, sample), four per block
  const unsigned bg = (unsigned)((ng + tg - 1) / tg), bp = (unsigned)((np * 32 + tp - 1) / tp);
  if (ng > 0) {
    if (dtype == QSIM_C128) coef_gate_kernel<double><<<bg, tg, 0, st>>>(a);
    else coef_gate_kernel<float><<<bg, tg, 0, st>>>(a);
    g_kernel_launches++;
  }
  // the frame's signs must exist before the coefficients are packed; the walk also writes the final frame
  // (the identity for a gate list without rotations, which has no sign array)
  if (a.frame_x) {
    frame_walk_kernel<<<(unsigned)((a.B + 31) / 32), 32, 0, st>>>(a);
    g_kernel_launches++;
  }
  if (dtype == QSIM_C128) coef_pass_kernel<double><<<bp, tp, 0, st>>>(a);
  else coef_pass_kernel<float><<<bp, tp, 0, st>>>(a);
  g_kernel_launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ fixed-order block reduction
__device__ __forceinline__ double block_sum(double v, double* sh) {
  // fixed tree: warp butterflies, then warp 0 over the warp totals -> same order every run
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nw ? sh[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
  }
  __syncthreads();
  return r;   // valid in thread 0
}

// z[b][q] from per-tile partials: block per (b, q).
__global__ void z_final_kernel(const double* zpart, int k, const uint8_t* Qnl, int n_nonlocal, int64_t tps,
                               int n, int B, double* z, const uint64_t* frame_x) {
  __shared__ double sh[32];
  const int b = blockIdx.x / n, q = blockIdx.x - (blockIdx.x / n) * n;
  int tbit = -1, nlbit = -1;   // qubit q is tile bit tbit or tile-index bit nlbit of the last pass
  for (int j = 0; j < k; j++)
    if (Qnl[j] == q) tbit = j;
  for (int j = 0; j < n_nonlocal; j++)
    if (Qnl[k + j] == q) nlbit = j;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < tps; t += blockDim.x) {
    const double* row = zpart + ((int64_t)b * tps + t) * (k + 1);
    if (tbit >= 0) acc += row[tbit];
    else acc += ((t >> nlbit) & 1) ? -row[k] : row[k];
  }
  acc = block_sum(acc, sh);
  if (frame_x && ((frame_x[b] >> q) & 1u)) acc = -acc;   // F^dag Z_q F = -Z_q where F holds X or Y on q
  if (threadIdx.x == 0) z[(int64_t)b * n + q] = acc;
}

cudaError_t launch_z_final(const double* zpart, int k, const uint8_t* d_Qnl, int n_nonlocal, int64_t tps, int n,
                           int B, double* z, cudaStream_t st, const uint64_t* frame_x) {
  if ((int64_t)B * n == 0) return cudaSuccess;
  // a block per (sample, qubit) over the sample's tiles: one warp when there are few (a one-pass
  // circuit has a single tile per sample)
  const int thr = tps >= 256 ? 256 : 32;
  z_final_kernel<<<(unsigned)(B * n), thr, 0, st>>>(zpart, k, d_Qnl, n_nonlocal, tps, n, B, z, frame_x);
  g_kernel_launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Pauli frame: returned states, loss signs
// out[b][i] = i^k (-1)^popc(zi & (i ^ xi)) S[b][i ^ xi], with xi, zi the frame's masks in index bits (qubit q
// at index bit n - 1 - q). A thread takes E consecutive elements i0..i0+E-1 (i0 a multiple of E): their
// sources are the aligned block at (i0 ^ xi) with E - 1 cleared, element e coming from position
// e ^ (xi & (E - 1)), so both sides move as 16-byte vectors.
template <typename T, int E>
__device__ __forceinline__ void ld_block(const T* p, T* re, T* im) {
  if constexpr (E == 4 && sizeof(T) == 4) {
    const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
    re[0] = u.x; im[0] = u.y; re[1] = u.z; im[1] = u.w; re[2] = v.x; im[2] = v.y; re[3] = v.z; im[3] = v.w;
  } else if constexpr (E == 4) {
#pragma unroll
    for (int e = 0; e < 4; e++) { const double2 u = reinterpret_cast<const double2*>(p)[e]; re[e] = u.x; im[e] = u.y; }
  } else {
#pragma unroll
    for (int e = 0; e < E; e++) { re[e] = p[2 * e]; im[e] = p[2 * e + 1]; }
  }
}
template <typename T, int E>
__device__ __forceinline__ void st_block(T* p, const T* re, const T* im) {
  if constexpr (E == 4 && sizeof(T) == 4) {
    reinterpret_cast<float4*>(p)[0] = make_float4(re[0], im[0], re[1], im[1]);
    reinterpret_cast<float4*>(p)[1] = make_float4(re[2], im[2], re[3], im[3]);
  } else if constexpr (E == 4) {
#pragma unroll
    for (int e = 0; e < 4; e++) reinterpret_cast<double2*>(p)[e] = make_double2(re[e], im[e]);
  } else {
#pragma unroll
    for (int e = 0; e < E; e++) { p[2 * e] = re[e]; p[2 * e + 1] = im[e]; }
  }
}

template <typename T, int E>
__global__ void frame_fixup_kernel(const T* S, T* out, const uint64_t* fx, const uint64_t* fz, const int32_t* fk,
                                   int n, int B) {
  const int64_t per = (int64_t)1 << n;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
  if (i0 >= per * B) return;
  const int64_t b = i0 >> n, i = i0 & (per - 1);
  // qubit q sits at index bit n - 1 - q: a 64-bit reversal, then a shift
  const uint64_t xi = (uint64_t)__brevll((unsigned long long)fx[b]) >> (64 - n);
  const uint64_t zi = (uint64_t)__brevll((unsigned long long)fz[b]) >> (64 - n);
  const int64_t j0 = (int64_t)(((uint64_t)i ^ xi) & ~(uint64_t)(E - 1));
  T re[E], im[E];
  ld_block<T, E>(S + 2 * (b * per + j0), re, im);
  // permute by the low bits of xi (conditional swaps: no dynamic register index)
#pragma unroll
  for (int m = 1; m < E; m <<= 1)
    if (xi & (uint64_t)m) {
#pragma unroll
      for (int e = 0; e < E; e++)
        if (!(e & m)) {
          const T r = re[e], v = im[e];
          re[e] = re[e | m]; im[e] = im[e | m];
          re[e | m] = r; im[e | m] = v;
        }
    }
  const int k = fk[b] & 3;
  T ro[E], io[E];
#pragma unroll
  for (int e = 0; e < E; e++) {
    T r = re[e], v = im[e];
    if (__popcll((unsigned long long)(zi & ((uint64_t)(i + e) ^ xi))) & 1) { r = -r; v = -v; }
    T r2 = r, i2 = v;   // times i^k
    if (k == 1) { r2 = -v; i2 = r; }
    else if (k == 2) { r2 = -r; i2 = -v; }
    else if (k == 3) { r2 = v; i2 = -r; }
    ro[e] = r2;
    io[e] = i2;
  }
  st_block<T, E>(out + 2 * (b * per + i), ro, io);
}

cudaError_t launch_frame_fixup(const void* S, void* out, const uint64_t* fx, const uint64_t* fz, const int32_t* fk,
                               int n, int B, int dtype, cudaStream_t st) {
  const int64_t tot = ((int64_t)1 << n) * B;
  if (tot == 0) return cudaSuccess;
  const int thr = 256;
  if (n >= 2) {   // 4 elements per thread: whole vectors on both sides
    const unsigned blocks = (unsigned)((tot / 4 + thr - 1) / thr);
    if (dtype == QSIM_C128)
      frame_fixup_kernel<double, 4><<<blocks, thr, 0, st>>>((const double*)S, (double*)out, fx, fz, fk, n, B);
    else
      frame_fixup_kernel<float, 4><<<blocks, thr, 0, st>>>((const float*)S, (float*)out, fx, fz, fk, n, B);
  } else {
    const unsigned blocks = (unsigned)((tot + thr - 1) / thr);
    if (dtype == QSIM_C128)
      frame_fixup_kernel<double, 1><<<blocks, thr, 0, st>>>((const double*)S, (double*)out, fx, fz, fk, n, B);
    else
      frame_fixup_kernel<float, 1><<<blocks, thr, 0, st>>>((const float*)S, (float*)out, fx, fz, fk, n, B);
  }
  g_kernel_launches++;
  return cudaGetLastError();
}

__global__ void frame_gsign_kernel(const double* g, const uint64_t* fx, int n, int B, double* out) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)n * B) return;
  const int64_t b = id / n;
  const int q = (int)(id - b * n);
  out[id] = ((fx[b] >> q) & 1u) ? -g[id] : g[id];
}

cudaError_t launch_frame_gsign(const double* grad_out, const uint64_t* fx, int n, int B, double* out,
                               cudaStream_t st) {
  const int64_t tot = (int64_t)n * B;
  if (tot == 0) return cudaSuccess;
  frame_gsign_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(grad_out, fx, n, B, out);
  g_kernel_launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gradients
// G[j][b] = gm[g_j][b] * sum over the sample's tiles of the slot's partials, in a fixed order: a thread
// per (j, b) when a sample has few tiles, else a warp (strided lane sums, then a butterfly).
__global__ void grad_gather_small_kernel(GradReduceArgs a) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (int64_t)a.n_occ * a.B) return;
  const int j = (int)(w / a.B), b = (int)(w - (w / a.B) * a.B);
  if (a.occ_slot[j] < 0) return;
  const double* src = a.gpart + ((int64_t)a.occ_slot[j] * a.B + b) * a.tiles_per_sample;
  double acc = 0.0;
  for (int64_t t = 0; t < a.tiles_per_sample; t++) acc += src[t];
  a.G[(int64_t)j * a.B + b] = acc * a.gm[(int64_t)a.occ_gate[j] * a.B + b];
}

__global__ void grad_gather_kernel(GradReduceArgs a) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)a.n_occ * a.B) return;
  const int j = (int)(w / a.B), b = (int)(w - (w / a.B) * a.B);
  if (a.occ_slot[j] < 0) return;   // a prefix rotation: no pass partials (launch_prefix_grad writes G)
  const double* src = a.gpart + ((int64_t)a.occ_slot[j] * a.B + b) * a.tiles_per_sample;
  double acc = 0.0;
  for (int64_t t = lane; t < a.tiles_per_sample; t += 32) acc += src[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) a.G[(int64_t)j * a.B + b] = acc * a.gm[(int64_t)a.occ_gate[j] * a.B + b];
}

// dparams[p] = sum over occurrences (fixed order) of sum_b G[j][b]; dinputs[b][c] likewise per sample.
__global__ void grad_scatter_kernel(GradReduceArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = a.dparams ? a.n_params : 0;
  const int64_t ni = a.dinputs ? (int64_t)a.B * a.n_inputs : 0;
  if (id < np) {
    double acc = 0.0;
    for (int o = a.p_ptr[id]; o < a.p_ptr[id + 1]; o++) {
      const double* row = a.G + (int64_t)a.p_occ[o] * a.B;
      for (int b = 0; b < a.B; b++) acc += row[b];
    }
    a.dparams[id] = a.weight_remap ? acc * remap_slope(a.params, id, a.dtype) : acc;
  } else if (id < np + ni) {
    const int64_t r = id - np;
    const int b = (int)(r / a.n_inputs), c = (int)(r - (r / a.n_inputs) * a.n_inputs);
    double acc = 0.0;
    for (int o = a.i_ptr[c]; o < a.i_ptr[c + 1]; o++) acc += a.G[(int64_t)a.i_occ[o] * a.B + b];
    a.dinputs[r] = a.weight_remap == 2 ? acc * remap_slope(a.inputs, r, a.dtype) : acc;
  }
}

cudaError_t launch_grad_reduce(const GradReduceArgs& a, cudaStream_t st) {
  cudaError_t e = launch_grad_gather(a, st);
  if (e != cudaSuccess) return e;
  return launch_grad_scatter(a, st);
}

cudaError_t launch_grad_gather(const GradReduceArgs& a, cudaStream_t st) {
  if (a.n_occ > 0 && a.B > 0) {
    const int64_t rows = (int64_t)a.n_occ * a.B;
    if (a.tiles_per_sample < 32) grad_gather_small_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
    else grad_gather_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(a);
    g_kernel_launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_scatter(const GradReduceArgs& a, cudaStream_t st) {
  const int64_t total = (a.dparams ? a.n_params : 0) + (a.dinputs ? (int64_t)a.B * a.n_inputs : 0);
  if (total > 0) {
    grad_scatter_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
    g_kernel_launches++;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ product-state prefix
// A single-qubit gate that acts on a qubit before any two-qubit gate touches it acts on that qubit's |0>
// factor alone, so the state after all of them is the product of phi_q = G_m ... G_1 |0> (the per-qubit
// embedding matrices of Sec. "Gate Matrix Caching", applied to |0> and merged). Complex 2x2 matrices in
// FP64, m[row][col] = (re, im).
struct C2 {
  double r, i;
};
__device__ __forceinline__ C2 cm(C2 a, C2 b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ C2 ca(C2 a, C2 b) { return {a.r + b.r, a.i + b.i}; }

template <typename T>
__device__ double prefix_angle(const PrefixArgs& a, int g, int b) {
  const int pr = a.gate_param[g];
  const T* params = reinterpret_cast<const T*>(a.params);
  const T* inputs = reinterpret_cast<const T*>(a.inputs);
  return pr >= 0 ? weight(params[pr], a.weight_remap)
                 : weight(inputs[(int64_t)b * a.n_inputs + (-2 - pr)], a.weight_remap == 2);
}

// matrix of gate type ty at angle th (rotations exp(-i th P / 2))
__device__ void gate_m(int ty, double th, C2 m[2][2]) {
  const double kH = 0.70710678118654752440;
  double s = 0.0, c = 1.0;
  if (ty <= QSIM_RZ) sincos(0.5 * th, &s, &c);
  switch (ty) {
    case QSIM_RX: m[0][0] = {c, 0}; m[0][1] = {0, -s}; m[1][0] = {0, -s}; m[1][1] = {c, 0}; break;
    case QSIM_RY: m[0][0] = {c, 0}; m[0][1] = {-s, 0}; m[1][0] = {s, 0}; m[1][1] = {c, 0}; break;
    case QSIM_RZ: m[0][0] = {c, -s}; m[0][1] = {0, 0}; m[1][0] = {0, 0}; m[1][1] = {c, s}; break;
    case QSIM_H: m[0][0] = {kH, 0}; m[0][1] = {kH, 0}; m[1][0] = {kH, 0}; m[1][1] = {-kH, 0}; break;
    default: m[0][0] = {0, 0}; m[0][1] = {1, 0}; m[1][0] = {1, 0}; m[1][1] = {0, 0}; break;   // X
  }
}

// thread per (sample, qubit)
template <typename T>
__global__ void prefix_phi_kernel(PrefixArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)a.B * a.n) return;
  const int b = (int)(id / a.n), q = (int)(id - (int64_t)b * a.n);
  C2 v0 = {1, 0}, v1 = {0, 0};
  for (int e = a.pfx_begin[q]; e < a.pfx_begin[q + 1]; e++) {
    const int g = a.pfx_gate[e], ty = a.gate_type[g];
    C2 m[2][2];
    gate_m(ty, ty <= QSIM_RZ ? prefix_angle<T>(a, g, b) : 0.0, m);
    const C2 w0 = ca(cm(m[0][0], v0), cm(m[0][1], v1)), w1 = ca(cm(m[1][0], v0), cm(m[1][1], v1));
    v0 = w0;
    v1 = w1;
  }
  T* out = reinterpret_cast<T*>(a.phi) + id * 4;
  out[0] = (T)v0.r; out[1] = (T)v0.i; out[2] = (T)v1.r; out[3] = (T)v1.i;
}

// Warp per (sample, qubit). mu_q(beta) = sum over the first pass's tiles of the tile's partial for q
// (tile qubit: slot 2j + beta; qubit outside the tile: slot 2K where the tile has bit beta) times the
// phi of the tile's other outside qubits. Then the adjoint of the short prefix chain: with r the row
// vector mu^T G_m ... G_{j+1} and v_j = G_j ... G_1 |0>,
//   dL/dtheta_j = 2 Re[ r (-i/2) P_j v_j ],
// walking j down from m (r <- r G_j, v <- G_j^dag v).
template <typename T>
__global__ void prefix_grad_kernel(PrefixArgs a) {
  const int b = blockIdx.x / a.n, q = blockIdx.x - (blockIdx.x / a.n) * a.n;
  const unsigned lane = threadIdx.x;
  int jq = -1, iq = -1;   // q as tile bit jq or tile-index bit iq of the first pass
  for (int j = 0; j < a.K; j++)
    if (a.Qnl[j] == q) jq = j;
  for (int i = 0; i < a.n_nonlocal; i++)
    if (a.Qnl[a.K + i] == q) iq = i;
  const T* ph = reinterpret_cast<const T*>(a.phi) + (int64_t)b * a.n * 4;
  const int NS = 2 * a.K + 1;
  C2 mu0 = {0, 0}, mu1 = {0, 0};
  for (int64_t t = lane; t < a.tps; t += 32) {
    C2 F = {1, 0};
    for (int i = 0; i < a.n_nonlocal; i++) {
      if (i == iq) continue;
      const T* f = ph + 4 * a.Qnl[a.K + i] + 2 * ((t >> i) & 1);
      F = cm(F, C2{(double)f[0], (double)f[1]});
    }
    const double* row = a.ppart + ((int64_t)b * a.tps + t) * NS * 2;
    if (jq >= 0) {
      mu0 = ca(mu0, cm(C2{row[4 * jq], row[4 * jq + 1]}, F));
      mu1 = ca(mu1, cm(C2{row[4 * jq + 2], row[4 * jq + 3]}, F));
    } else {
      const C2 v = cm(C2{row[4 * a.K], row[4 * a.K + 1]}, F);
      if ((t >> iq) & 1) mu1 = ca(mu1, v);
      else mu0 = ca(mu0, v);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {   // fixed tree: the same order every run
    mu0.r += __shfl_xor_sync(0xffffffffu, mu0.r, off);
    mu0.i += __shfl_xor_sync(0xffffffffu, mu0.i, off);
    mu1.r += __shfl_xor_sync(0xffffffffu, mu1.r, off);
    mu1.i += __shfl_xor_sync(0xffffffffu, mu1.i, off);
  }
  if (lane != 0) return;
  // v = phi_q in FP64, then the chain backwards
  C2 v0 = {1, 0}, v1 = {0, 0};
  const int e0 = a.pfx_begin[q], e1 = a.pfx_begin[q + 1];
  for (int e = e0; e < e1; e++) {
    const int g = a.pfx_gate[e], ty = a.gate_type[g];
    C2 m[2][2];
    gate_m(ty, ty <= QSIM_RZ ? prefix_angle<T>(a, g, b) : 0.0, m);
    const C2 w0 = ca(cm(m[0][0], v0), cm(m[0][1], v1)), w1 = ca(cm(m[1][0], v0), cm(m[1][1], v1));
    v0 = w0;
    v1 = w1;
  }
  C2 r0 = mu0, r1 = mu1;
  for (int e = e1 - 1; e >= e0; e--) {
    const int g = a.pfx_gate[e], ty = a.gate_type[g];
    C2 m[2][2];
    gate_m(ty, ty <= QSIM_RZ ? prefix_angle<T>(a, g, b) : 0.0, m);
    if (ty <= QSIM_RZ && a.pfx_occ[e] >= 0) {
      // P v with P = X, Y or Z, then times -i/2
      C2 p0, p1;
      if (ty == QSIM_RX) { p0 = v1; p1 = v0; }
      else if (ty == QSIM_RY) { p0 = {v1.i, -v1.r}; p1 = {-v0.i, v0.r}; }   // Y = [[0, -i], [i, 0]]
      else { p0 = v0; p1 = {-v1.r, -v1.i}; }
      const C2 d0 = {0.5 * p0.i, -0.5 * p0.r}, d1 = {0.5 * p1.i, -0.5 * p1.r};   // (-i/2) P v
      const C2 s = ca(cm(r0, d0), cm(r1, d1));
      a.G[(int64_t)a.pfx_occ[e] * a.B + b] = 2.0 * s.r;
    }
    // r <- r G_j ; v <- G_j^dag v
    const C2 n0 = ca(cm(r0, m[0][0]), cm(r1, m[1][0])), n1 = ca(cm(r0, m[0][1]), cm(r1, m[1][1]));
    r0 = n0;
    r1 = n1;
    const C2 c00 = {m[0][0].r, -m[0][0].i}, c01 = {m[1][0].r, -m[1][0].i};   // rows of G^dag
    const C2 c10 = {m[0][1].r, -m[0][1].i}, c11 = {m[1][1].r, -m[1][1].i};
    const C2 u0 = ca(cm(c00, v0), cm(c01, v1)), u1 = ca(cm(c10, v0), cm(c11, v1));
    v0 = u0;
    v1 = u1;
  }
}

cudaError_t launch_prefix_phi(const PrefixArgs& a, int dtype, cudaStream_t st) {
  const int64_t tot = (int64_t)a.B * a.n;
  if (tot == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((tot + 127) / 128);
  if (dtype == QSIM_C128) prefix_phi_kernel<double><<<blocks, 128, 0, st>>>(a);
  else prefix_phi_kernel<float><<<blocks, 128, 0, st>>>(a);
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_prefix_grad(const PrefixArgs& a, int dtype, cudaStream_t st) {
  const int64_t tot = (int64_t)a.B * a.n;
  if (tot == 0) return cudaSuccess;
  if (dtype == QSIM_C128) prefix_grad_kernel<double><<<(unsigned)tot, 32, 0, st>>>(a);
  else prefix_grad_kernel<float><<<(unsigned)tot, 32, 0, st>>>(a);
  g_kernel_launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ several circuits
// <Z>: block per (circuit, sample, qubit), flattened in circuit order; circuit found by bisection.
__global__ void z_final_multi_kernel(ZMultiArgs a) {
  __shared__ double sh[32];
  const int64_t gz = blockIdx.x;
  int lo = 0, hi = a.C;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if ((int64_t)a.B * a.zq_off[mid] <= gz) lo = mid;
    else hi = mid;
  }
  const int c = lo;
  const ZCirc d = a.circ[c];
  if (d.k < 0) return;   // a circuit run by its own single-circuit plan writes its <Z> itself
  const int64_t r = gz - (int64_t)a.B * a.zq_off[c];
  const int b = (int)(r / d.n), q = (int)(r - (int64_t)b * d.n);
  const uint8_t* Qnl = a.bits + d.bits_off;   // logical qubits of the last pass's tile and tile-index bits
  int tbit = -1, nlbit = -1;
  for (int j = 0; j < d.k; j++)
    if (Qnl[j] == q) tbit = j;
  for (int j = 0; j < d.n_nonlocal; j++)
    if (Qnl[d.k + j] == q) nlbit = j;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < d.tps; t += blockDim.x) {
    const double* row = a.zpart + d.zp_off + ((int64_t)b * d.tps + t) * (d.k + 1);
    if (tbit >= 0) acc += row[tbit];
    else acc += ((t >> nlbit) & 1) ? -row[d.k] : row[d.k];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) a.z[gz] = acc;
}

cudaError_t launch_z_final_multi(const ZMultiArgs& a, int64_t total, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  z_final_multi_kernel<<<(unsigned)total, 256, 0, st>>>(a);
  g_kernel_launches++;
  return cudaGetLastError();
}

// gradients: G[j][b] = gm * sum over tiles of the occurrence's partials (block per (j, b))
__global__ void grad_gather_multi_kernel(GradMultiArgs a) {
  __shared__ double sh[32];
  const int j = blockIdx.x / a.B, b = blockIdx.x - (blockIdx.x / a.B) * a.B;
  const int64_t tps = a.occ_tps[j];
  const double* src = a.gpart + a.occ_base[j] + (int64_t)b * tps;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < tps; t += blockDim.x) acc += src[t];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) a.G[(int64_t)j * a.B + b] = acc * a.gm[(int64_t)a.occ_gate[j] * a.B + b];
}

__global__ void grad_scatter_multi_kernel(GradMultiArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = a.dparams ? a.n_params : 0;
  const int64_t ni = a.dinputs ? (int64_t)a.n_cols * a.B : 0;
  if (id < np) {
    double acc = 0.0;
    for (int o = a.p_ptr[id]; o < a.p_ptr[id + 1]; o++) {
      const double* row = a.G + (int64_t)a.p_occ[o] * a.B;
      for (int b = 0; b < a.B; b++) acc += row[b];
    }
    a.dparams[id] = a.weight_remap ? acc * remap_slope(a.params, id, a.dtype) : acc;
  } else if (id < np + ni) {
    const int64_t r = id - np;
    const int64_t gc = r / a.B;
    const int b = (int)(r - gc * a.B);
    double acc = 0.0;
    for (int o = a.i_ptr[gc]; o < a.i_ptr[gc + 1]; o++) acc += a.G[(int64_t)a.i_occ[o] * a.B + b];
    a.dinputs[(int64_t)a.B * a.col_circ_off[gc] + (int64_t)b * a.col_stride[gc] + a.col_index[gc]] = acc;
  }
}

cudaError_t launch_grad_reduce_multi(const GradMultiArgs& a, cudaStream_t st) {
  if (a.n_occ > 0 && a.B > 0) {
    grad_gather_multi_kernel<<<(unsigned)(a.n_occ * a.B), 256, 0, st>>>(a);
    g_kernel_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t total = (a.dparams ? a.n_params : 0) + (a.dinputs ? (int64_t)a.n_cols * a.B : 0);
  if (total > 0) {
    grad_scatter_multi_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
    g_kernel_launches++;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ standalone <Z>
// Block = 2^ZB consecutive amplitudes of one sample (ZB = min(n, 12)); each thread accumulates
// its elements' |psi|^2 and signed sums over the index bits that vary inside its own elements,
// the block turns those into (ZB + 1) partials, a final pass maps bits to qubits.
constexpr int kZBits = 12;
constexpr int kZThreads = 256;

template <typename T>
__global__ void z_partials_kernel(const T* states, int n, int zb, double* part) {
  __shared__ double sred[kZThreads * 6];
  const int64_t blocks_per_sample = (int64_t)1 << (n - zb);
  const int64_t blk = blockIdx.x;
  const int b = (int)(blk / blocks_per_sample);
  const int64_t base = ((int64_t)b << n) + ((blk - (int64_t)b * blocks_per_sample) << zb);
  const int nthr = blockDim.x;
  int lg = 0;
  while ((1 << lg) < nthr) lg++;
  const int per = (1 << zb) >> lg;          // elements per thread (>= 1), stride nthr
  int nb = 0;
  while ((1 << nb) < per) nb++;
  double tot = 0.0, sg[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < per; i++) {
    const int64_t x = base + threadIdx.x + (int64_t)i * nthr;
    const double re = (double)states[2 * x], im = (double)states[2 * x + 1];
    const double p = re * re + im * im;
    tot += p;
    for (int r = 0; r < nb; r++) sg[r] += ((i >> r) & 1) ? -p : p;
  }
  sred[threadIdx.x * 6] = tot;
  for (int r = 0; r < 5; r++) sred[threadIdx.x * 6 + 1 + r] = sg[r];
  __syncthreads();
  for (int j = threadIdx.x; j <= zb; j += nthr) {
    double acc = 0.0;
    if (j == zb) {
      for (int u = 0; u < nthr; u++) acc += sred[u * 6];
    } else if (j < lg) {
      for (int u = 0; u < nthr; u++) acc += ((u >> j) & 1) ? -sred[u * 6] : sred[u * 6];
    } else {
      for (int u = 0; u < nthr; u++) acc += sred[u * 6 + 1 + (j - lg)];
    }
    part[blk * (zb + 1) + j] = acc;
  }
}

__global__ void z_block_final_kernel(const double* part, int n, int zb, int B, double* z) {
  __shared__ double sh[32];
  const int b = blockIdx.x / n, q = blockIdx.x - (blockIdx.x / n) * n;
  const int pos = n - 1 - q;
  const int64_t bps = (int64_t)1 << (n - zb);
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < bps; t += blockDim.x) {
    const double* row = part + ((int64_t)b * bps + t) * (zb + 1);
    if (pos < zb) acc += row[pos];
    else acc += ((t >> (pos - zb)) & 1) ? -row[zb] : row[zb];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) z[(int64_t)b * n + q] = acc;
}

int64_t z_partials_count(int n, int B) {
  const int zb = n < kZBits ? n : kZBits;
  return (int64_t)B * ((int64_t)1 << (n - zb)) * (zb + 1);
}

cudaError_t launch_expval_z(const void* states, int n, int B, int dtype, double* scratch, double* z,
                            cudaStream_t st);

// ------------------------------------------------------------------ <Z> without allocation
// Partial sums for callers that cannot allocate device memory live in this fixed array. It is part
// of the library's device image, so every GPU that loads the library holds it until the process
// exits. All calls share it: calls that overlap on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller. Nothing in it has to start at zero: each
// call writes every partial it later reads.
static __device__ __align__(256) double g_noalloc_zpart[kNoAllocZPartials];

namespace {
std::mutex g_noalloc_mu;
struct NoAllocSlot {
  void* ctx = nullptr;   // context the address was looked up in
  void* ptr = nullptr;   // address of g_noalloc_zpart on that device, in that context
};
NoAllocSlot g_noalloc[256];   // per device

// The CUDA driver API's cuCtxGetCurrent, reached through the runtime (no link against libcuda):
// the current context identifies the module instance that holds the array.
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

void* current_ctx() {
  void* c = nullptr;
  CtxGetCurrentFn fn = ctx_get_current();
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}
}  // namespace

cudaError_t launch_expval_z_noalloc(const void* states, int n, int B, int dtype, double* z, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  void* ptr = nullptr;
  {
    // set-up per device, with that device current: the host-side name of the array is not a device
    // address, so its device address is looked up and cached. The cache is keyed on the current
    // context, so a context re-created after cudaDeviceReset (a new instance of the array) is looked
    // up again instead of reusing a stale address.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot& slot = g_noalloc[dev];
    void* ctx = current_ctx();
    if (!slot.ptr || !ctx || ctx != slot.ctx) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_zpart);   // also makes the primary context current
      if (e != cudaSuccess) {
        slot = NoAllocSlot{};
        return e;
      }
      slot.ptr = p;
      slot.ctx = current_ctx();
    }
    ptr = slot.ptr;
  }
  return launch_expval_z(states, n, B, dtype, reinterpret_cast<double*>(ptr), z, st);
}

cudaError_t launch_expval_z(const void* states, int n, int B, int dtype, double* scratch, double* z,
                            cudaStream_t st) {
  if ((int64_t)B * n == 0) return cudaSuccess;
  const int zb = n < kZBits ? n : kZBits;
  int thr = kZThreads;
  while (thr > (1 << zb)) thr >>= 1;
  if (thr < 32) thr = 32;
  const int64_t blocks = (int64_t)B << (n - zb);
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  if ((1 << zb) < thr) {
    // fewer amplitudes than a warp: the per-thread loop would be empty for some threads
    thr = 1 << zb;
  }
  if (dtype == QSIM_C128)
    z_partials_kernel<double><<<(unsigned)blocks, thr, 0, st>>>(reinterpret_cast<const double*>(states), n, zb, scratch);
  else
    z_partials_kernel<float><<<(unsigned)blocks, thr, 0, st>>>(reinterpret_cast<const float*>(states), n, zb, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  z_block_final_kernel<<<(unsigned)(B * n), 256, 0, st>>>(scratch, n, zb, B, z);
  g_kernel_launches += 2;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gradient landscape
template <typename T>
__global__ void landscape_rows_kernel(const T* base, const T* values, int P, int V, T* rows, const double* w, int n,
                                      double* gout) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t B = (int64_t)P * V;
  if (id < B * P) {
    const int64_t b = id / P;
    const int j = (int)(id - b * P), k = (int)(b / V), v = (int)(b - (int64_t)k * V);
    rows[id] = j == k ? values[v] : base[j];
  }
  if (id < B * n) gout[id] = w[id % n];
}

__global__ void landscape_gather_kernel(const double* dinputs, int P, int V, double* grid) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)P * V) return;
  const int k = (int)(id / V);
  grid[id] = dinputs[id * P + k];   // sample id = k * V + v varied parameter k
}

cudaError_t launch_landscape_inputs(const void* base, const void* values, int P, int V, int dtype, void* rows,
                                    const double* weights, int n, double* gout, cudaStream_t st) {
  const int64_t B = (int64_t)P * V, total = std::max<int64_t>(B * P, B * n);
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (dtype == QSIM_C128)
    landscape_rows_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(base),
        static_cast<const double*>(values), P, V, static_cast<double*>(rows), weights, n, gout);
  else
    landscape_rows_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(base),
        static_cast<const float*>(values), P, V, static_cast<float*>(rows), weights, n, gout);
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_landscape_gather(const double* dinputs, int P, int V, double* grid, cudaStream_t st) {
  const int64_t total = (int64_t)P * V;
  if (total == 0) return cudaSuccess;
  landscape_gather_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dinputs, P, V, grid);
  g_kernel_launches++;
  return cudaGetLastError();
}

}  // namespace qsim

// Host test hook: the frame walk over one op list (types, target / control qubits, cotangent flags),
// returning each op's sign and the final frame.
extern "C" int qsim_frame_walk_host(const int32_t* types, const int32_t* q0, const int32_t* q1, const uint8_t* cot,
                                    int32_t n_ops, int8_t* sigma, uint64_t* x, uint64_t* z, int32_t* k) {
  if (n_ops < 0 || (n_ops > 0 && (!types || !q0 || !q1 || !cot || !sigma)) || !x || !z || !k) return QSIM_ERR_ARG;
  qsim::Frame f;
  for (int i = 0; i < n_ops; i++) sigma[i] = (int8_t)qsim::frame_step(f, types[i], q0[i], q1[i], cot[i]);
  *x = f.x;
  *z = f.z;
  *k = f.k;
  return QSIM_OK;
}


