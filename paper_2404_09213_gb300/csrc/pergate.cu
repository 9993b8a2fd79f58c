// Plain one-kernel-per-gate path: every gate is one full sweep over the batched state.
//
// This is the direct GPU counterpart of the paper's Sec. "Concept of Shapes" single-qubit update (reshape the
// state so the target qubit is its own axis, multiply by the 2x2) with no fusion at all. It is kept
// as the comparison baseline for the fused path and uses the same precision and reductions.
#include <cuda_runtime.h>

#include <type_traits>

#include "launch.hpp"

namespace qsim {

template <typename T> struct PgV2;
template <> struct PgV2<float> { using type = float2; };
template <> struct PgV2<double> { using type = double2; };

constexpr int kPgThreads = 256;
constexpr int kPgPairsPerThread = 4;
constexpr int kPgPairsPerBlock = kPgThreads * kPgPairsPerThread;

int pg_blocks_per_sample(int n) {
  const int64_t pairs = (int64_t)1 << (n > 0 ? n - 1 : 0);
  const int64_t b = (pairs + kPgPairsPerBlock - 1) / kPgPairsPerBlock;
  return (int)(b < 1 ? 1 : b);
}

// Full (unscaled) 2x2 of a gate from its stored scaled coefficient: M = scale * M_form(c).
template <typename T>
struct Mat2 {
  T ar, ai, br, bi, cr, ci, dr, di;   // [[a, b], [c, d]]
};

template <typename T>
__device__ __forceinline__ Mat2<T> gate_matrix(int type, T c, int form, T s) {
  Mat2<T> m{};
  const T one = T(1);
  if (type == QSIM_RY) {
    if (form == 0) m = {s, 0, -s * c, 0, s * c, 0, s, 0};
    else m = {s * c, 0, -s, 0, s, 0, s * c, 0};
  } else if (type == QSIM_RX) {
    if (form == 0) m = {s, 0, 0, -s * c, 0, -s * c, s, 0};
    else m = {s * c, 0, 0, -s, 0, -s, s * c, 0};
  } else if (type == QSIM_RZ) {
    if (form == 0) m = {s, -s * c, 0, 0, 0, 0, s, s * c};
    else m = {s * c, -s, 0, 0, 0, 0, s * c, s};
  } else if (type == QSIM_H) {
    m = {s, 0, s, 0, s, 0, -s, 0};
  } else {  // X
    m = {0, 0, one, 0, one, 0, 0, 0};
  }
  return m;
}

template <typename T, typename V>
__device__ __forceinline__ void apply2(const Mat2<T>& m, V& x, V& y) {
  const T xr = x.x, xi = x.y, yr = y.x, yi = y.y;
  x.x = m.ar * xr - m.ai * xi + m.br * yr - m.bi * yi;
  x.y = m.ar * xi + m.ai * xr + m.br * yi + m.bi * yr;
  y.x = m.cr * xr - m.ci * xi + m.dr * yr - m.di * yi;
  y.y = m.cr * xi + m.ci * xr + m.dr * yi + m.di * yr;
}

__device__ __forceinline__ int64_t insert_zero(int64_t v, int pos) {
  const int64_t lo = v & (((int64_t)1 << pos) - 1);
  return ((v >> pos) << (pos + 1)) | lo;
}

template <typename T>
__global__ void pg_init_kernel(typename PgV2<T>::type* st, const typename PgV2<T>::type* init, int n, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (init) st[i] = init[i];
    else {
      const bool one = (i & (((int64_t)1 << n) - 1)) == 0;
      st[i].x = one ? T(1) : T(0);
      st[i].y = T(0);
    }
  }
}

template <typename T>
__global__ void pg_gate_kernel(PerGateArgs a, typename PgV2<T>::type* st, bool inverse) {
  using V = typename PgV2<T>::type;
  const int n = a.n;
  const int64_t pairs = (int64_t)a.B << (n - 1);
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < pairs; id += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(id >> (n - 1));
    const int64_t base = (int64_t)b << n;
    const int64_t r = id - ((int64_t)b << (n - 1));
    if (a.type == QSIM_CNOT || a.type == QSIM_CZ) {
      // pairs over the target bit; act only where the control bit is 1
      const int64_t x0 = insert_zero(r, a.pos_t);
      if (!((x0 >> a.pos_c) & 1)) continue;
      const int64_t x1 = x0 | ((int64_t)1 << a.pos_t);
      if (a.type == QSIM_CNOT) {
        V u = st[base + x0], v = st[base + x1];
        st[base + x0] = v;
        st[base + x1] = u;
      } else {
        V v = st[base + x1];
        v.x = -v.x; v.y = -v.y;
        st[base + x1] = v;
      }
      continue;
    }
    const int64_t x0 = insert_zero(r, a.pos_t), x1 = x0 | ((int64_t)1 << a.pos_t);
    T c = T(0), s = T(1);
    int form = 0;
    if (a.type <= QSIM_RZ) {
      c = reinterpret_cast<const T*>(a.coef)[(int64_t)a.gate * a.B + b];
      form = a.form[(int64_t)a.gate * a.B + b];
      if (inverse) c = -c;
    }
    if (a.type <= QSIM_RZ || a.type == QSIM_H) s = reinterpret_cast<const T*>(a.scale)[b];
    const Mat2<T> m = gate_matrix<T>(a.type, c, form, s);
    V u = st[base + x0], v = st[base + x1];
    apply2(m, u, v);
    st[base + x0] = u;
    st[base + x1] = v;
  }
}

// Backward of one gate: gradient partial Im<lam|P|psi> (before undoing), then psi, lam <- U^dagger.
template <typename T>
__global__ void pg_bwd_kernel(PerGateArgs a, typename PgV2<T>::type* psi, typename PgV2<T>::type* lam,
                              double* gpart, int bps) {
  using V = typename PgV2<T>::type;
  using A = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  __shared__ double sh[kPgThreads / 32];
  const int n = a.n;
  const int b = blockIdx.x / bps;
  const int blk = blockIdx.x - b * bps;
  const int64_t base = (int64_t)b << n;
  const int64_t pairs_per_sample = (int64_t)1 << (n - 1);
  const bool rot = a.type <= QSIM_RZ;
  T c = T(0), s = T(1);
  int form = 0;
  if (rot) {
    c = -reinterpret_cast<const T*>(a.coef)[(int64_t)a.gate * a.B + b];
    form = a.form[(int64_t)a.gate * a.B + b];
  }
  if (rot || a.type == QSIM_H) s = reinterpret_cast<const T*>(a.scale)[b];
  const Mat2<T> m = (a.type == QSIM_CNOT || a.type == QSIM_CZ) ? Mat2<T>{} : gate_matrix<T>(a.type, c, form, s);
  A g = 0;
  for (int j = 0; j < kPgPairsPerThread; j++) {
    const int64_t r = (int64_t)blk * kPgPairsPerBlock + (int64_t)j * kPgThreads + threadIdx.x;
    if (r >= pairs_per_sample) break;
    const int64_t x0 = insert_zero(r, a.pos_t), x1 = x0 | ((int64_t)1 << a.pos_t);
    V p0 = psi[base + x0], p1 = psi[base + x1], l0 = lam[base + x0], l1 = lam[base + x1];
    if (a.type == QSIM_CNOT || a.type == QSIM_CZ) {
      if (!((x0 >> a.pos_c) & 1)) continue;
      if (a.type == QSIM_CNOT) {
        psi[base + x0] = p1; psi[base + x1] = p0;
        lam[base + x0] = l1; lam[base + x1] = l0;
      } else {
        p1.x = -p1.x; p1.y = -p1.y; l1.x = -l1.x; l1.y = -l1.y;
        psi[base + x1] = p1; lam[base + x1] = l1;
      }
      continue;
    }
    if (a.type == QSIM_RY) {
      g += (A)l1.x * (A)p0.x + (A)l1.y * (A)p0.y - (A)l0.x * (A)p1.x - (A)l0.y * (A)p1.y;
    } else if (a.type == QSIM_RX) {
      g += (A)l0.x * (A)p1.y - (A)l0.y * (A)p1.x + (A)l1.x * (A)p0.y - (A)l1.y * (A)p0.x;
    } else if (a.type == QSIM_RZ) {
      g += ((A)l0.x * (A)p0.y - (A)l0.y * (A)p0.x) - ((A)l1.x * (A)p1.y - (A)l1.y * (A)p1.x);
    }
    apply2(m, p0, p1);
    apply2(m, l0, l1);
    psi[base + x0] = p0; psi[base + x1] = p1;
    lam[base + x0] = l0; lam[base + x1] = l1;
  }
  if (!rot) return;
  double gd = (double)g;
  for (int off = 16; off > 0; off >>= 1) gd += __shfl_xor_sync(0xffffffffu, gd, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = gd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int w = 0; w < kPgThreads / 32; w++) acc += sh[w];
    gpart[(int64_t)b * bps + blk] = acc;
  }
}

template <typename T>
__global__ void pg_lambda_kernel(const typename PgV2<T>::type* st, typename PgV2<T>::type* psi,
                                 typename PgV2<T>::type* lam, const double* g, int n, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i >> n);
    const int64_t x = i - ((int64_t)b << n);
    double d = 0.0;
    for (int q = 0; q < n; q++) {
      const double gq = g[(int64_t)b * n + q];
      d += ((x >> (n - 1 - q)) & 1) ? -gq : gq;
    }
    auto v = st[i];
    psi[i] = v;
    lam[i].x = (T)(d * v.x);
    lam[i].y = (T)(d * v.y);
  }
}

static unsigned grid_for(int64_t work, int thr) {
  int64_t b = (work + thr - 1) / thr;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_pg_init(void* states, const void* init, int n, int B, int dtype, cudaStream_t st) {
  const int64_t total = (int64_t)B << n;
  if (total == 0) return cudaSuccess;
  if (init == states) return cudaSuccess;
  if (dtype == QSIM_C128)
    pg_init_kernel<double><<<grid_for(total, 256), 256, 0, st>>>(reinterpret_cast<double2*>(states),
                                                                 reinterpret_cast<const double2*>(init), n, total);
  else
    pg_init_kernel<float><<<grid_for(total, 256), 256, 0, st>>>(reinterpret_cast<float2*>(states),
                                                                reinterpret_cast<const float2*>(init), n, total);
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_pg_gate(const PerGateArgs& a, void* states, bool inverse, cudaStream_t st) {
  const int64_t pairs = (int64_t)a.B << (a.n - 1);
  if (pairs == 0) return cudaSuccess;
  if (a.dtype == QSIM_C128)
    pg_gate_kernel<double><<<grid_for(pairs, 256), 256, 0, st>>>(a, reinterpret_cast<double2*>(states), inverse);
  else
    pg_gate_kernel<float><<<grid_for(pairs, 256), 256, 0, st>>>(a, reinterpret_cast<float2*>(states), inverse);
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_pg_bwd_gate(const PerGateArgs& a, void* psi, void* lam, double* gpart_slot, int bps,
                               cudaStream_t st) {
  const int64_t blocks = (int64_t)a.B * bps;
  if (blocks == 0) return cudaSuccess;
  if (a.dtype == QSIM_C128)
    pg_bwd_kernel<double><<<(unsigned)blocks, kPgThreads, 0, st>>>(a, reinterpret_cast<double2*>(psi),
                                                                   reinterpret_cast<double2*>(lam), gpart_slot, bps);
  else
    pg_bwd_kernel<float><<<(unsigned)blocks, kPgThreads, 0, st>>>(a, reinterpret_cast<float2*>(psi),
                                                                  reinterpret_cast<float2*>(lam), gpart_slot, bps);
  g_kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_pg_lambda_init(const void* states, void* psi, void* lam, const double* g, int n, int B, int dtype,
                                  cudaStream_t st) {
  const int64_t total = (int64_t)B << n;
  if (total == 0) return cudaSuccess;
  if (dtype == QSIM_C128)
    pg_lambda_kernel<double><<<grid_for(total, 256), 256, 0, st>>>(
        reinterpret_cast<const double2*>(states), reinterpret_cast<double2*>(psi), reinterpret_cast<double2*>(lam), g, n, total);
  else
    pg_lambda_kernel<float><<<grid_for(total, 256), 256, 0, st>>>(
        reinterpret_cast<const float2*>(states), reinterpret_cast<float2*>(psi), reinterpret_cast<float2*>(lam), g, n, total);
  g_kernel_launches++;
  return cudaGetLastError();
}

}  // namespace qsim
