// Device code of the specialised fused-pass kernels. This file is compiled at plan time by NVRTC
// together with a generated "Spec" struct per distinct pass structure (register phases, op list
// and shared-memory layouts as compile-time constants); it includes no host or std headers.
//
// A CTA owns one tile: the 2^K amplitudes of one sample whose index bits outside the pass's local
// set are fixed (the reshape to (rest, group) of the paper's Sec. "Circuit Splitting", with the group axis held
// in shared memory). Load: 16-byte L2-cached global loads (ld.global.cg) of runs of 2^c contiguous
// amplitudes straight into registers. Compute:
// register phases of 2^R amplitudes per thread; rotations use the scaled one-FMA forms
//   RY: [[1,-t],[t,1]] / [[u,-1],[1,u]],  RX: [[1,-it],[-it,1]] / [[u,-i],[-i,u]],
//   RZ: diag(1-it, 1+it) / diag(u-i, u+i),   t = tan(theta/2), u = cot(theta/2),
// (the factored cos / sin is applied once per pass as the tile is stored), H as [[1,1],[1,-1]].
// The backward reverses every op with the negated coefficient and accumulates Im<lambda|P|psi>.

namespace qj {

typedef unsigned int u32;
typedef long long i64;
typedef unsigned char u8;

struct Args {
  const void* in;        // forward: states in (nullptr -> |0...0>); backward: psi in
  void* out;             // forward: states out; backward: psi out (nullptr -> not stored)
  const void* lam_in;    // backward: lambda in (nullptr -> lambda = (sum_i g_i Z_i) psi)
  void* lam_out;         // backward: lambda out
  const void* cfp;       // [B][n_ops] this pass's op coefficients per sample (backward: already negated)
  const u8* fmp;         // [B][n_ops] 0: tangent form, 1: cotangent form
  const void* scale;     // [B] this pass's scale (forward) or inverse scale (backward)
  double* zpart;         // forward <Z> partials [(B * tps) x (K + 1)] or nullptr
  double* gpart;         // backward gradient partials
  const double* grad_out;   // backward: dL/d<Z> (B x n)
  const void* phi;       // product-state prefix: [B][n][4] phi_q(0), phi_q(1) (first pass only; else nullptr)
  double* ppart;         // backward of the first pass: prefix contraction partials [(B * tps) x (2K + 1) x 2]
  i64 tps;               // tiles per sample
  i64 gpart_offset;      // first gradient slot of this pass
  i64 ntiles;            // tiles of the launch
  int n_nonlocal, n, B, b0;   // b0: first sample of this launch
  u8 L[16];              // tile bit j: physical bit in the layout the pass reads
  u8 nonlocal[40];       // tile-index bit i: physical bit in the layout the pass reads
  u8 Lo[16];             // the same in the layout the pass writes (qubits remapped between passes)
  u8 nonlocal_o[40];
  u8 Q[16];              // logical qubit of tile bit j
  u8 QN[40];             // logical qubit of tile-index bit i
};

__device__ __forceinline__ float fm(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fm(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------- register gates (stride S = 1 << bit)
template <int N, int S, typename T>
__device__ __forceinline__ void ry(T* re, T* im, T c, int f) {
  if (f == 0) {
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
        re[i] = fm(-c, br, ar); im[i] = fm(-c, bi, ai);
        re[j] = fm(c, ar, br);  im[j] = fm(c, ai, bi);
      }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
        re[i] = fm(c, ar, -br); im[i] = fm(c, ai, -bi);
        re[j] = fm(c, br, ar);  im[j] = fm(c, bi, ai);
      }
  }
}

template <int N, int S, typename T>
__device__ __forceinline__ void rx(T* re, T* im, T c, int f) {
  if (f == 0) {
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
        re[i] = fm(c, bi, ar);  im[i] = fm(-c, br, ai);
        re[j] = fm(c, ai, br);  im[j] = fm(-c, ar, bi);
      }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
        re[i] = fm(c, ar, bi);  im[i] = fm(c, ai, -br);
        re[j] = fm(c, br, ai);  im[j] = fm(c, bi, -ar);
      }
  }
}

template <int N, int S, typename T>
__device__ __forceinline__ void rz(T* re, T* im, T c, int f) {
  if (f == 0) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      const T cs = (i & S) ? -c : c;
      const T r = re[i], m = im[i];
      re[i] = fm(cs, m, r);
      im[i] = fm(-cs, r, m);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) {
      const T r = re[i], m = im[i];
      if (i & S) { re[i] = fm(c, r, -m); im[i] = fm(c, m, r); }
      else       { re[i] = fm(c, r, m);  im[i] = fm(c, m, -r); }
    }
  }
}

// RZ on a thread bit: s = +1 (bit 0) or -1 (bit 1) for all of the thread's elements
template <int N, typename T>
__device__ __forceinline__ void rz_t(T* re, T* im, T c, int f, T s) {
  if (f == 0) {
    const T cs = s * c;
#pragma unroll
    for (int i = 0; i < N; i++) {
      const T r = re[i], m = im[i];
      re[i] = fm(cs, m, r);
      im[i] = fm(-cs, r, m);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) {
      const T r = re[i], m = im[i];
      re[i] = fm(c, r, s * m);
      im[i] = fm(c, m, -s * r);
    }
  }
}

template <int N, int S, typename T>
__device__ __forceinline__ void hd(T* re, T* im) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
      re[i] = ar + br; im[i] = ai + bi;
      re[j] = ar - br; im[j] = ai - bi;
    }
}

// X and CNOT with both operands in registers: swaps (register renaming after inlining)
template <int N, int SA, int SB, typename T>
__device__ __forceinline__ void swp(T* re, T* im) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SB) == SB && !(i & SA)) {
      const int j = i | SA;
      const T tr = re[i], ti = im[i];
      re[i] = re[j]; im[i] = im[j];
      re[j] = tr; im[j] = ti;
    }
}

// p != 0 ? a : b as a predicated select. Written as C++ conditionals, the register swaps of a CNOT
// whose control is a thread bit were compiled as branches that kept both register assignments live.
__device__ __forceinline__ float sel(u32 p, float a, float b) {
  float r;
  asm("{ .reg .pred q; setp.ne.u32 q, %1, 0; selp.f32 %0, %2, %3, q; }" : "=f"(r) : "r"(p), "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ double sel(u32 p, double a, double b) {
  double r;
  asm("{ .reg .pred q; setp.ne.u32 q, %1, 0; selp.f64 %0, %2, %3, q; }" : "=d"(r) : "r"(p), "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ float2 sel2(u32 p, float2 a, float2 b) { return make_float2(sel(p, a.x, b.x), sel(p, a.y, b.y)); }

template <int N, int SA, typename T>
__device__ __forceinline__ void cnot_t(T* re, T* im, bool ctl) {
  const u32 p = ctl ? 1u : 0u;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & SA)) {
      const int j = i | SA;
      const T ar = re[i], ai = im[i], br = re[j], bi = im[j];
      re[i] = sel(p, br, ar); im[i] = sel(p, bi, ai);
      re[j] = sel(p, ar, br); im[j] = sel(p, ai, bi);
    }
}

template <int N, int SA, int SB, typename T>
__device__ __forceinline__ void cz(T* re, T* im) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SA) && (i & SB)) { re[i] = -re[i]; im[i] = -im[i]; }
}

template <int N, int SA, typename T>
__device__ __forceinline__ void cz_t(T* re, T* im, bool o) {
  const T sg = o ? T(-1) : T(1);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (i & SA) { re[i] *= sg; im[i] *= sg; }
}

template <int N, typename T>
__device__ __forceinline__ void scal(T* re, T* im, T s) {
#pragma unroll
  for (int i = 0; i < N; i++) { re[i] *= s; im[i] *= s; }
}

// ---------------------------------------------------------------- backward, psi and lambda packed (complex64)
// X[i] = (Re psi_i, Re lambda_i), Y[i] = (Im psi_i, Im lambda_i). psi and lambda take the same update in
// the backward, so with the tangent form only (Pauli frame) each update of both states is one packed
// FP32x2 FMA: 2 packed FMAs per amplitude and rotation instead of 4 scalar ones.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int N, int S>
__device__ __forceinline__ void ry_p(float2* X, float2* Y, float c) {
  const float2 cp = f2(c), cn = f2(-c);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      const float2 a = X[i], u = Y[i], b = X[j], v = Y[j];
      X[i] = pfma(cn, b, a); Y[i] = pfma(cn, v, u);
      X[j] = pfma(cp, a, b); Y[j] = pfma(cp, u, v);
    }
}

template <int N, int S>
__device__ __forceinline__ void rx_p(float2* X, float2* Y, float c) {
  const float2 cp = f2(c), cn = f2(-c);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      const float2 a = X[i], u = Y[i], b = X[j], v = Y[j];
      X[i] = pfma(cp, v, a); Y[i] = pfma(cn, b, u);
      X[j] = pfma(cp, u, b); Y[j] = pfma(cn, a, v);
    }
}

template <int N, int S>
__device__ __forceinline__ void rz_p(float2* X, float2* Y, float c) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    const float cs = (i & S) ? -c : c;
    const float2 r = X[i], m = Y[i];
    X[i] = pfma(f2(cs), m, r);
    Y[i] = pfma(f2(-cs), r, m);
  }
}

// RZ on a thread bit: s = +1 (bit 0) or -1 (bit 1) for all of the thread's elements
template <int N>
__device__ __forceinline__ void rz_tp(float2* X, float2* Y, float c, float s) {
  const float2 cp = f2(s * c), cn = f2(-s * c);
#pragma unroll
  for (int i = 0; i < N; i++) {
    const float2 r = X[i], m = Y[i];
    X[i] = pfma(cp, m, r);
    Y[i] = pfma(cn, r, m);
  }
}

template <int N, int S>
__device__ __forceinline__ void hd_p(float2* X, float2* Y) {
  const float2 m1 = f2(-1.f);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      const float2 a = X[i], u = Y[i], b = X[j], v = Y[j];
      X[i] = __fadd2_rn(a, b); Y[i] = __fadd2_rn(u, v);
      X[j] = pfma(m1, b, a); Y[j] = pfma(m1, v, u);
    }
}

template <int N, int SA, int SB>
__device__ __forceinline__ void swp_p(float2* X, float2* Y) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SB) == SB && !(i & SA)) {
      const int j = i | SA;
      const float2 t = X[i], w = Y[i];
      X[i] = X[j]; Y[i] = Y[j];
      X[j] = t; Y[j] = w;
    }
}

template <int N, int SA>
__device__ __forceinline__ void cnot_tp(float2* X, float2* Y, bool ctl) {
  const u32 p = ctl ? 1u : 0u;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & SA)) {
      const int j = i | SA;
      const float2 a = X[i], u = Y[i], b = X[j], v = Y[j];
      X[i] = sel2(p, b, a); Y[i] = sel2(p, v, u);
      X[j] = sel2(p, a, b); Y[j] = sel2(p, u, v);
    }
}

template <int N, int SA, int SB>
__device__ __forceinline__ void cz_p(float2* X, float2* Y) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SA) && (i & SB)) { X[i] = __fmul2_rn(X[i], f2(-1.f)); Y[i] = __fmul2_rn(Y[i], f2(-1.f)); }
}

template <int N, int SA>
__device__ __forceinline__ void cz_tp(float2* X, float2* Y, bool o) {
  const float2 sg = f2(o ? -1.f : 1.f);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (i & SA) { X[i] = __fmul2_rn(X[i], sg); Y[i] = __fmul2_rn(Y[i], sg); }
}

template <int N>
__device__ __forceinline__ void scal_p(float2* X, float2* Y, float s) {
#pragma unroll
  for (int i = 0; i < N; i++) { X[i] = __fmul2_rn(X[i], f2(s)); Y[i] = __fmul2_rn(Y[i], f2(s)); }
}

// ---------------------------------------------------------------- gradient partials (before undoing)
template <typename T> struct Acc { typedef float t; };
template <> struct Acc<double> { typedef double t; };

// Gradient inner products over the thread's N amplitude pairs. Four partial sums (by pair index mod 4)
// keep the FMA dependency chains short; they are added in a fixed order.
template <typename A>
__device__ __forceinline__ A sum4(const A* g) { return (g[0] + g[1]) + (g[2] + g[3]); }

template <int N, int S, typename T>
__device__ __forceinline__ typename Acc<T>::t g_ry(const T* pr, const T* pi, const T* lr, const T* li) {
  typedef typename Acc<T>::t A;
  A g[4] = {0, 0, 0, 0};
  int n = 0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Re(l1* p0) - Re(l0* p1)
      A& h = g[n++ & 3];
      h = fm((A)lr[j], (A)pr[i], h);
      h = fm((A)li[j], (A)pi[i], h);
      h = fm(-(A)lr[i], (A)pr[j], h);
      h = fm(-(A)li[i], (A)pi[j], h);
    }
  return sum4(g);
}

template <int N, int S, typename T>
__device__ __forceinline__ typename Acc<T>::t g_rx(const T* pr, const T* pi, const T* lr, const T* li) {
  typedef typename Acc<T>::t A;
  A g[4] = {0, 0, 0, 0};
  int n = 0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Im(l0* p1) + Im(l1* p0)
      A& h = g[n++ & 3];
      h = fm((A)lr[i], (A)pi[j], h);
      h = fm(-(A)li[i], (A)pr[j], h);
      h = fm((A)lr[j], (A)pi[i], h);
      h = fm(-(A)li[j], (A)pr[i], h);
    }
  return sum4(g);
}

template <int N, int S, typename T>
__device__ __forceinline__ typename Acc<T>::t g_rz(const T* pr, const T* pi, const T* lr, const T* li) {
  typedef typename Acc<T>::t A;
  A g[4] = {0, 0, 0, 0};   // [0], [1]: amplitudes with the bit clear; [2], [3]: set
  int n0 = 0, n1 = 0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    A& h = (i & S) ? g[2 + (n1++ & 1)] : g[n0++ & 1];
    h = fm((A)lr[i], (A)pi[i], h);
    h = fm(-(A)li[i], (A)pr[i], h);
  }
  return (g[0] + g[1]) - (g[2] + g[3]);
}

template <int N, typename T>
__device__ __forceinline__ typename Acc<T>::t g_im(const T* pr, const T* pi, const T* lr, const T* li) {
  typedef typename Acc<T>::t A;
  A g[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < N; i++) {
    A& h = g[i & 3];
    h = fm((A)lr[i], (A)pi[i], h);
    h = fm(-(A)li[i], (A)pr[i], h);
  }
  return sum4(g);
}

// The same inner products on packed registers (psi = .x, lambda = .y; X real parts, Y imaginary parts).
template <int N, int S>
__device__ __forceinline__ float g_ry_p(const float2* X, const float2* Y) {
  float g[4] = {0, 0, 0, 0};
  int n = 0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Re(l1* p0) - Re(l0* p1)
      float& h = g[n++ & 3];
      h = fm(X[j].y, X[i].x, h);
      h = fm(Y[j].y, Y[i].x, h);
      h = fm(-X[i].y, X[j].x, h);
      h = fm(-Y[i].y, Y[j].x, h);
    }
  return sum4(g);
}

template <int N, int S>
__device__ __forceinline__ float g_rx_p(const float2* X, const float2* Y) {
  float g[4] = {0, 0, 0, 0};
  int n = 0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Im(l0* p1) + Im(l1* p0)
      float& h = g[n++ & 3];
      h = fm(X[i].y, Y[j].x, h);
      h = fm(-Y[i].y, X[j].x, h);
      h = fm(X[j].y, Y[i].x, h);
      h = fm(-Y[j].y, X[i].x, h);
    }
  return sum4(g);
}

template <int N, int S>
__device__ __forceinline__ float g_rz_p(const float2* X, const float2* Y) {
  float g[4] = {0, 0, 0, 0};   // [0], [1]: amplitudes with the bit clear; [2], [3]: set
  int n0 = 0, n1 = 0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    float& h = (i & S) ? g[2 + (n1++ & 1)] : g[n0++ & 1];
    h = fm(X[i].y, Y[i].x, h);
    h = fm(-Y[i].y, X[i].x, h);
  }
  return (g[0] + g[1]) - (g[2] + g[3]);
}

template <int N>
__device__ __forceinline__ float g_im_p(const float2* X, const float2* Y) {
  float g[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < N; i++) {
    float& h = g[i & 3];
    h = fm(X[i].y, Y[i].x, h);
    h = fm(-Y[i].y, X[i].x, h);
  }
  return sum4(g);
}

// Shared memory of the packed backward: one 16-byte word (Re psi, Re lambda, Im psi, Im lambda) per
// amplitude; a register pair (elements e, e ^ 1) is two words.
__device__ __forceinline__ void ldpp(const void* tile, u32 w, float2& x0, float2& y0, float2& x1, float2& y1) {
  const float4 a = reinterpret_cast<const float4*>(tile)[w], b = reinterpret_cast<const float4*>(tile)[w ^ 1u];
  x0 = make_float2(a.x, a.y); y0 = make_float2(a.z, a.w);
  x1 = make_float2(b.x, b.y); y1 = make_float2(b.z, b.w);
}
__device__ __forceinline__ u32 smem_u32(const void* p) {
  u32 r;
  asm("{ .reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t; }" : "=r"(r) : "l"(p));
  return r;
}
// The stores go out as two 8-byte halves per word, each straight from its register pair: written as
// one 16-byte store, the compiler first copied X and Y into four adjacent registers (about 3 MOVs per
// amplitude and exchange).
template <int OFF>
__device__ __forceinline__ void sts2o(u32 a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0+%3], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y), "n"(OFF) : "memory");
}
__device__ __forceinline__ void stpp(void* tile, u32 w, float2 x0, float2 y0, float2 x1, float2 y1) {
  const u32 base = smem_u32(tile);
  const u32 a0 = base + 16u * w, a1 = base + 16u * (w ^ 1u);
  sts2o<0>(a0, x0); sts2o<8>(a0, y0);
  sts2o<0>(a1, x1); sts2o<8>(a1, y1);
}
template <bool ADD>
__device__ __forceinline__ void ldppx(const void* tile, u32 s, u32 c, float2& x0, float2& y0, float2& x1, float2& y1) {
  ldpp(tile, ADD ? s + c : s ^ c, x0, y0, x1, y1);
}
template <bool ADD>
__device__ __forceinline__ void stppx(void* tile, u32 s, u32 c, float2 x0, float2 y0, float2 x1, float2 y1) {
  stpp(tile, ADD ? s + c : s ^ c, x0, y0, x1, y1);
}

// Sum over the NTHR threads of a tile group. Groups are aligned blocks of NTHR lanes; when several
// groups share a warp (CTA >= 32) every lane takes part, and xor offsets below NTHR stay inside a group.
template <int NTHR, typename A, int CTA = NTHR>
__device__ __forceinline__ A warp_sum(A v) {
  constexpr unsigned mask = CTA >= 32 ? 0xffffffffu : ((1u << CTA) - 1u);
#pragma unroll
  for (int off = (NTHR >= 32 ? 16 : NTHR / 2); off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
  return v;
}

// Sum over aligned groups of W neighbouring lanes (W a power of two <= 32); every lane gets its
// group's sum. Lanes outside a CTA of fewer than 32 threads do not take part.
template <int W, typename A, int CTA>
__device__ __forceinline__ A part_sum(A v) {
  constexpr unsigned mask = CTA >= 32 ? 0xffffffffu : ((1u << CTA) - 1u);
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
  return v;
}

// ---------------------------------------------------------------- pair access in shared memory
__device__ __forceinline__ void ldp(const void* tile, u32 w, float& r0, float& i0, float& r1, float& i1) {
  const float4 v = reinterpret_cast<const float4*>(tile)[w >> 1];
  r0 = v.x; i0 = v.y; r1 = v.z; i1 = v.w;
}
__device__ __forceinline__ void stp(void* tile, u32 w, float r0, float i0, float r1, float i1) {
  reinterpret_cast<float4*>(tile)[w >> 1] = make_float4(r0, i0, r1, i1);
}
__device__ __forceinline__ void ldp(const void* tile, u32 w, double& r0, double& i0, double& r1, double& i1) {
  const double2 a = reinterpret_cast<const double2*>(tile)[w], b = reinterpret_cast<const double2*>(tile)[w ^ 1u];
  r0 = a.x; i0 = a.y; r1 = b.x; i1 = b.y;
}
__device__ __forceinline__ void stp(void* tile, u32 w, double r0, double i0, double r1, double i1) {
  reinterpret_cast<double2*>(tile)[w] = make_double2(r0, i0);
  reinterpret_cast<double2*>(tile)[w ^ 1u] = make_double2(r1, i1);
}

// Pair access at element s ^ c, s the thread's part and c a compile-time constant (both with bit 0
// clear). ADD: s and c have no bit in common, so s ^ c == s + c and the constant becomes the
// instruction's address offset.
template <bool ADD, typename T>
__device__ __forceinline__ void ldpx(const void* tile, u32 s, u32 c, T& r0, T& i0, T& r1, T& i1) {
  if constexpr (sizeof(T) == 4) {
    const u32 q = ADD ? (s >> 1) + (c >> 1) : ((s ^ c) >> 1);
    const float4 v = reinterpret_cast<const float4*>(tile)[q];
    r0 = v.x; i0 = v.y; r1 = v.z; i1 = v.w;
  } else {
    ldp(tile, ADD ? s + c : s ^ c, r0, i0, r1, i1);
  }
}
template <bool ADD, typename T>
__device__ __forceinline__ void stpx(void* tile, u32 s, u32 c, T r0, T i0, T r1, T i1) {
  if constexpr (sizeof(T) == 4) {
    const u32 q = ADD ? (s >> 1) + (c >> 1) : ((s ^ c) >> 1);
    reinterpret_cast<float4*>(tile)[q] = make_float4(r0, i0, r1, i1);
  } else {
    stp(tile, ADD ? s + c : s ^ c, r0, i0, r1, i1);
  }
}

// ---------------------------------------------------------------- direct global <-> register I/O
// The first register phase loads its amplitudes straight from global memory and the last one stores
// them straight back; the planner keeps tile bits 1..3 as thread bits there, so lanes 0..7 of a warp
// cover one contiguous run of 16 amplitudes (128 bytes for complex64).
__device__ __forceinline__ void ldg_pair(const float* p, float& r0, float& i0, float& r1, float& i1) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  r0 = v.x; i0 = v.y; r1 = v.z; i1 = v.w;
}
__device__ __forceinline__ void ldg_pair(const double* p, double& r0, double& i0, double& r1, double& i1) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  r0 = a.x; i0 = a.y; r1 = b.x; i1 = b.y;
}
__device__ __forceinline__ void stg_pair(float* p, float r0, float i0, float r1, float i1) {
  *reinterpret_cast<float4*>(p) = make_float4(r0, i0, r1, i1);
}
__device__ __forceinline__ void stg_pair(double* p, double r0, double i0, double r1, double i1) {
  reinterpret_cast<double2*>(p)[0] = make_double2(r0, i0);
  reinterpret_cast<double2*>(p)[1] = make_double2(r1, i1);
}

// Per-tile context handed to the generated phase code.
template <typename T>
struct Ctx {
  const Args* a;
  void* tile;            // forward: the tile; backward: psi
  void* tile2;           // backward: lambda
  T* cf;                 // op coefficients of this tile's sample, [NOPS] = pass scale (shared memory)
  T* tab;                // factor tables of the merged diagonal runs (shared memory, 16-byte aligned)
  u8* fm;                // op forms (shared memory)
  T* gq;                 // backward, lambda init: g of every tile bit, [K] = fixed-bit part
  i64 base;              // element offset of the tile (bits outside the tile) in the batched state, read layout
  i64 base_out;          // the same in the layout the pass writes
  i64 b, t;              // sample, tile within the sample
  u32 tid;
  bool valid;
};

// ---------------------------------------------------------------- product-state prefix
// The qubits' prefix states phi_q (per sample: phi_q(0), phi_q(1) as four reals) multiply into the first
// pass's starting state psi(x) = prod_q phi_q(x_q). In the backward of that pass, with lambda the
// adjoint state at the same point, the prefix gradients need
//   mu_q(b) = sum_{x: x_q = b} conj(lambda(x)) prod_{q' != q} phi_q'(x_q'),
// which each tile contributes to through 2K + 1 complex partials: for tile bit j and b, the sum over
// the tile's elements with bit j = b of conj(lambda) times the product of the other tile qubits' phi
// (slot 2j + b), and the full contraction over the tile (slot 2K); the qubits outside the tile enter on
// the host side of the reduction (prefix_grad_kernel).
template <typename T>
__device__ __forceinline__ void cmul(T& ar, T& ai, T br, T bi) {
  const T r = ar * br - ai * bi;
  ai = ar * bi + ai * br;
  ar = r;
}

// A diagonal-run table entry (re at p[0], im at p[di]); with di = 1 one vector load.
__device__ __forceinline__ void ldtab(const float* p, int di, float& r, float& i) {
  if (di == 1) { const float2 v = *reinterpret_cast<const float2*>(p); r = v.x; i = v.y; }
  else { r = p[0]; i = p[di]; }
}
__device__ __forceinline__ void ldtab(const double* p, int di, double& r, double& i) {
  if (di == 1) { const double2 v = *reinterpret_cast<const double2*>(p); r = v.x; i = v.y; }
  else { r = p[0]; i = p[di]; }
}

// product of phi over the tile-index bits of tile t (the qubits outside the tile)
template <typename T>
__device__ __forceinline__ void phi_nonlocal(const Args& a, const T* ph, i64 t, T& re, T& im) {
  re = T(1);
  im = T(0);
  for (int i = 0; i < a.n_nonlocal; i++) {
    const T* f = ph + 4 * a.QN[i] + 2 * ((t >> i) & 1);
    cmul(re, im, f[0], f[1]);
  }
}

// Contraction of the thread's N = 2^R register elements w_i = conj(lambda_i) with the register qubits'
// factors f_r(bit r of i): S = full contraction; nu[r][b] = the same over elements with bit r = b,
// leaving factor r out. The high bits are contracted one at a time (C_r: w contracted over bits
// r..R-1, 2^r values); nu[r][b] pairs the half of C_(r+1) with bit r = b with the product state P_r of
// the factors of bits 0..r-1. About 5N complex multiply-adds instead of 3RN for per-element prefix and
// suffix products.
template <typename T, int R, int r>
struct PrefixStep {   // bit r of the contraction (compile-time r: every register index is a constant)
  static __device__ __forceinline__ void run(T* cr, T* ci, const T (*fr)[2], const T (*fi)[2], T (*nr)[2], T (*ni)[2]) {
    constexpr int H = 1 << r;
    T pr[H], pi[H];   // P_r
    pr[0] = T(1); pi[0] = T(0);
#pragma unroll
    for (int q = 0; q < r; q++)
#pragma unroll
      for (int j = 0; j < (1 << q); j++) {
        pr[j + (1 << q)] = pr[j]; pi[j + (1 << q)] = pi[j];
        cmul(pr[j + (1 << q)], pi[j + (1 << q)], fr[q][1], fi[q][1]);
        cmul(pr[j], pi[j], fr[q][0], fi[q][0]);
      }
#pragma unroll
    for (int b = 0; b < 2; b++) {
      T ar = T(0), ai = T(0);
#pragma unroll
      for (int j = 0; j < H; j++) {
        const T xr = cr[j + b * H], xi = ci[j + b * H];
        ar += xr * pr[j] - xi * pi[j];
        ai += xr * pi[j] + xi * pr[j];
      }
      nr[r][b] = ar; ni[r][b] = ai;
    }
#pragma unroll
    for (int j = 0; j < H; j++) {
      T ar = cr[j], ai = ci[j], br = cr[j + H], bi = ci[j + H];
      cmul(ar, ai, fr[r][0], fi[r][0]);
      cmul(br, bi, fr[r][1], fi[r][1]);
      cr[j] = ar + br; ci[j] = ai + bi;
    }
    PrefixStep<T, R, r - 1>::run(cr, ci, fr, fi, nr, ni);
  }
};
template <typename T, int R>
struct PrefixStep<T, R, -1> {
  static __device__ __forceinline__ void run(T*, T*, const T (*)[2], const T (*)[2], T (*)[2], T (*)[2]) {}
};

template <typename T, int N, int R>
__device__ __forceinline__ void prefix_contract(const T* wr, const T* wi, const T (*fr)[2], const T (*fi)[2],
                                                T& Sr, T& Si, T (*nr)[2], T (*ni)[2]) {
  T cr[N], ci[N];
#pragma unroll
  for (int i = 0; i < N; i++) { cr[i] = wr[i]; ci[i] = wi[i]; }
  PrefixStep<T, R, R - 1>::run(cr, ci, fr, fi, nr, ni);
  Sr = cr[0]; Si = ci[0];
}

// One prefix partial slot (re, im) of this thread into the per-warp sums in shared memory (ws, one row
// of 2 * NS values per warp); the caller synchronises before the first and after the last slot.
template <typename T, int NTHR, int CTA>
__device__ __forceinline__ void prefix_put(T vr, T vi, int slot, T* ws, int NS, u32 tid) {
  vr = warp_sum<NTHR, T, CTA>(vr);
  vi = warp_sum<NTHR, T, CTA>(vi);
  if ((tid & 31u) == 0u) {
    ws[(tid >> 5) * 2 * NS + 2 * slot] = vr;
    ws[(tid >> 5) * 2 * NS + 2 * slot + 1] = vi;
  }
}

// The tile's NS slots: warps summed in a fixed order (FP64), times the pass's backward scale sc
// (lambda_true = sc * lambda in the kernel), into ppart.
template <typename T, int NTHR>
__device__ __forceinline__ void prefix_store(const Ctx<T>& c, const T* ws, int NS, T sc) {
  constexpr int NW = NTHR >= 32 ? NTHR / 32 : 1;
  const Args& a = *c.a;
  for (int v = (int)c.tid; v < 2 * NS; v += NTHR) {
    double s = 0.0;
    for (int w = 0; w < NW; w++) s += (double)ws[w * 2 * NS + v];
    if (c.valid) a.ppart[(c.b * a.tps + c.t) * (2 * NS) + v] = s * (double)sc;
  }
}

// Block reduction of the <Z> partials of the last forward phase into zrow[0..K]: row[j] is the
// signed sum over tile bit j, row[K] the tile total. zmap[j] >= 0: register bit; else thread bit -1-zmap[j].
template <typename T, int K, int R, int NTHR, class Spec>
__device__ __forceinline__ void z_reduce_regs(void* smem, typename Acc<T>::t zt, const typename Acc<T>::t* zs,
                                              double* zrow, u32 tid, bool valid) {
  typedef typename Acc<T>::t A;
  constexpr int NZ = R + 1;
  A* red = reinterpret_cast<A*>(smem);
  __syncthreads();
  red[tid * NZ] = zt;
#pragma unroll
  for (int r = 0; r < R; r++) red[tid * NZ + 1 + r] = zs[r];
  __syncthreads();
  // row j of the tile's partials: K = total probability, register bit r = sum of zs[r], thread bit =
  // zt with the sign of that bit of the thread. In the state's precision inside the tile (a warp per
  // row: strided lane sums, then a butterfly); rows are FP64 from here on (z_final sums the tiles).
  auto term = [&](int j, int u) -> A {
    if (j == K) return red[u * NZ];
    const int zm = Spec::zmap(j);
    if (zm >= 0) return red[u * NZ + 1 + zm];
    const A x = red[u * NZ];
    return ((u >> (-1 - zm)) & 1) ? -x : x;
  };
  if constexpr (NTHR >= 32) {
    const u32 lane = tid & 31u, w = tid >> 5;
    for (int j = (int)w; j <= K; j += NTHR / 32) {
      A v = 0;
#pragma unroll
      for (int i = 0; i < NTHR / 32; i++) v += term(j, (int)lane + 32 * i);
      v = warp_sum<32, A, 32>(v);
      if (lane == 0u && valid) zrow[j] = (double)v;
    }
  } else {
    for (int j = (int)tid; j <= K; j += NTHR) {
      A v = 0;
      for (int u = 0; u < NTHR; u++) v += term(j, u);
      if (valid) zrow[j] = (double)v;
    }
  }
}

__device__ __forceinline__ void tile_coords(const Args& a, i64 tile, i64& b, i64& t, i64& base, i64& base_out) {
  b = tile / a.tps + a.b0;
  t = tile - (b - a.b0) * a.tps;
  base = b << a.n;
  base_out = base;
  for (int j = 0; j < a.n_nonlocal; j++)
    if ((t >> j) & 1) {
      base += (i64)1 << a.nonlocal[j];
      base_out += (i64)1 << a.nonlocal_o[j];
    }
}

// ---------------------------------------------------------------- forward pass
// Shared-memory bytes of one tile group (forward): tile (also the <Z> reduction area), coefficients and
// the pass scale (NOPS + 1 values), forms.
template <typename T, int K, int NOPS, int NTAB>
struct FwdGroupSmem {
  static constexpr int NO = NOPS + 1;
  static constexpr int TILE = (2 * (int)sizeof(T)) << K;
  static constexpr int TB = TILE;                               // diagonal-run factor tables
  static constexpr int CF = TB + NTAB * (int)sizeof(T);
  static constexpr int BYTES = (CF + NO * (int)sizeof(T) + NO + 15) & ~15;
};

// One tile (sample b0 + tile / tps) processed by the NTHR threads `tid` of a group owning `smem`.
// Every thread of the CTA calls this together (barriers are CTA-wide); a group with valid == false
// computes on another tile's data but writes nothing to global memory.
template <typename T, int K, int R, int NTHR, class Spec>
__device__ __forceinline__ void fwd_tile(const Args& a, i64 tile, bool valid, u32 tid, unsigned char* smem) {
  typedef FwdGroupSmem<T, K, Spec::NOPS, Spec::NTAB> SM;
  T* cf = reinterpret_cast<T*>(smem + SM::CF);
  Ctx<T> c;
  c.a = &a;
  c.tile = smem;
  c.tile2 = nullptr;
  c.cf = cf;
  c.tab = reinterpret_cast<T*>(smem + SM::TB);
  c.fm = reinterpret_cast<u8*>(cf + SM::NO);
  c.gq = nullptr;
  c.tid = tid;
  c.valid = valid;
  tile_coords(a, tile, c.b, c.t, c.base, c.base_out);
  Spec::template fwd_phases<T>(c);   // the first phase issues its loads, then calls stage_fwd and syncs
}

// Per-tile constants into shared memory: op coefficients and forms of sample c.b, the pass scale in
// slot NOPS. Called after the first phase has issued its global loads so the latencies overlap; the
// caller synchronises before the first op.
template <typename T, int NTHR, class Spec>
__device__ __forceinline__ void stage_fwd(Ctx<T>& c) {
  const Args& a = *c.a;
  T* cf = c.cf;
  u8* fm = c.fm;
  const T* src = reinterpret_cast<const T*>(a.cfp) + c.b * Spec::NOPS;
  const u8* fsrc = a.fmp + c.b * Spec::NOPS;
  for (int i = c.tid; i < Spec::NOPS; i += NTHR) {
    cf[i] = src[i];
    fm[i] = fsrc[i];
  }
  if (c.tid == (u32)(NTHR - 1)) cf[Spec::NOPS] = reinterpret_cast<const T*>(a.scale)[c.b];
  Spec::template build_tables<T>(c, src);
}

template <typename T, int K, int R, int NTHR, class Spec>
__device__ __forceinline__ void fwd_pass(const Args& a) {
  extern __shared__ __align__(16) unsigned char smem[];
  fwd_tile<T, K, R, NTHR, Spec>(a, (i64)blockIdx.x, true, threadIdx.x, smem);
}

// ---------------------------------------------------------------- backward pass
// Shared-memory bytes of one tile group (backward): psi, lambda, gradient warp partials, g per tile
// bit, coefficients and forms.
template <typename T, int K, int R, int NTHR, int NOPS, int NGS, int GS, int NTAB>
struct BwdGroupSmem {
  typedef typename Acc<T>::t A;
  static constexpr int NW = (NTHR + 31) / 32;
  static constexpr int NG = NGS > 0 ? NGS : 1;
  static constexpr int NO = NOPS + 1;
  static constexpr int TILE = (2 * (int)sizeof(T)) << K;
  // gradient partials [NG][NTHR >> GS]: one per slot and group of 2^GS neighbouring threads
  static constexpr int RED = 2 * TILE;
  static constexpr int GQ = (RED + NG * (NTHR >> GS) * (int)sizeof(A) + 15) & ~15;
  static constexpr int TB = (GQ + (K + 2) * 8 + 15) & ~15;     // diagonal-run factor tables
  static constexpr int CF = TB + NTAB * (int)sizeof(T);
  static constexpr int FM = CF + NO * (int)sizeof(T);
  static constexpr int BYTES = (FM + NO + 15) & ~15;
};

// Backward per-tile constants: negated op coefficients, forms, the inverse pass scale (slot NOPS) and,
// when lambda is formed on load, g of every tile bit ([K]: the fixed-bit part of the tile).
template <typename T, int K, int NTHR, class Spec>
__device__ __forceinline__ void stage_bwd(Ctx<T>& c) {
  const Args& a = *c.a;
  T* cf = c.cf;
  u8* fm = c.fm;
  const T* src = reinterpret_cast<const T*>(a.cfp) + c.b * Spec::NOPS;
  const u8* fsrc = a.fmp + c.b * Spec::NOPS;
  for (int i = c.tid; i < Spec::NOPS; i += NTHR) {
    cf[i] = src[i];
    fm[i] = fsrc[i];
  }
  if (c.tid == (u32)(NTHR - 1)) cf[Spec::NOPS] = reinterpret_cast<const T*>(a.scale)[c.b];
  Spec::template build_tables<T>(c, src);
  if (a.lam_in == nullptr) {
    // g in T: lambda = d psi is formed in T, and T sums keep the FP64 pipe (a small fraction of the
    // FP32 rate) out of the per-thread work; the fixed-bit part is summed in FP64 by one warp
    T* gq = c.gq;
    for (int j = c.tid; j < K; j += NTHR) gq[j] = (T)a.grad_out[c.b * a.n + a.Q[j]];
    if constexpr (NTHR >= 32) {
      if (c.tid < 32u) {
        double dc = 0.0;
        for (int q = (int)c.tid; q < a.n_nonlocal; q += 32) {
          const double g = a.grad_out[c.b * a.n + a.QN[q]];
          dc += ((c.t >> q) & 1) ? -g : g;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dc += __shfl_xor_sync(0xffffffffu, dc, o);
        if (c.tid == 0u) gq[K] = (T)dc;
      }
    } else if (c.tid == 0u) {
      double dc = 0.0;
      for (int q = 0; q < a.n_nonlocal; q++) {
        const double g = a.grad_out[c.b * a.n + a.QN[q]];
        dc += ((c.t >> q) & 1) ? -g : g;
      }
      gq[K] = (T)dc;
    }
  }
}

template <typename T, int K, int R, int NTHR, class Spec>
__device__ __forceinline__ void bwd_tile(const Args& a, i64 tile, bool valid, u32 tid, unsigned char* smem) {
  typedef typename Acc<T>::t A;
  typedef BwdGroupSmem<T, K, R, NTHR, Spec::NOPS, Spec::NGS, Spec::GS, Spec::NTAB> SM;
  A* red = reinterpret_cast<A*>(smem + SM::RED);
  Ctx<T> c;
  c.a = &a;
  c.tile = smem;
  c.tile2 = smem + SM::TILE;
  c.cf = reinterpret_cast<T*>(smem + SM::CF);
  c.tab = reinterpret_cast<T*>(smem + SM::TB);
  c.fm = smem + SM::FM;
  c.gq = reinterpret_cast<T*>(smem + SM::GQ);             // [K + 1]
  c.tid = tid;
  c.valid = valid;
  tile_coords(a, tile, c.b, c.t, c.base, c.base_out);
  Spec::template bwd_phases<T>(c, red);
  __syncthreads();
  // Every op stored one partial per group of 2^GS neighbouring threads (summed by shuffles first);
  // sum each gradient slot over the NP = NTHR >> GS partials in a fixed order: a warp per slot
  // (strided lane sums, then a butterfly) when there are at least 32, else a thread per slot.
  constexpr int NP = NTHR >> Spec::GS;
  if constexpr (NP >= 32) {
    const u32 lane = tid & 31u, w = tid >> 5;
    for (int sl = (int)w; sl < Spec::NGS; sl += NTHR / 32) {
      A v = 0;
#pragma unroll
      for (int j = 0; j < NP / 32; j++) v += red[sl * NP + (int)lane + 32 * j];
      v = warp_sum<32, A, 32>(v);
      if (lane == 0u && valid) a.gpart[((a.gpart_offset + sl) * a.B + c.b) * a.tps + c.t] = (double)v;
    }
  } else {
    for (int sl = (int)tid; sl < Spec::NGS; sl += NTHR) {
      A v = 0;
      for (int u = 0; u < NP; u++) v += red[sl * NP + u];
      if (valid) a.gpart[((a.gpart_offset + sl) * a.B + c.b) * a.tps + c.t] = (double)v;
    }
  }
}

template <typename T, int K, int R, int NTHR, class Spec>
__device__ __forceinline__ void bwd_pass(const Args& a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bwd_tile<T, K, R, NTHR, Spec>(a, (i64)blockIdx.x, true, threadIdx.x, smem);
}

// ---------------------------------------------------------------- persistent multi-circuit queue
// One work item = up to CTA/NTHR tiles of one pass of one circuit. Items are ordered so that every
// item a CTA waits on was claimed earlier by a resident CTA, so the waits always end; they are still
// bounded (globaltimer) and report QSIM_ERR_TIMEOUT (-8) through *status instead of hanging.
struct Item {
  int kind;          // pass structure (switch case of the queue kernel)
  int arg;           // index of the pass's Args
  i64 tile0;         // first tile of the item
  i64 ntiles;        // tiles of the whole pass launch (B * tiles per sample)
  int wait;          // counter to wait on (-1: none)
  int wait_target;   // value it must reach (items of the previous pass of this circuit)
  int done;          // counter incremented when the item is finished
  int pad;
};

struct MultiArgs {
  const Item* items;
  i64 n_items;
  unsigned long long* head;   // next item to claim
  int* counters;
  int* status;
  const Args* args;
  i64 timeout_ns;
  i64 withhold;               // test hook: item whose completion is never signalled (-1: none)
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: wait until the item's dependency is complete. false = gave up (status set to timeout), or
// another item has already recorded an error, so later items stop waiting at once.
__device__ __forceinline__ bool wait_dependency(const MultiArgs& m, const Item& it) {
  if (it.wait < 0) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned polls = 0; ld_acquire(m.counters + it.wait) < it.wait_target; polls++) {
    if ((polls & 31u) == 31u && *reinterpret_cast<const volatile int*>(m.status) != 0) return false;
    if ((long long)(gtimer() - t0) > m.timeout_ns) {
      atomicExch(m.status, -8);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}

}  // namespace qj
