// Register-level gate kernels on a thread's 2^R amplitudes (planar re[] / im[] arrays).
//
// Rotations R_P(theta) = exp(-i theta P / 2) are applied in a scaled form with one unit
// coefficient so that every output component costs one FMA (the paper's Eq. 1 writes R_x as
// cos(theta/2) R_xa + (-i sin(theta/2)) R_xb; factoring out the larger of cos/sin leaves a matrix
// with unit diagonal or unit off-diagonal):
//   form 0 (|tan| <= 1): R = cos(theta/2) * M0(t),  t = tan(theta/2)
//   form 1 (|tan| >  1): R = sin(theta/2) * M1(u),  u = cot(theta/2)
//   RY: M0 = [[1,-t],[t,1]]      M1 = [[u,-1],[1,u]]
//   RX: M0 = [[1,-it],[-it,1]]   M1 = [[u,-i],[-i,u]]
//   RZ: M0 = diag(1-it, 1+it)    M1 = diag(u-i, u+i)
// The scalar factors are multiplied into the pass's scale, applied once when the tile is stored.
// The inverse of each form is the same form with the coefficient negated (and the scale negated
// for form 1), so the backward reuses these routines. H is applied as [[1,1],[1,-1]] (scale 1/sqrt2).
#pragma once
#include <cuda_runtime.h>

#include "plan_types.h"

namespace qsim {

template <int R, int A>
struct RegRY {
  template <typename T>
  __device__ __forceinline__ static void run(T* re, T* im, T c, int form) {
    constexpr int N = 1 << R, S = 1 << A;
    if (form == 0) {
#pragma unroll
      for (int i = 0; i < N; i++)
        if (!(i & S)) {
          const int j = i | S;
          T ar = re[i], ai = im[i], br = re[j], bi = im[j];
          re[i] = fma(-c, br, ar); im[i] = fma(-c, bi, ai);
          re[j] = fma(c, ar, br);  im[j] = fma(c, ai, bi);
        }
    } else {
#pragma unroll
      for (int i = 0; i < N; i++)
        if (!(i & S)) {
          const int j = i | S;
          T ar = re[i], ai = im[i], br = re[j], bi = im[j];
          re[i] = fma(c, ar, -br); im[i] = fma(c, ai, -bi);
          re[j] = fma(c, br, ar);  im[j] = fma(c, bi, ai);
        }
    }
  }
};

template <int R, int A>
struct RegRX {
  template <typename T>
  __device__ __forceinline__ static void run(T* re, T* im, T c, int form) {
    constexpr int N = 1 << R, S = 1 << A;
    if (form == 0) {
#pragma unroll
      for (int i = 0; i < N; i++)
        if (!(i & S)) {
          const int j = i | S;
          T ar = re[i], ai = im[i], br = re[j], bi = im[j];
          re[i] = fma(c, bi, ar);  im[i] = fma(-c, br, ai);
          re[j] = fma(c, ai, br);  im[j] = fma(-c, ar, bi);
        }
    } else {
#pragma unroll
      for (int i = 0; i < N; i++)
        if (!(i & S)) {
          const int j = i | S;
          T ar = re[i], ai = im[i], br = re[j], bi = im[j];
          re[i] = fma(c, ar, bi);  im[i] = fma(c, ai, -br);
          re[j] = fma(c, br, ai);  im[j] = fma(c, bi, -ar);
        }
    }
  }
};

template <int R, int A>
struct RegRZ {
  template <typename T>
  __device__ __forceinline__ static void run(T* re, T* im, T c, int form) {
    constexpr int N = 1 << R, S = 1 << A;
    if (form == 0) {
#pragma unroll
      for (int i = 0; i < N; i++) {
        const T cs = (i & S) ? -c : c;     // (1 - i s c): s = +1 for bit 0, -1 for bit 1
        T r = re[i], m = im[i];
        re[i] = fma(cs, m, r);
        im[i] = fma(-cs, r, m);
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; i++) {
        T r = re[i], m = im[i];
        if (i & S) { re[i] = fma(c, r, -m); im[i] = fma(c, m, r); }    // (u + i)
        else       { re[i] = fma(c, r, m);  im[i] = fma(c, m, -r); }   // (u - i)
      }
    }
  }
};

template <int R, int A>
struct RegH {
  template <typename T>
  __device__ __forceinline__ static void run(T* re, T* im, T, int) {
    constexpr int N = 1 << R, S = 1 << A;
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        T ar = re[i], ai = im[i], br = re[j], bi = im[j];
        re[i] = ar + br; im[i] = ai + bi;
        re[j] = ar - br; im[j] = ai - bi;
      }
  }
};

template <int R, int A>
struct RegX {
  template <typename T>
  __device__ __forceinline__ static void run(T* re, T* im, T, int) {
    constexpr int N = 1 << R, S = 1 << A;
#pragma unroll
    for (int i = 0; i < N; i++)
      if (!(i & S)) {
        const int j = i | S;
        T tr = re[i], ti = im[i];
        re[i] = re[j]; im[i] = im[j];
        re[j] = tr; im[j] = ti;
      }
  }
};

// RZ on a thread bit: sign s (+1 for bit 0, -1 for bit 1) is the same for all of the thread's elements.
template <int R, typename T>
__device__ __forceinline__ void reg_rz_thread(T* re, T* im, T c, int form, T s) {
  constexpr int N = 1 << R;
  if (form == 0) {
    const T cs = s * c;
#pragma unroll
    for (int i = 0; i < N; i++) {
      T r = re[i], m = im[i];
      re[i] = fma(cs, m, r);
      im[i] = fma(-cs, r, m);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) {
      T r = re[i], m = im[i];
      re[i] = fma(c, r, s * m);
      im[i] = fma(c, m, -s * r);
    }
  }
}

// CNOT with target register A and control register B.
template <int R, int A, int B, typename T>
__device__ __forceinline__ void reg_cnot_rr_t(T* re, T* im) {
  constexpr int N = 1 << R, SA = 1 << A, SB = 1 << B;
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SB) && !(i & SA)) {
      const int j = i | SA;
      T tr = re[i], ti = im[i];
      re[i] = re[j]; im[i] = im[j];
      re[j] = tr; im[j] = ti;
    }
}

// CNOT with target register A and a per-thread control value.
template <int R, int A, typename T>
__device__ __forceinline__ void reg_cnot_rt(T* re, T* im, bool ctl) {
  constexpr int N = 1 << R, SA = 1 << A;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & SA)) {
      const int j = i | SA;
      T ar = re[i], ai = im[i], br = re[j], bi = im[j];
      re[i] = ctl ? br : ar; im[i] = ctl ? bi : ai;
      re[j] = ctl ? ar : br; im[j] = ctl ? ai : bi;
    }
}

template <int R, int A, int B, typename T>
__device__ __forceinline__ void reg_cz_rr(T* re, T* im) {
  constexpr int N = 1 << R, SA = 1 << A, SB = 1 << B;
#pragma unroll
  for (int i = 0; i < N; i++)
    if ((i & SA) && (i & SB)) { re[i] = -re[i]; im[i] = -im[i]; }
}

template <int R, int A, typename T>
__device__ __forceinline__ void reg_cz_rt(T* re, T* im, bool other) {
  constexpr int N = 1 << R, SA = 1 << A;
  const T sg = other ? T(-1) : T(1);
#pragma unroll
  for (int i = 0; i < N; i++)
    if (i & SA) { re[i] *= sg; im[i] *= sg; }
}

template <int R, typename T>
__device__ __forceinline__ void reg_scale(T* re, T* im, T s) {
#pragma unroll
  for (int i = 0; i < (1 << R); i++) { re[i] *= s; im[i] *= s; }
}

// ---------------------------------------------------------------- gradient partials
// Im<lambda|P|psi> over the thread's pairs on register bit A (before the gate is undone).
template <int R, int A, typename T>
__device__ __forceinline__ float grad_ry(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  float g = 0.f;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Re(l1* p0) - Re(l0* p1)
      g = fmaf((float)lr[j], (float)pr[i], g);
      g = fmaf((float)li[j], (float)pi[i], g);
      g = fmaf(-(float)lr[i], (float)pr[j], g);
      g = fmaf(-(float)li[i], (float)pi[j], g);
    }
  return g;
}

template <int R, int A, typename T>
__device__ __forceinline__ double grad_ry_d(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  double g = 0.0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      g += (double)lr[j] * pr[i] + (double)li[j] * pi[i] - (double)lr[i] * pr[j] - (double)li[i] * pi[j];
    }
  return g;
}

template <int R, int A, typename T>
__device__ __forceinline__ float grad_rx(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  float g = 0.f;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;   // Im(l0* p1) + Im(l1* p0);  Im(l* p) = lr pi - li pr
      g = fmaf((float)lr[i], (float)pi[j], g);
      g = fmaf(-(float)li[i], (float)pr[j], g);
      g = fmaf((float)lr[j], (float)pi[i], g);
      g = fmaf(-(float)li[j], (float)pr[i], g);
    }
  return g;
}

template <int R, int A, typename T>
__device__ __forceinline__ double grad_rx_d(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  double g = 0.0;
#pragma unroll
  for (int i = 0; i < N; i++)
    if (!(i & S)) {
      const int j = i | S;
      g += (double)lr[i] * pi[j] - (double)li[i] * pr[j] + (double)lr[j] * pi[i] - (double)li[j] * pr[i];
    }
  return g;
}

// RZ: sum over elements of s(e) Im(l* p), s = +1 where bit A is 0.
template <int R, int A, typename T>
__device__ __forceinline__ float grad_rz(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  float g0 = 0.f, g1 = 0.f;
#pragma unroll
  for (int i = 0; i < N; i++) {
    float t = fmaf((float)lr[i], (float)pi[i], -(float)li[i] * (float)pr[i]);
    if (i & S) g1 += t; else g0 += t;
  }
  return g0 - g1;
}

template <int R, int A, typename T>
__device__ __forceinline__ double grad_rz_d(const T* pr, const T* pi, const T* lr, const T* li) {
  constexpr int N = 1 << R, S = 1 << A;
  double g = 0.0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    double t = (double)lr[i] * pi[i] - (double)li[i] * pr[i];
    g += (i & S) ? -t : t;
  }
  return g;
}

template <int R, typename T>
__device__ __forceinline__ float grad_imsum(const T* pr, const T* pi, const T* lr, const T* li) {
  float g = 0.f;
#pragma unroll
  for (int i = 0; i < (1 << R); i++) g += fmaf((float)lr[i], (float)pi[i], -(float)li[i] * (float)pr[i]);
  return g;
}

template <int R, typename T>
__device__ __forceinline__ double grad_imsum_d(const T* pr, const T* pi, const T* lr, const T* li) {
  double g = 0.0;
#pragma unroll
  for (int i = 0; i < (1 << R); i++) g += (double)lr[i] * pi[i] - (double)li[i] * pr[i];
  return g;
}

}  // namespace qsim
