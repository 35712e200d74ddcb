// Device helpers shared by the wave kernels.
//
// The composed Laplacian L = -G^T G of the staggered scheme (paper Sec. 2,
// Eq. wave_equation; order 2M, radius R = 2M-1) is evaluated along each axis
// in the zero-sum form
//
//     (L P)_i = sum_{m=1..R} w_m ((P_{i+m} + P_{i-m}) - 2 P_i),
//
// so that L annihilates constants exactly in FP32 whatever the rounding of
// w_m.  (The usual form w_0 P_i + sum w_m (P_{i+m} + P_{i-m}) with a rounded
// w_0 adds a spurious mass term that shifts the low-frequency modes and, over
// a few thousand leapfrog steps, costs ~1e-5 relative accuracy.)
#pragma once

#include <cuda_runtime.h>

namespace pat {

__device__ __forceinline__ float f4get(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Pair term of one stencil offset: (a + b) - 2c, or in the difference form
// (a - c) + (b - c), whose differences are exact (Sterbenz) wherever the
// field is smooth, so the rounding error follows the local variation rather
// than the field's magnitude.
template <bool DIFF>
__device__ __forceinline__ float pair_term(float a, float b, float c, float c2) {
  return DIFF ? (a - c) + (b - c) : (a + b) - c2;
}

// Laplacian of a 2 (rows) x 4 (cols) block from a shared-memory tile,
// accumulated into L (ACC) or written to it.
//   S      tile base, row pitch `pitch` floats (pitch % 4 == 0)
//   srow   tile row of the block's first row (>= R, with R rows of halo
//          above and R + 1 below available)
//   scol   tile column of the block's first column (multiple of 4, >= 8,
//          with 8 columns of halo on the left and right available)
template <int R, bool DIFF = false, bool ACC = false>
__device__ __forceinline__ void lap_2x4(const float* __restrict__ S, int pitch, int srow, int scol,
                                        const float* __restrict__ w, float L[2][4]) {
  // y direction: the block's four columns over rows srow-R .. srow+1+R
  float4 col[2 + 2 * R];
#pragma unroll
  for (int i = 0; i < 2 + 2 * R; ++i) col[i] = *reinterpret_cast<const float4*>(S + (srow - R + i) * pitch + scol);
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float c = f4get(col[rr + R], j);
      const float c2 = c + c;
      float acc = ACC ? L[rr][j] : 0.f;
#pragma unroll
      for (int m = 1; m <= R; ++m)
        acc = fmaf(w[m], pair_term<DIFF>(f4get(col[rr + R + m], j), f4get(col[rr + R - m], j), c, c2), acc);
      L[rr][j] = acc;
    }
  }
  // x direction: each row over columns scol-8 .. scol+11
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    float f[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(S + (srow + rr) * pitch + scol - 8 + 4 * q);
      f[4 * q + 0] = v.x;
      f[4 * q + 1] = v.y;
      f[4 * q + 2] = v.z;
      f[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float c = f[8 + j];
      const float c2 = c + c;
      float acc = L[rr][j];
#pragma unroll
      for (int m = 1; m <= R; ++m) acc = fmaf(w[m], pair_term<DIFF>(f[8 + j + m], f[8 + j - m], c, c2), acc);
      L[rr][j] = acc;
    }
  }
}

// ------------------------------------------------ packed FP32x2 arithmetic
// Blackwell issues two FP32 lanes per instruction (FADD2 / FFMA2 / FMUL2);
// each lane rounds exactly as the scalar instruction does.  A pair term in
// this form, fma(c, -2, a + b), equals (a + b) - 2c rounded once, i.e. the
// scalar pair form bit for bit.
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Pair-form Laplacian of a 2 (rows) x 4 (cols) block as four packed pairs,
// L[rr][p] = cells (2p, 2p+1) of row rr; same operand order as lap_2x4<R,
// false, false> (y taps, then x taps), so the results agree bit for bit.
template <int R>
__device__ __forceinline__ void lap_2x4_x2(const float* __restrict__ S, int pitch, int srow, int scol,
                                           const float2 (&w2)[R + 1], float2 L[2][2]) {
  const float2 m2 = dup2(-2.f);
  float4 col[2 + 2 * R];
#pragma unroll
  for (int i = 0; i < 2 + 2 * R; ++i) col[i] = *reinterpret_cast<const float4*>(S + (srow - R + i) * pitch + scol);
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 c = p ? hi2(col[rr + R]) : lo2(col[rr + R]);
      float2 acc = dup2(0.f);
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 a = p ? hi2(col[rr + R + m]) : lo2(col[rr + R + m]);
        const float2 b = p ? hi2(col[rr + R - m]) : lo2(col[rr + R - m]);
        acc = __ffma2_rn(w2[m], __ffma2_rn(c, m2, __fadd2_rn(a, b)), acc);
      }
      L[rr][p] = acc;
    }
  }
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    float f[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(S + (srow + rr) * pitch + scol - 8 + 4 * q);
      f[4 * q + 0] = v.x;
      f[4 * q + 1] = v.y;
      f[4 * q + 2] = v.z;
      f[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 c = make_float2(f[8 + 2 * p], f[9 + 2 * p]);
      float2 acc = L[rr][p];
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 a = make_float2(f[8 + 2 * p + m], f[9 + 2 * p + m]);
        const float2 b = make_float2(f[8 + 2 * p - m], f[9 + 2 * p - m]);
        acc = __ffma2_rn(w2[m], __ffma2_rn(c, m2, __fadd2_rn(a, b)), acc);
      }
      L[rr][p] = acc;
    }
  }
}

// Packed pair term: (a + b) - 2c as fma(c, -2, a + b), or the difference form
// (a - c) + (b - c) with -c formed exactly; either equals its scalar form bit
// for bit in each lane.
template <bool DIFF>
__device__ __forceinline__ float2 pair_term2(float2 a, float2 b, float2 c, float2 nc) {
  return DIFF ? __fadd2_rn(__fadd2_rn(a, nc), __fadd2_rn(b, nc)) : __ffma2_rn(c, dup2(-2.f), __fadd2_rn(a, b));
}

// lap_2x4<R, DIFF, ACC> in packed FP32x2 arithmetic: same operand order and
// rounding (y taps, then x taps), L[rr][j] as scalars for the callers.
template <int R, bool DIFF = false, bool ACC = false>
__device__ __forceinline__ void lap_2x4_p(const float* __restrict__ S, int pitch, int srow, int scol,
                                          const float2 (&w2)[R + 1], float L[2][4]) {
  float4 col[2 + 2 * R];
#pragma unroll
  for (int i = 0; i < 2 + 2 * R; ++i) col[i] = *reinterpret_cast<const float4*>(S + (srow - R + i) * pitch + scol);
  float2 A[2][2];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 c = p ? hi2(col[rr + R]) : lo2(col[rr + R]);
      const float2 nc = __fmul2_rn(c, dup2(-1.f));
      float2 acc = ACC ? make_float2(L[rr][2 * p], L[rr][2 * p + 1]) : dup2(0.f);
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 a = p ? hi2(col[rr + R + m]) : lo2(col[rr + R + m]);
        const float2 b = p ? hi2(col[rr + R - m]) : lo2(col[rr + R - m]);
        acc = __ffma2_rn(w2[m], pair_term2<DIFF>(a, b, c, nc), acc);
      }
      A[rr][p] = acc;
    }
  }
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    float f[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(S + (srow + rr) * pitch + scol - 8 + 4 * q);
      f[4 * q + 0] = v.x;
      f[4 * q + 1] = v.y;
      f[4 * q + 2] = v.z;
      f[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 c = make_float2(f[8 + 2 * p], f[9 + 2 * p]);
      const float2 nc = __fmul2_rn(c, dup2(-1.f));
      float2 acc = A[rr][p];
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 a = make_float2(f[8 + 2 * p + m], f[9 + 2 * p + m]);
        const float2 b = make_float2(f[8 + 2 * p - m], f[9 + 2 * p - m]);
        acc = __ffma2_rn(w2[m], pair_term2<DIFF>(a, b, c, nc), acc);
      }
      L[rr][2 * p] = acc.x;
      L[rr][2 * p + 1] = acc.y;
    }
  }
}

// 16-byte load of data read once per launch (streamed: no L1 allocation)
__device__ __forceinline__ float4 ld_stream4(const float* p) {
  float4 v;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Knuth's TwoSum: returns s = fl(a + b) and sets e so that s + e == a + b
// exactly (no reassociation: the library is built without fast-math).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
  return s;
}

// ---------------------------------------------------------------- memory ops
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_gpu_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace pat
