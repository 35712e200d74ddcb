// Row helpers of the 2D tile kernels (TMA per-step and batched): a thread owns
// 4 columns of a shared-memory box row (80 floats: 8 halo columns each side of
// a 64-column tile) and slides a register window of 2R+1 rows down its run.
#pragma once

#include "stencil.cuh"

namespace pat {

// 20 floats of a box row starting 8 columns left of the thread's first column
__device__ __forceinline__ void load_row20(const float* __restrict__ row, float (&f)[20]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const float4 v = *reinterpret_cast<const float4*>(row + 4 * q);
    f[4 * q + 0] = v.x;
    f[4 * q + 1] = v.y;
    f[4 * q + 2] = v.z;
    f[4 * q + 3] = v.w;
  }
}

// Zero-sum Laplacian of column j (0..3) of the thread's row: sum over the x and y taps
// w_m [(a + b) - 2c] (pair form, 3 FP operations per tap) or w_m [(a - c) + (b - c)]
// (difference form, rounding relative to the differences: for fields with a large smooth part).
// `win` holds box rows row-R .. row+R of the thread's 4 columns, `f` the row itself (load_row20).
template <int R, bool DIFF>
__device__ __forceinline__ float stencil_cell(const float4 (&win)[2 * R + 1], const float (&f)[20], int j,
                                              const float* __restrict__ w) {
  const float c = f[8 + j];
  const float c2 = c + c;
  float acc = 0.f;
#pragma unroll
  for (int m = 1; m <= R; ++m) acc = fmaf(w[m], pair_term<DIFF>(f4get(win[R + m], j), f4get(win[R - m], j), c, c2), acc);
#pragma unroll
  for (int m = 1; m <= R; ++m) acc = fmaf(w[m], pair_term<DIFF>(f[8 + j + m], f[8 + j - m], c, c2), acc);
  return acc;
}

// stencil_cell for all four columns in packed FP32x2 arithmetic (pairs of columns 0-1, 2-3); each
// lane takes the scalar function's operations in the same order, so acc[j] equals stencil_cell(.., j, ..).
template <int R, bool DIFF>
__device__ __forceinline__ void stencil_cells2(const float4 (&win)[2 * R + 1], const float (&f)[20],
                                               const float2 (&w2)[R + 1], float (&acc)[4]) {
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 c = make_float2(f[8 + 2 * p], f[9 + 2 * p]);
    const float2 nc = __fmul2_rn(c, dup2(-1.f));
    float2 a2 = dup2(0.f);
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      const float2 up = p ? hi2(win[R + m]) : lo2(win[R + m]);
      const float2 dn = p ? hi2(win[R - m]) : lo2(win[R - m]);
      a2 = __ffma2_rn(w2[m], pair_term2<DIFF>(up, dn, c, nc), a2);
    }
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      const float2 rt = make_float2(f[8 + 2 * p + m], f[9 + 2 * p + m]);
      const float2 lt = make_float2(f[8 + 2 * p - m], f[9 + 2 * p - m]);
      a2 = __ffma2_rn(w2[m], pair_term2<DIFF>(rt, lt, c, nc), a2);
    }
    acc[2 * p] = a2.x;
    acc[2 * p + 1] = a2.y;
  }
}

// Laplacian of the 4 x RUN cells a thread owns in a box (pitch BW floats, R halo rows above the tile,
// the thread's columns at XH + c0): lo[rr][j] for row r0 + rr.  For the low part of a compensated
// pair (a field of the order of the rounding error of its high part), so it takes the cheapest form,
// sum_m w_m (a + b) - w_c c with the centre weight w_c = 4 sum_m w_m summed in FP32 (R additions and
// a multiply, so up to R + 1 roundings): 2 FP operations per tap; the rounded w_c departs from a
// zero-sum stencil by a relative ~R 2^-24 of a field that is itself ~2^-24 of the state.
// (Packed FP32x2 arithmetic, pairs of columns 0-1 and 2-3, each lane in the scalar operation order.)
template <int R, int RUN, int BW, int XH>
__device__ __forceinline__ void stencil_run(const float* __restrict__ box, int r0, int c0,
                                            const float* __restrict__ w, float (&lo)[RUN][4]) {
  float wc = 0.f;
#pragma unroll
  for (int m = 1; m <= R; ++m) wc += w[m];
  wc *= 4.f;
  const float2 nwc = dup2(-wc);
  float2 w2[R + 1];
#pragma unroll
  for (int m = 0; m <= R; ++m) w2[m] = dup2(w[m]);
  float4 win[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) win[i] = *reinterpret_cast<const float4*>(box + (r0 + i) * BW + XH + c0);
#pragma unroll
  for (int rr = 0; rr < RUN; ++rr) {
    win[2 * R] = *reinterpret_cast<const float4*>(box + (r0 + rr + 2 * R) * BW + XH + c0);
    float f[20];
    load_row20(box + (r0 + rr + R) * BW + c0 + XH - 8, f);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float2 acc = __fmul2_rn(nwc, make_float2(f[8 + 2 * p], f[9 + 2 * p]));
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 up = p ? hi2(win[R + m]) : lo2(win[R + m]);
        const float2 dn = p ? hi2(win[R - m]) : lo2(win[R - m]);
        acc = __ffma2_rn(w2[m], __fadd2_rn(up, dn), acc);
      }
#pragma unroll
      for (int m = 1; m <= R; ++m)
        acc = __ffma2_rn(w2[m],
                         __fadd2_rn(make_float2(f[8 + 2 * p + m], f[9 + 2 * p + m]),
                                    make_float2(f[8 + 2 * p - m], f[9 + 2 * p - m])),
                         acc);
      lo[rr][2 * p] = acc.x;
      lo[rr][2 * p + 1] = acc.y;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) win[i] = win[i + 1];
  }
}

}  // namespace pat
