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

// Laplacian of the 4 x RUN cells a thread owns in a box (pitch BW floats, R halo rows above the tile,
// the thread's columns at XH + c0): lo[rr][j] for row r0 + rr.  For the low part of a compensated
// pair (a field of the order of the rounding error of its high part), so it takes the cheapest form,
// sum_m w_m (a + b) - w_c c with the centre weight w_c = 4 sum_m w_m summed in FP32 (R additions and
// a multiply, so up to R + 1 roundings): 2 FP operations per tap; the rounded w_c departs from a
// zero-sum stencil by a relative ~R 2^-24 of a field that is itself ~2^-24 of the state.
template <int R, int RUN, int BW, int XH>
__device__ __forceinline__ void stencil_run(const float* __restrict__ box, int r0, int c0,
                                            const float* __restrict__ w, float (&lo)[RUN][4]) {
  float wc = 0.f;
#pragma unroll
  for (int m = 1; m <= R; ++m) wc += w[m];
  wc *= 4.f;
  float4 win[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) win[i] = *reinterpret_cast<const float4*>(box + (r0 + i) * BW + XH + c0);
#pragma unroll
  for (int rr = 0; rr < RUN; ++rr) {
    win[2 * R] = *reinterpret_cast<const float4*>(box + (r0 + rr + 2 * R) * BW + XH + c0);
    float f[20];
    load_row20(box + (r0 + rr + R) * BW + c0 + XH - 8, f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc = -wc * f[8 + j];
#pragma unroll
      for (int m = 1; m <= R; ++m) acc = fmaf(w[m], f4get(win[R + m], j) + f4get(win[R - m], j), acc);
#pragma unroll
      for (int m = 1; m <= R; ++m) acc = fmaf(w[m], f[8 + j + m] + f[8 + j - m], acc);
      lo[rr][j] = acc;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) win[i] = win[i + 1];
  }
}

}  // namespace pat
