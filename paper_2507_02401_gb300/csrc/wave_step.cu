// One-launch-per-time-step wave kernels: the general path for 3D grids and for
// 2D grids too large to keep on chip (HBM-streaming regime).
//
// Recurrence (paper Sec. 2, Eq. wave_equation; staggered leapfrog of order 2M
// with the velocity eliminated, pressure zero outside the grid):
//
//   forward  P^1 = P^0 + 1/2 kappa L P^0,  P^{n+1} = 2 P^n - P^{n-1} + kappa L P^n
//   adjoint  Q^n = S^T r_n + 2 Q^{n+1} - Q^{n+2} + L(kappa Q^{n+1}),
//            x = S^T r_0 + Q^1 - Q^2 + 1/2 L(kappa Q^1)
//
// 2D kernels step the increment form (D^{n+1} = D^n + kappa L P^n,
// P^{n+1} = P^n + D^{n+1}; adjoint G/Q likewise): 16 B (20 B with a varying
// medium) per point-update, but FP32 rounding is not amplified in the smooth
// modes, which keeps thousands of steps within 1e-5 of FP64.  The 3D kernel
// steps the three-level form, next = c_cur cur - c_prev prev + c_lap kappa L
// cur: 12 B (16 B) per point-update for the HBM-bound volumes, whose step
// counts stay in the hundreds.  Halo re-reads hit L2/shared memory.  Sensor
// sampling of `cur` is fused into the same launch.
#include "internal.h"
#include "stencil.cuh"

namespace pat {
namespace {

// ----------------------------------------------------------------- sampling
__device__ __forceinline__ void fused_sample(const StepArgs& a, long long gtid) {
  if (a.y == nullptr || gtid >= a.ns) return;
  const int s = (int)gtid;
  float v = 0.f;
  for (int k = 0; k < a.corners; ++k) v = fmaf(a.sens_w[s * a.corners + k], a.cur[a.sens_cell[s * a.corners + k]], v);
  a.y[(long long)s * a.nt + a.t_sample] = v;
}

// ---------------------------------------------------------------- 2D, tiled
constexpr int S2_TX = 64, S2_TY = 32, S2_THREADS = 256, S2_XOFF = 8, S2_PITCH = S2_TX + 16;

template <int R, bool ADJ, bool VARC>
__global__ void __launch_bounds__(S2_THREADS) step2d_kernel(const StepArgs a) {
  constexpr int NF = ADJ ? 2 : 1;  // forward: P ; adjoint: kappa*Q as hi + lo
  constexpr int SB = (S2_TY + 2 * R) * S2_PITCH;
  __shared__ __align__(16) float S[NF * SB];
  const int t = threadIdx.x;
  const long long bid = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  fused_sample(a, bid * S2_THREADS + t);

  const int nx = a.nx, ny = a.ny;
  const int gx0 = blockIdx.x * S2_TX, gy0 = blockIdx.y * S2_TY;
  // stage the stencil input with its halo: P, or kappa (Q + Ql) split as hi + lo
  auto stage = [&](int gx, int gy, int sidx) {
    float hi = 0.f, lo = 0.f;
    if (gx >= 0 && gy >= 0 && gx < nx && gy < ny) {
      const long long gi = (long long)gy * nx + gx;
      const float q = a.cur[gi];
      if (ADJ) {
        const float k = VARC ? a.kappa[gi] : a.kappa0;
        const float kl = VARC ? a.kappa_lo[gi] : a.kappa0_lo;
        const float ql = a.cur_lo[gi];
        hi = k * q;
        lo = fmaf(k, q, -hi) + fmaf(k, ql, kl * q);
      } else {
        hi = q;
      }
    }
    S[sidx] = hi;
    if (ADJ) S[SB + sidx] = lo;
  };
  // interior + north/south halo rows (full tile width)
  for (int i = t; i < (S2_TY + 2 * R) * S2_TX; i += S2_THREADS) {
    const int row = i / S2_TX, col = i % S2_TX;
    stage(gx0 + col, gy0 + row - R, row * S2_PITCH + S2_XOFF + col);
  }
  // west/east halo columns
  for (int i = t; i < S2_TY * 2 * R; i += S2_THREADS) {
    const int row = i / (2 * R), j = i % (2 * R);
    const int col = j < R ? -R + j : S2_TX + (j - R);
    stage(gx0 + col, gy0 + row, (row + R) * S2_PITCH + S2_XOFF + col);
  }
  __syncthreads();

  const int c0 = (t % (S2_TX / 4)) * 4, r0 = (t / (S2_TX / 4)) * 2;
  float L[2][4];
  lap_2x4<R, true, false>(S, S2_PITCH, r0 + R, S2_XOFF + c0, a.w, L);
  if (ADJ) lap_2x4<R, false, true>(S + SB, S2_PITCH, r0 + R, S2_XOFF + c0, a.w, L);
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gx = gx0 + c0 + j, gy = gy0 + r0 + rr;
      if (gx >= nx || gy >= ny) continue;
      const long long gi = (long long)gy * nx + gx;
      // absorbing layer: factors a, b of the damped update (1 outside the layer)
      const float fa = a.sp_a ? a.sp_a[gi] : 1.f, fb = a.sp_a ? a.sp_b[gi] : 1.f;
      const bool layer = fa != 1.f || fb != 1.f;
      if (ADJ) {
        const float g0 = a.dbuf[gi], gl0 = a.dbuf_lo[gi];
        if (a.final_step) {  // x = S^T r_0 (already in G) + G + 1/2 L(kappa Q^1) [+ ((a-1)/b) Q^1]
          float xv = fmaf(a.c_lap, L[rr][j], g0 + gl0);
          if (layer) xv = fmaf((fa - 1.f) / fb, a.cur[gi] + a.cur_lo[gi], xv);
          a.next[gi] = xv;
          continue;
        }
        float e;
        const float g = two_sum(g0, L[rr][j] + gl0, e);  // G += L(kappa Q)  (compensated)
        a.dbuf[gi] = g;
        a.dbuf_lo[gi] = e;
        if (layer) {  // Q^n = a Q^{n+1} + b G (inside the damping layer, compensation carried approximately)
          a.next[gi] = fmaf(fa, a.cur[gi], fb * g);
          a.next_lo[gi] = fmaf(fa, a.cur_lo[gi], fb * e);
        } else {
          const float q = two_sum(a.cur[gi], g, e);  // Q^n = Q^{n+1} + G  (compensated)
          a.next[gi] = q;
          a.next_lo[gi] = a.cur_lo[gi] + e;
        }
      } else {
        const float kap = VARC ? a.kappa[gi] : a.kappa0;
        const float kap_lo = VARC ? a.kappa_lo[gi] : a.kappa0_lo;
        const float cur = S[(r0 + rr + R) * S2_PITCH + S2_XOFF + c0 + j];
        // (kappa_hi + kappa_lo) L rounded once, before it meets the much larger increment
        const float inc = fmaf(a.c_lap * kap, L[rr][j], (a.c_lap * kap_lo) * L[rr][j]);
        float d = (a.d_zero ? 0.f : a.dbuf[gi]) + inc;
        if (layer) d = a.d_zero ? fmaf(fa - 1.f, cur, fb * inc) : fmaf(fa, a.dbuf[gi], fb * inc);
        a.dbuf[gi] = d;
        a.next[gi] = cur + d;
      }
    }
}

// --------------------------------------------------------- 3D, z-marching
// CTA: 32 (x) x 16 (y) columns, each thread a row segment of 4 cells in x,
// marching over a chunk of z planes with a register queue of 2R+1 planes for
// the z-direction; the x/y neighbours of the current plane come from shared
// memory.
constexpr int S3_TX = 32, S3_TY = 16, S3_THREADS = (S3_TX / 4) * S3_TY, S3_XP = 8, S3_PITCH = S3_TX + 2 * S3_XP;
constexpr int S3_ZCHUNK = 32;

template <int R, bool ADJ, bool VARC>
__global__ void __launch_bounds__(S3_THREADS) step3d_kernel(const StepArgs a) {
  __shared__ __align__(16) float S[(S3_TY + 2 * R) * S3_PITCH];
  const int t = threadIdx.x;
  const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  fused_sample(a, bid * S3_THREADS + t);

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  const int tx = t % (S3_TX / 4), ty = t / (S3_TX / 4);
  const int gx0 = blockIdx.x * S3_TX, gy0 = blockIdx.y * S3_TY;
  const int gx = gx0 + tx * 4, gy = gy0 + ty;
  const int z0 = blockIdx.z * S3_ZCHUNK;
  const int z1 = min(z0 + S3_ZCHUNK, nz);
  const bool row_ok = gy < ny;

  auto load_own = [&](int z, float v[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int x = gx + j;
      float val = 0.f;
      if (row_ok && x < nx && z >= 0 && z < nz) {
        const long long gi = (long long)z * plane + (long long)gy * nx + x;
        val = a.cur[gi];
        if (ADJ && VARC) val *= a.kappa[gi];
      }
      v[j] = val;
    }
  };
  auto fetch = [&](int x, int y, int z) -> float {
    if (x < 0 || y < 0 || x >= nx || y >= ny) return 0.f;
    const long long gi = (long long)z * plane + (long long)y * nx + x;
    float v = a.cur[gi];
    if (ADJ && VARC) v *= a.kappa[gi];
    return v;
  };

  float q[2 * R + 1][4];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) load_own(z0 - R + i, q[i]);

  for (int z = z0; z < z1; ++z) {
    load_own(z + R, q[2 * R]);
    __syncthreads();  // previous plane's readers are done
    *reinterpret_cast<float4*>(S + (ty + R) * S3_PITCH + S3_XP + tx * 4) = make_float4(q[R][0], q[R][1], q[R][2], q[R][3]);
    for (int i = t; i < 2 * R * S3_TX; i += S3_THREADS) {  // north/south halo rows
      const int r = i / S3_TX, col = i % S3_TX;
      const int row = r < R ? r : S3_TY + R + (r - R);
      S[row * S3_PITCH + S3_XP + col] = fetch(gx0 + col, gy0 + row - R, z);
    }
    for (int i = t; i < S3_TY * 2 * R; i += S3_THREADS) {  // west/east halo columns
      const int row = i / (2 * R), j = i % (2 * R);
      const int col = j < R ? -R + j : S3_TX + (j - R);
      S[(row + R) * S3_PITCH + S3_XP + col] = fetch(gx0 + col, gy0 + row, z);
    }
    __syncthreads();

    float L[4];
    {
      const float* rowp = S + (ty + R) * S3_PITCH + S3_XP + tx * 4;
      float f[20];
#pragma unroll
      for (int qq = 0; qq < 5; ++qq) {
        const float4 v = *reinterpret_cast<const float4*>(rowp - 8 + 4 * qq);
        f[4 * qq] = v.x;
        f[4 * qq + 1] = v.y;
        f[4 * qq + 2] = v.z;
        f[4 * qq + 3] = v.w;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float c = q[R][j];
        const float c2 = c + c;
        float acc = 0.f;
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          acc = fmaf(a.w[m], (f[8 + j + m] + f[8 + j - m]) - c2, acc);
          const float4 up = *reinterpret_cast<const float4*>(rowp + m * S3_PITCH);
          const float4 dn = *reinterpret_cast<const float4*>(rowp - m * S3_PITCH);
          acc = fmaf(a.w[m], (f4get(up, j) + f4get(dn, j)) - c2, acc);
          acc = fmaf(a.w[m], (q[R + m][j] + q[R - m][j]) - c2, acc);
        }
        L[j] = acc;
      }
    }
    if (row_ok) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = gx + j;
        if (x >= nx) continue;
        const long long gi = (long long)z * plane + (long long)gy * nx + x;
        const float cur = (ADJ && VARC) ? a.cur[gi] : q[R][j];
        // kappa as hi + lo (a coherent rounding of a constant kappa would drift the phase)
        const float kap = ADJ ? (VARC ? 1.f : a.kappa0) : (VARC ? a.kappa[gi] : a.kappa0);
        const float kap_lo = ADJ ? (VARC ? 0.f : a.kappa0_lo) : (VARC ? a.kappa_lo[gi] : a.kappa0_lo);
        float v = a.c_cur * cur;
        if (a.prev) v -= a.c_prev * a.prev[gi];
        v += fmaf(a.c_lap * kap, L[j], (a.c_lap * kap_lo) * L[j]);
        a.next[gi] = v;
      }
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) q[i][j] = q[i + 1][j];
  }
}

// ------------------------------------------------------------- small kernels
__global__ void sample_kernel(const float* __restrict__ P, int ns, int nt, int tsamp, const int* __restrict__ cell,
                              const float* __restrict__ w, int corners, float* __restrict__ y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  float v = 0.f;
  for (int k = 0; k < corners; ++k) v = fmaf(w[s * corners + k], P[cell[s * corners + k]], v);
  y[(long long)s * nt + tsamp] = v;
}

// Q[cell] += scale * sum_e w_e r[sensor_e, t] over each injected cell's entries
__global__ void inject_kernel(float* __restrict__ Q, int n_inj, const int* __restrict__ inj_cell,
                              const int* __restrict__ inj_ptr, const int* __restrict__ ent_sensor,
                              const float* __restrict__ ent_w, const float* __restrict__ r, int nt, int tt,
                              float scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inj) return;
  float s = 0.f;
  for (int e = inj_ptr[i]; e < inj_ptr[i + 1]; ++e) s = fmaf(ent_w[e], r[(long long)ent_sensor[e] * nt + tt], s);
  Q[inj_cell[i]] += scale * s;
}

__global__ void fill_kernel(float* p, long long n, float v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void copy_kernel(float* __restrict__ d, const float* __restrict__ s, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = s[i];
}

template <bool ADJ, bool VARC>
cudaError_t launch2d_r(int R, const StepArgs& a, dim3 grid, cudaStream_t st) {
  switch (R) {
    case 1: step2d_kernel<1, ADJ, VARC><<<grid, S2_THREADS, 0, st>>>(a); break;
    case 3: step2d_kernel<3, ADJ, VARC><<<grid, S2_THREADS, 0, st>>>(a); break;
    case 5: step2d_kernel<5, ADJ, VARC><<<grid, S2_THREADS, 0, st>>>(a); break;
    case 7: step2d_kernel<7, ADJ, VARC><<<grid, S2_THREADS, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool ADJ, bool VARC>
cudaError_t launch3d_r(int R, const StepArgs& a, dim3 grid, cudaStream_t st) {
  switch (R) {
    case 1: step3d_kernel<1, ADJ, VARC><<<grid, S3_THREADS, 0, st>>>(a); break;
    case 3: step3d_kernel<3, ADJ, VARC><<<grid, S3_THREADS, 0, st>>>(a); break;
    case 5: step3d_kernel<5, ADJ, VARC><<<grid, S3_THREADS, 0, st>>>(a); break;
    case 7: step3d_kernel<7, ADJ, VARC><<<grid, S3_THREADS, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t step2d_launch(int R, bool adj, const StepArgs& a, cudaStream_t st) {
  dim3 grid((a.nx + S2_TX - 1) / S2_TX, (a.ny + S2_TY - 1) / S2_TY);
  // enough threads for the fused sampling
  const long long nthreads = (long long)grid.x * grid.y * S2_THREADS;
  if (a.y && a.ns > nthreads) return cudaErrorInvalidValue;
  const bool varc = a.kappa != nullptr;
  if (adj) return varc ? launch2d_r<true, true>(R, a, grid, st) : launch2d_r<true, false>(R, a, grid, st);
  return varc ? launch2d_r<false, true>(R, a, grid, st) : launch2d_r<false, false>(R, a, grid, st);
}

cudaError_t step3d_launch(int R, bool adj, const StepArgs& a, cudaStream_t st) {
  dim3 grid((a.nx + S3_TX - 1) / S3_TX, (a.ny + S3_TY - 1) / S3_TY, (a.nz + S3_ZCHUNK - 1) / S3_ZCHUNK);
  const long long nthreads = (long long)grid.x * grid.y * grid.z * S3_THREADS;
  if (a.y && a.ns > nthreads) return cudaErrorInvalidValue;
  const bool varc = a.kappa != nullptr;
  if (adj) return varc ? launch3d_r<true, true>(R, a, grid, st) : launch3d_r<true, false>(R, a, grid, st);
  return varc ? launch3d_r<false, true>(R, a, grid, st) : launch3d_r<false, false>(R, a, grid, st);
}

cudaError_t sample_launch(const float* P, int ns, int nt, int t, const int* cell, const float* w, int corners,
                          float* y, cudaStream_t st) {
  if (ns <= 0) return cudaSuccess;
  sample_kernel<<<(ns + 127) / 128, 128, 0, st>>>(P, ns, nt, t, cell, w, corners, y);
  return cudaGetLastError();
}

cudaError_t inject_launch(float* Q, int n_inj, const int* inj_cell, const int* inj_ptr, const int* ent_sensor,
                          const float* ent_w, const float* r, int nt, int t, float scale, cudaStream_t st) {
  if (n_inj <= 0) return cudaSuccess;
  inject_kernel<<<(n_inj + 127) / 128, 128, 0, st>>>(Q, n_inj, inj_cell, inj_ptr, ent_sensor, ent_w, r, nt, t, scale);
  return cudaGetLastError();
}

cudaError_t fill_launch(float* p, long long n, float v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<<<grid_for(n), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t copy_launch(float* d, const float* s, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  copy_kernel<<<grid_for(n), 256, 0, st>>>(d, s, n);
  return cudaGetLastError();
}


// ---------------------------------------------------------- medium gradient
// gacc[i] += coef * (Q[i] + Qlo[i]) * (L P)[i]: one term of
//   d<r, K x>/d kappa = sum_{n>=1} Q^{n+1} .* L P^n + 1/2 Q^1 .* L P^0,
// the explicit kappa-dependence of P^{n+1} = 2P^n - P^{n-1} + kappa .* L P^n
// weighted by the adjoint state.  L P is the zero-sum difference form with
// zero outside the grid; the sum over steps is kept in FP64.
namespace {
template <int R>
__global__ void grad_acc_kernel(double* __restrict__ gacc, const float* __restrict__ Q, const float* __restrict__ Qlo,
                                const float* __restrict__ P, float coef, int nx, int ny, int nz, int dim, int zform,
                                const StepArgs a) {
  const long long N = (long long)nx * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((long long)nx * ny));
    const float c = P[i];
    float acc = 0.f;
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      const float xp = (x + m < nx) ? P[i + m] : 0.f;
      const float xm = (x - m >= 0) ? P[i - m] : 0.f;
      const float yp = (y + m < ny) ? P[i + (long long)m * nx] : 0.f;
      const float ym = (y - m >= 0) ? P[i - (long long)m * nx] : 0.f;
      float t = ((xp - c) + (xm - c)) + ((yp - c) + (ym - c));
      if (dim == 3) {
        const long long pl = (long long)nx * ny;
        const float zp = (z + m < nz) ? P[i + m * pl] : 0.f;
        const float zm = (z - m >= 0) ? P[i - m * pl] : 0.f;
        t += (zp - c) + (zm - c);
      }
      acc = fmaf(a.w[m], t, acc);
    }
    double q = (double)Q[i] + (Qlo ? (double)Qlo[i] : 0.0);
    if (zform)  // the state holds Z = kappa Q
      q /= a.kappa ? (double)a.kappa[i] + (double)a.kappa_lo[i] : (double)a.kappa0 + (double)a.kappa0_lo;
    gacc[i] += (double)coef * q * (double)acc;
  }
}

__global__ void d2f_kernel(float* __restrict__ out, const double* __restrict__ in, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void dfill_kernel(double* __restrict__ p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.0;
}
}  // namespace

cudaError_t grad_acc_launch(int R, double* gacc, const float* Q, const float* Qlo, const float* P, float coef,
                            const StepArgs& a, int dim, bool zform, cudaStream_t st) {
  const long long N = (long long)a.nx * a.ny * a.nz;
  const int blocks = grid_for(N);
  switch (R) {
    case 1: grad_acc_kernel<1><<<blocks, 256, 0, st>>>(gacc, Q, Qlo, P, coef, a.nx, a.ny, a.nz, dim, zform, a); break;
    case 3: grad_acc_kernel<3><<<blocks, 256, 0, st>>>(gacc, Q, Qlo, P, coef, a.nx, a.ny, a.nz, dim, zform, a); break;
    case 5: grad_acc_kernel<5><<<blocks, 256, 0, st>>>(gacc, Q, Qlo, P, coef, a.nx, a.ny, a.nz, dim, zform, a); break;
    case 7: grad_acc_kernel<7><<<blocks, 256, 0, st>>>(gacc, Q, Qlo, P, coef, a.nx, a.ny, a.nz, dim, zform, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t d2f_launch(float* out, const double* in, long long n, cudaStream_t st) {
  d2f_kernel<<<grid_for(n), 256, 0, st>>>(out, in, n);
  return cudaGetLastError();
}

cudaError_t dfill_launch(double* p, long long n, cudaStream_t st) {
  dfill_kernel<<<grid_for(n), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

}  // namespace pat
