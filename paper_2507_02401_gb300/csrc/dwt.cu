// Periodic orthonormal Daubechies DWT levels with fused level scaling
// (paper Sec. 4: the fast wavelet transform W, W^{-1} = W^T, and the diagonal
// scaling D of the detail blocks, Prop. 4.2).
//
// One analysis level along an axis of even length n with filters h, g
// (g_j = (-1)^j h_{L-1-j}):
//   a_k = sum_j h_j x[(2k+j) mod n],  d_k = sum_j g_j x[(2k+j) mod n];
// synthesis is the transpose: x[(2k+j) mod n] += h_j a_k + g_j d_k.
//
// 2D levels are fused: one CTA loads a periodic input window into shared
// memory, filters along x, then along y, and writes the four bands (details
// times the level weight).  3D levels run as separable 1D passes.
#include "internal.h"

namespace pat {
namespace {

struct Filt {
  float h[kMaxTaps];
  float g[kMaxTaps];
  int L;
};

__device__ __forceinline__ int pmod(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------- 2D analysis
constexpr int A_OX = 32, A_OY = 8, A_THREADS = 256;
constexpr int A_WX = 2 * A_OX + kMaxTaps - 2;  // input window width (70)
constexpr int A_WY = 2 * A_OY + kMaxTaps - 2;  // input window height (22)

__global__ void __launch_bounds__(A_THREADS) dwt2d_analysis_kernel(const float* __restrict__ in, int nx, int ny,
                                                                   float* __restrict__ A, float* __restrict__ Hb,
                                                                   float* __restrict__ Vb, float* __restrict__ Db,
                                                                   float wdet, const Filt f) {
  __shared__ float win[A_WY][A_WX + 1];
  __shared__ float lo[A_WY][A_OX + 1];
  __shared__ float hi[A_WY][A_OX + 1];
  const int t = threadIdx.x;
  const int nx2 = nx >> 1, ny2 = ny >> 1;
  const int kx0 = blockIdx.x * A_OX, ky0 = blockIdx.y * A_OY;
  const int L = f.L;
  const int wx = 2 * A_OX + L - 2, wy = 2 * A_OY + L - 2;
  for (int i = t; i < wy * wx; i += A_THREADS) {
    const int r = i / wx, c = i % wx;
    const int gy = pmod(2 * ky0 + r, ny), gx = pmod(2 * kx0 + c, nx);
    win[r][c] = in[(long long)gy * nx + gx];
  }
  __syncthreads();
  for (int i = t; i < wy * A_OX; i += A_THREADS) {  // along x
    const int r = i / A_OX, k = i % A_OX;
    float sl = 0.f, sh = 0.f;
    for (int j = 0; j < L; ++j) {
      const float v = win[r][2 * k + j];
      sl = fmaf(f.h[j], v, sl);
      sh = fmaf(f.g[j], v, sh);
    }
    lo[r][k] = sl;
    hi[r][k] = sh;
  }
  __syncthreads();
  for (int i = t; i < A_OY * A_OX; i += A_THREADS) {  // along y
    const int ky = i / A_OX, kx = i % A_OX;
    const int oy = ky0 + ky, ox = kx0 + kx;
    if (oy >= ny2 || ox >= nx2) continue;
    float a = 0.f, hh = 0.f, vv = 0.f, dd = 0.f;
    for (int j = 0; j < L; ++j) {
      const float l = lo[2 * ky + j][kx], h = hi[2 * ky + j][kx];
      a = fmaf(f.h[j], l, a);
      hh = fmaf(f.g[j], l, hh);  // x low, y high
      vv = fmaf(f.h[j], h, vv);  // x high, y low
      dd = fmaf(f.g[j], h, dd);
    }
    const long long o = (long long)oy * nx2 + ox;
    A[o] = a;
    Hb[o] = wdet * hh;
    Vb[o] = wdet * vv;
    Db[o] = wdet * dd;
  }
}

// --------------------------------------------------------- 2D synthesis
constexpr int S_OX = 64, S_OY = 16, S_THREADS = 256;
constexpr int S_KX = S_OX / 2 + kMaxTaps / 2;  // coefficient window width (36)
constexpr int S_KY = S_OY / 2 + kMaxTaps / 2;  // (12)

__global__ void __launch_bounds__(S_THREADS) dwt2d_synthesis_kernel(const float* __restrict__ A,
                                                                    const float* __restrict__ Hb,
                                                                    const float* __restrict__ Vb,
                                                                    const float* __restrict__ Db, float wdet, int nx,
                                                                    int ny, float* __restrict__ out, const Filt f) {
  __shared__ float ca[S_KY][S_KX + 1], ch[S_KY][S_KX + 1], cv[S_KY][S_KX + 1], cd[S_KY][S_KX + 1];
  __shared__ float lo[S_OY][S_KX + 1], hi[S_OY][S_KX + 1];
  const int t = threadIdx.x;
  const int nx2 = nx >> 1, ny2 = ny >> 1;
  const int i0 = blockIdx.y * S_OY, j0 = blockIdx.x * S_OX;  // even
  const int L = f.L;
  const int kyl = i0 / 2 - (L / 2 - 1), kxl = j0 / 2 - (L / 2 - 1);
  const int ky_n = S_OY / 2 + L / 2 - 1, kx_n = S_OX / 2 + L / 2 - 1;
  for (int i = t; i < ky_n * kx_n; i += S_THREADS) {
    const int r = i / kx_n, c = i % kx_n;
    const long long o = (long long)pmod(kyl + r, ny2) * nx2 + pmod(kxl + c, nx2);
    ca[r][c] = A[o];
    ch[r][c] = wdet * Hb[o];
    cv[r][c] = wdet * Vb[o];
    cd[r][c] = wdet * Db[o];
  }
  __syncthreads();
  // along y: rows i0 .. i0+S_OY-1, coefficient columns kxl .. kxl+kx_n-1
  for (int i = t; i < S_OY * kx_n; i += S_THREADS) {
    const int r = i / kx_n, c = i % kx_n;
    const int iy = i0 + r;
    float sl = 0.f, sh = 0.f;
    for (int j = (iy & 1); j < L; j += 2) {
      const int k = ((iy - j) >> 1) - kyl;  // (iy - j) even
      sl = fmaf(f.h[j], ca[k][c], sl);
      sl = fmaf(f.g[j], ch[k][c], sl);
      sh = fmaf(f.h[j], cv[k][c], sh);
      sh = fmaf(f.g[j], cd[k][c], sh);
    }
    lo[r][c] = sl;
    hi[r][c] = sh;
  }
  __syncthreads();
  for (int i = t; i < S_OY * S_OX; i += S_THREADS) {  // along x
    const int r = i / S_OX, c = i % S_OX;
    const int iy = i0 + r, ix = j0 + c;
    if (iy >= ny || ix >= nx) continue;
    float v = 0.f;
    for (int j = (ix & 1); j < L; j += 2) {
      const int k = ((ix - j) >> 1) - kxl;
      v = fmaf(f.h[j], lo[r][k], v);
      v = fmaf(f.g[j], hi[r][k], v);
    }
    out[(long long)iy * nx + ix] = v;
  }
}

// ------------------------------------------------- separable 1D (3D grids)
// Array extents (n0 = fastest, n1, n2).  Analysis halves extent `axis`.
__global__ void dwt1d_analysis_kernel(const float* __restrict__ in, int n0, int n1, int n2, int axis,
                                      float* __restrict__ lo, float* __restrict__ hi, float wlo, float whi,
                                      const Filt f) {
  int m[3] = {n0, n1, n2};
  m[axis] >>= 1;
  const long long total = (long long)m[0] * m[1] * m[2];
  const long long st_in[3] = {1, n0, (long long)n0 * n1};
  const int na = (axis == 0 ? n0 : (axis == 1 ? n1 : n2));
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    const int c0 = (int)(o % m[0]);
    const int c1 = (int)((o / m[0]) % m[1]);
    const int c2 = (int)(o / ((long long)m[0] * m[1]));
    int c[3] = {c0, c1, c2};
    const int k = c[axis];
    c[axis] = 0;
    const long long b = c[0] * st_in[0] + c[1] * st_in[1] + c[2] * st_in[2];
    const long long sa = st_in[axis];
    float sl = 0.f, sh = 0.f;
    for (int j = 0; j < f.L; ++j) {
      const float v = in[b + (long long)pmod(2 * k + j, na) * sa];
      sl = fmaf(f.h[j], v, sl);
      sh = fmaf(f.g[j], v, sh);
    }
    lo[o] = wlo * sl;
    hi[o] = whi * sh;
  }
}

// Synthesis doubles extent `axis` of (n0, n1, n2) (the coefficient extents).
__global__ void dwt1d_synthesis_kernel(const float* __restrict__ lo, const float* __restrict__ hi, float wlo,
                                       float whi, int n0, int n1, int n2, int axis, float* __restrict__ out,
                                       const Filt f) {
  int m[3] = {n0, n1, n2};
  m[axis] <<= 1;
  const long long total = (long long)m[0] * m[1] * m[2];
  const long long st_c[3] = {1, n0, (long long)n0 * n1};
  const int nc = (axis == 0 ? n0 : (axis == 1 ? n1 : n2));
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    const int c0 = (int)(o % m[0]);
    const int c1 = (int)((o / m[0]) % m[1]);
    const int c2 = (int)(o / ((long long)m[0] * m[1]));
    int c[3] = {c0, c1, c2};
    const int i = c[axis];
    c[axis] = 0;
    const long long b = c[0] * st_c[0] + c[1] * st_c[1] + c[2] * st_c[2];
    const long long sa = st_c[axis];
    float v = 0.f;
    for (int j = (i & 1); j < f.L; j += 2) {
      const long long idx = b + (long long)pmod((i - j) >> 1, nc) * sa;
      v = fmaf(f.h[j] * wlo, lo[idx], v);
      v = fmaf(f.g[j] * whi, hi[idx], v);
    }
    out[o] = v;
  }
}

__global__ void scale_copy_kernel(float* __restrict__ d, const float* __restrict__ s, long long n, float w) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = w * s[i];
}

Filt make_filt(const float* h, const float* g, int L) {
  Filt f{};
  for (int j = 0; j < L; ++j) {
    f.h[j] = h[j];
    f.g[j] = g[j];
  }
  f.L = L;
  return f;
}

int grid1d(long long n) {
  long long b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t dwt2d_analysis_level(const float* in, int nx, int ny, float* approx, float* bandH, float* bandV,
                                 float* bandD, float wdet, const float* h, const float* g, int L, cudaStream_t st) {
  const Filt f = make_filt(h, g, L);
  dim3 grid(((nx >> 1) + A_OX - 1) / A_OX, ((ny >> 1) + A_OY - 1) / A_OY);
  dwt2d_analysis_kernel<<<grid, A_THREADS, 0, st>>>(in, nx, ny, approx, bandH, bandV, bandD, wdet, f);
  return cudaGetLastError();
}

cudaError_t dwt2d_synthesis_level(const float* approx, const float* bandH, const float* bandV, const float* bandD,
                                  float wdet, int nx, int ny, float* out, const float* h, const float* g, int L,
                                  cudaStream_t st) {
  const Filt f = make_filt(h, g, L);
  dim3 grid((nx + S_OX - 1) / S_OX, (ny + S_OY - 1) / S_OY);
  dwt2d_synthesis_kernel<<<grid, S_THREADS, 0, st>>>(approx, bandH, bandV, bandD, wdet, nx, ny, out, f);
  return cudaGetLastError();
}

cudaError_t dwt1d_synthesis_axis(const float* lo, const float* hi, float wlo, float whi, int n0, int n1, int n2,
                                 int axis, float* out, const float* h, const float* g, int L, cudaStream_t st) {
  const Filt f = make_filt(h, g, L);
  int m[3] = {n0, n1, n2};
  m[axis] <<= 1;
  dwt1d_synthesis_kernel<<<grid1d((long long)m[0] * m[1] * m[2]), 256, 0, st>>>(lo, hi, wlo, whi, n0, n1, n2, axis,
                                                                                 out, f);
  return cudaGetLastError();
}

cudaError_t dwt1d_analysis_axis(const float* in, int n0, int n1, int n2, int axis, float* lo, float* hi, float wlo,
                                  float whi, const float* h, const float* g, int L, cudaStream_t st) {
  const Filt f = make_filt(h, g, L);
  int m[3] = {n0, n1, n2};
  m[axis] >>= 1;
  dwt1d_analysis_kernel<<<grid1d((long long)m[0] * m[1] * m[2]), 256, 0, st>>>(in, n0, n1, n2, axis, lo, hi, wlo,
                                                                                whi, f);
  return cudaGetLastError();
}

cudaError_t scale_copy_launch(float* dst, const float* src, long long n, float w, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scale_copy_kernel<<<grid1d(n), 256, 0, st>>>(dst, src, n, w);
  return cudaGetLastError();
}

}  // namespace pat
