// Fourier form of the prior (paper Sec. 4, implementation: the adjoint
// embedding acts as multiplication by the Bessel potential
// (1 + 4 pi^2 |xi|^2)^{-s} in the Fourier domain, E_s* X = ifft(B fft(X))).
// In the coefficient formulation of this library the paper's operator is the
// covariance E_s E_s*, so the prior's E_s is the real, even filter with the
// square root of the potential; E_s* = E_s.  Lengths are in units of
// `length_cells` cells: DFT index k of an n-cell axis is xi = k' length_cells / n
// with k' = k for k < n/2 and k - n otherwise.
//
// 2D, power-of-two extents up to 4096.  One application:
//   x-direction FFT of every row (one CTA per row, radix-2 in shared memory),
//   transpose, y-direction FFT of every column + filter + inverse FFT (fused,
//   one CTA per column), transpose back, inverse x-direction FFT keeping the
//   real part.  Twiddle factors are tabulated in FP64 on the host and rounded.
#include <cmath>
#include <vector>

#include "plan.h"

namespace pat {
namespace {

constexpr int FT = 256;  // threads of the row kernels

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ unsigned bitrev(unsigned i, int logn) { return __brev(i) >> (32 - logn); }

// in-place decimation in time on bit-reversed input -> natural order (forward: w = tw, inverse: conj)
__device__ void fft_dit(float2* s, int n, int logn, const float2* __restrict__ tw, bool inverse) {
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1, stride = n / len;
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int grp = t / half, pos = t - grp * half;
      const int i = grp * len + pos, j = i + half;
      float2 w = tw[pos * stride];
      if (inverse) w.y = -w.y;
      const float2 u = s[i], v = cmul(s[j], w);
      s[i] = make_float2(u.x + v.x, u.y + v.y);
      s[j] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

// in-place decimation in frequency on natural input -> bit-reversed order
__device__ void fft_dif(float2* s, int n, int logn, const float2* __restrict__ tw, bool inverse) {
  for (int len = n; len >= 2; len >>= 1) {
    const int half = len >> 1, stride = n / len;
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
      const int grp = t / half, pos = t - grp * half;
      const int i = grp * len + pos, j = i + half;
      float2 w = tw[pos * stride];
      if (inverse) w.y = -w.y;
      const float2 u = s[i], v = s[j];
      s[i] = make_float2(u.x + v.x, u.y + v.y);
      s[j] = cmul(make_float2(u.x - v.x, u.y - v.y), w);
    }
    __syncthreads();
  }
}

// forward FFT of every row of a real nx x ny field -> complex rows (natural order)
__global__ void __launch_bounds__(FT) fft_rows_fwd_kernel(const float* __restrict__ in, float2* __restrict__ out,
                                                           int n, int logn, const float2* __restrict__ tw) {
  extern __shared__ float2 s[];
  const long long row = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += FT) s[bitrev(i, logn)] = make_float2(in[row * n + i], 0.f);
  __syncthreads();
  fft_dit(s, n, logn, tw, false);
  for (int i = threadIdx.x; i < n; i += FT) out[row * n + i] = s[i];
}

// inverse FFT of every complex row; keeps the real part times `scale`
__global__ void __launch_bounds__(FT) fft_rows_inv_kernel(const float2* __restrict__ in, float* __restrict__ out,
                                                           int n, int logn, const float2* __restrict__ tw, float scale) {
  extern __shared__ float2 s[];
  const long long row = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += FT) s[i] = in[row * n + i];
  __syncthreads();
  fft_dif(s, n, logn, tw, true);
  for (int i = threadIdx.x; i < n; i += FT) out[row * n + bitrev(i, logn)] = s[i].x * scale;
}

// one column (a row of the transposed spectrum, fixed x frequency kx = blockIdx.x): forward FFT along y,
// multiplication by (1 + 4 pi^2 |xi|^2)^{-s/2}, inverse FFT along y
__global__ void __launch_bounds__(FT) fft_cols_filter_kernel(float2* __restrict__ data, int n, int logn, int nx,
                                                              const float2* __restrict__ tw, float ex, float lc) {
  extern __shared__ float2 s[];
  const long long row = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += FT) s[bitrev(i, logn)] = data[row * n + i];
  __syncthreads();
  fft_dit(s, n, logn, tw, false);
  const int kx = (int)row < nx / 2 ? (int)row : (int)row - nx;
  const float xix = (float)kx * lc / (float)nx;
  const float fourpi2 = 39.47841760435743f;  // 4 pi^2
  for (int i = threadIdx.x; i < n; i += FT) {
    const int ky = i < n / 2 ? i : i - n;
    const float xiy = (float)ky * lc / (float)n;
    const float m = powf(1.f + fourpi2 * (xix * xix + xiy * xiy), ex);
    s[i] = make_float2(s[i].x * m, s[i].y * m);
  }
  __syncthreads();
  fft_dif(s, n, logn, tw, true);
  for (int i = threadIdx.x; i < n; i += FT) data[row * n + bitrev(i, logn)] = s[i];
}

// out (cols x rows) = transpose of in (rows x cols), 32 x 32 tiles
__global__ void transpose_kernel(const float2* __restrict__ in, float2* __restrict__ out, int rows, int cols) {
  __shared__ float2 t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < rows && c < cols) t[j][threadIdx.x] = in[(long long)r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = bx + j, c = by + threadIdx.x;  // out row = in column
    if (r < cols && c < rows) out[(long long)r * rows + c] = t[threadIdx.x][j];
  }
}

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

std::vector<float2> twiddles(int n) {
  std::vector<float2> t(n / 2 > 0 ? n / 2 : 1);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n / 2; ++k)
    t[k] = make_float2((float)std::cos(-2.0 * pi * k / n), (float)std::sin(-2.0 * pi * k / n));
  return t;
}

}  // namespace

bool fourier_supported(int dim, int nx, int ny) {
  auto pow2 = [](int n) { return n >= 2 && n <= 4096 && (n & (n - 1)) == 0; };
  return dim == 2 && pow2(nx) && pow2(ny);
}

pat_status fourier_setup(pat_plan* p, double length_cells, cudaStream_t st) {
  const int nx = p->n[0], ny = p->n[1];
  if (!p->d_fc) {
    PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->d_fc), sizeof(float2) * 2 * (size_t)p->N, "Fourier buffers"));
    PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->d_tw), sizeof(float2) * (size_t)(nx / 2 + ny / 2 + 2),
                       "twiddles"));
    std::vector<float2> tx = twiddles(nx), ty = twiddles(ny);
    PAT_TRY_CUDA(cudaMemcpyAsync(p->d_tw, tx.data(), sizeof(float2) * tx.size(), cudaMemcpyHostToDevice, st));
    PAT_TRY_CUDA(cudaMemcpyAsync(p->d_tw + (nx / 2 + 1), ty.data(), sizeof(float2) * ty.size(), cudaMemcpyHostToDevice,
                                 st));
    PAT_TRY_CUDA(cudaStreamSynchronize(st));
  }
  p->fourier_lc = length_cells;
  return PAT_OK;
}

// out = E_s in (= E_s* in): the Fourier-form filter with exponent -s/2
pat_status fourier_apply(pat_plan* p, double s, const float* in, float* out, cudaStream_t st) {
  const int nx = p->n[0], ny = p->n[1], lx = log2i(nx), ly = log2i(ny);
  float2* A = p->d_fc;
  float2* B = p->d_fc + p->N;
  const float2* twx = p->d_tw;
  const float2* twy = p->d_tw + (nx / 2 + 1);
  fft_rows_fwd_kernel<<<ny, FT, sizeof(float2) * nx, st>>>(in, A, nx, lx, twx);
  transpose_kernel<<<dim3((nx + 31) / 32, (ny + 31) / 32), dim3(32, 8), 0, st>>>(A, B, ny, nx);
  fft_cols_filter_kernel<<<nx, FT, sizeof(float2) * ny, st>>>(B, ny, ly, nx, twy, (float)(-0.5 * s),
                                                               (float)p->fourier_lc);
  transpose_kernel<<<dim3((ny + 31) / 32, (nx + 31) / 32), dim3(32, 8), 0, st>>>(B, A, nx, ny);
  fft_rows_inv_kernel<<<ny, FT, sizeof(float2) * nx, st>>>(A, out, nx, lx, twx, 1.f / ((float)nx * (float)ny));
  PAT_TRY_CUDA(cudaGetLastError());
  return PAT_OK;
}

}  // namespace pat
