// GMRES (the paper's solver, Sec. 4 and 5) on the image-space system
//   A x = f,  A = Gamma K* K + alpha I,  f = Gamma K* y,  Gamma = E_s E_s*,
// and the Landweber iteration u <- u - omega (H u - b) on the coefficient
// system H = E_s* K* K E_s + alpha I, b = E_s* K* y, both logging the
// objective J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 per iterate.
//
// Vectors are FP32 on the device; inner products are FP64 reductions in a
// fixed order (per-block partial sums over a fixed grid, then one block sums
// the partials in block order), so results are reproducible.  GMRES keeps its
// (iters+1) x iters Hessenberg matrix and Givens rotations on the host in
// FP64 (Arnoldi with classical Gram-Schmidt applied twice, all projections of
// a pass in one launch; the least-squares problem is reduced by Givens
// rotations as the basis grows; one host synchronisation per iteration).
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.h"

namespace pat {
namespace {

constexpr int KT = 256;  // threads per block
constexpr int KB = 296;  // blocks of the reductions (a fixed count keeps the summation order fixed)

__device__ __forceinline__ double block_reduce(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < KT / 32; ++w) s += sh[w];
  return s;
}

// partial[b] = sum over this block's grid-stride share of a_i * b_i (or (a_i - b_i)^2)
template <bool DIFF>
__global__ void __launch_bounds__(KT) dot_partial_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                         long long n, double* __restrict__ partial) {
  __shared__ double sh[KT / 32];
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)gridDim.x * KT) {
    const double x = a[i], y = b[i];
    v += DIFF ? (x - y) * (x - y) : x * y;
  }
  const double s = block_reduce(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(KT) dot_final_kernel(const double* __restrict__ partial, int nb,
                                                       double* __restrict__ out) {
  __shared__ double sh[KT / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += KT) v += partial[i];
  const double s = block_reduce(v, sh);
  if (threadIdx.x == 0) *out = s;
}

// y = y + a x
__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ x, float a, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

// x = a x
__global__ void scal_kernel(float* __restrict__ x, float a, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= a;
}

// Landweber step: u <- u - omega ((q + alpha u) - b), q = E_s* K* K E_s u
__global__ void lw_update_kernel(float* __restrict__ u, const float* __restrict__ b, const float* __restrict__ q,
                                 float omega, float alpha, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float ui = u[i];
    u[i] = fmaf(-omega, fmaf(alpha, ui, q[i]) - b[i], ui);
  }
}

// partial[i * KB + b] = block b's share of <V_i, w> for i = blockIdx.y (all basis vectors in one launch)
__global__ void __launch_bounds__(KT) mdot_partial_kernel(const float* __restrict__ V, const float* __restrict__ w,
                                                          long long n, double* __restrict__ partial) {
  __shared__ double sh[KT / 32];
  const float* v = V + (size_t)blockIdx.y * n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * KT + threadIdx.x; i < n; i += (long long)gridDim.x * KT)
    acc += (double)v[i] * (double)w[i];
  const double s = block_reduce(acc, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * KB + blockIdx.x] = s;
}

// h[i] (+)= sum of block partials of vector i (block i), in block order
__global__ void __launch_bounds__(KT) mdot_final_kernel(const double* __restrict__ partial, double* __restrict__ h,
                                                        int accumulate) {
  __shared__ double sh[KT / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < KB; b += KT) v += partial[(size_t)blockIdx.x * KB + b];
  const double s = block_reduce(v, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = accumulate ? h[blockIdx.x] + s : s;
}

// w -= sum_i c_i V_i with c the latest projection coefficients (device, FP64)
__global__ void maxpy_kernel(float* __restrict__ w, const float* __restrict__ V, const double* __restrict__ c, int k,
                             long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < k; ++i) acc -= c[i] * (double)V[(size_t)i * n + e];
    w[e] = (float)acc;
  }
}

// w /= sqrt(*nrm2) (left unchanged when the norm is zero)
__global__ void normalize_kernel(float* __restrict__ w, const double* __restrict__ nrm2, long long n) {
  const double s = *nrm2;
  if (!(s > 0.0)) return;
  const float inv = (float)(1.0 / sqrt(s));
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    w[e] *= inv;
}

int grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

// FP64 inner product (or squared distance) of two device vectors, returned to the host.
pat_status dot_host(pat_plan* p, const float* a, const float* b, long long n, bool diff, double* out,
                    cudaStream_t st) {
  if (!p->d_kr) PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->d_kr), sizeof(double) * (KB + 1), "reductions"));
  if (diff)
    dot_partial_kernel<true><<<KB, KT, 0, st>>>(a, b, n, p->d_kr);
  else
    dot_partial_kernel<false><<<KB, KT, 0, st>>>(a, b, n, p->d_kr);
  dot_final_kernel<<<1, KT, 0, st>>>(p->d_kr, KB, p->d_kr + KB);
  PAT_TRY_CUDA(cudaGetLastError());
  PAT_TRY_CUDA(cudaMemcpyAsync(out, p->d_kr + KB, sizeof(double), cudaMemcpyDeviceToHost, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

cudaError_t axpy(float* y, const float* x, double a, long long n, cudaStream_t st) {
  axpy_kernel<<<grid_of(n), 256, 0, st>>>(y, x, (float)a, n);
  return cudaGetLastError();
}

cudaError_t scal(float* x, double a, long long n, cudaStream_t st) {
  scal_kernel<<<grid_of(n), 256, 0, st>>>(x, (float)a, n);
  return cudaGetLastError();
}

// J = 1/2 ||K x - y||^2 + alpha/2 ||u||^2 for an image x = E_s u; K x lands in the plan's data buffer.
pat_status objective(pat_plan* p, const float* x, const float* u, const float* y, double alpha, double* J,
                     cudaStream_t st) {
  PAT_TRY(wave_forward(p, x, p->d_ybuf, st));
  double rr = 0.0, uu = 0.0;
  PAT_TRY(dot_host(p, p->d_ybuf, y, (long long)p->ns * p->nt, true, &rr, st));
  PAT_TRY(dot_host(p, u, u, p->N, false, &uu, st));
  *J = 0.5 * rr + 0.5 * alpha * uu;
  return PAT_OK;
}

}  // namespace

// J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 (FP64 reductions) and, when
// grad != nullptr, its gradient E_s* K* (K E_s u - y) + alpha u (FP32).
pat_status objective_device(pat_plan* p, const float* y, double alpha, double s, const float* u, double* J,
                            float* grad, cudaStream_t st) {
  const long long N = p->N, M = (long long)p->ns * p->nt;
  PAT_TRY(apply_Es(p, s, u, p->d_img, st));
  PAT_TRY(wave_forward(p, p->d_img, p->d_ybuf, st));
  PAT_TRY_CUDA(axpy(p->d_ybuf, y, -1.0, M, st));  // r = K E_s u - y
  double rr = 0.0, uu = 0.0;
  PAT_TRY(dot_host(p, p->d_ybuf, p->d_ybuf, M, false, &rr, st));
  PAT_TRY(dot_host(p, u, u, N, false, &uu, st));
  *J = 0.5 * rr + 0.5 * alpha * uu;
  if (grad) {
    PAT_TRY(wave_adjoint(p, p->d_ybuf, p->d_img, st));
    PAT_TRY(apply_EsT(p, s, p->d_img, grad, st));
    PAT_TRY_CUDA(axpy(grad, u, alpha, N, st));
  }
  return PAT_OK;
}

pat_status landweber_device(pat_plan* p, const float* y, double alpha, double s, int iters, double omega, float* u,
                            float* x, double* J, cudaStream_t st) {
  const long long N = p->N, M = (long long)p->ns * p->nt;
  float* uu = u ? u : p->d_u;
  float* b = p->d_r;
  PAT_TRY(wave_adjoint(p, y, p->d_img, st));  // b = E_s* K* y
  PAT_TRY(apply_EsT(p, s, p->d_img, b, st));
  PAT_TRY_CUDA(fill_launch(uu, N, 0.f, st));
  for (int k = 0; k < iters; ++k) {
    PAT_TRY(apply_Es(p, s, uu, p->d_img, st));
    PAT_TRY(wave_forward(p, p->d_img, p->d_ybuf, st));  // K E_s u_k (also the residual of J)
    if (J) {
      double rr = 0.0, u2 = 0.0;
      PAT_TRY(dot_host(p, p->d_ybuf, y, M, true, &rr, st));
      PAT_TRY(dot_host(p, uu, uu, N, false, &u2, st));
      J[k] = 0.5 * rr + 0.5 * alpha * u2;
    }
    PAT_TRY(wave_adjoint(p, p->d_ybuf, p->d_img, st));
    PAT_TRY(apply_EsT(p, s, p->d_img, p->d_q, st));
    lw_update_kernel<<<grid_of(N), 256, 0, st>>>(uu, b, p->d_q, (float)omega, (float)alpha, N);
    PAT_TRY_CUDA(cudaGetLastError());
  }
  float* xx = x ? x : p->d_img;
  PAT_TRY(apply_Es(p, s, uu, xx, st));
  if (J) PAT_TRY(objective(p, xx, uu, y, alpha, &J[iters], st));
  return PAT_OK;
}

pat_status gmres_device(pat_plan* p, const float* y, double alpha, double s, int iters, float* x, double* res,
                        double* J, cudaStream_t st) {
  const long long N = p->N;
  float* V = nullptr;  // Krylov basis, (iters + 1) x N
  {
    const cudaError_t e = cudaMalloc(&V, sizeof(float) * (size_t)N * (iters + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("GMRES basis of %d x %lld floats: %s", iters + 1, N, cudaGetErrorString(e));
      return PAT_ERR_OOM;
    }
  }
  struct Free {
    void* v;
    ~Free() { cudaFree(v); }
  } guard{V};
  // device scratch of the orthogonalisation: block partials of up to iters+1 inner products, the
  // accumulated and per-pass coefficients and the norm
  const int kk_max = iters + 1;
  double* dP = nullptr;
  {
    const cudaError_t e = cudaMalloc(&dP, sizeof(double) * ((size_t)KB * kk_max + 2 * kk_max + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("GMRES scratch: %s", cudaGetErrorString(e));
      return PAT_ERR_OOM;
    }
  }
  Free guard2{dP};
  double* dH = dP + (size_t)KB * kk_max;
  auto Vj = [&](int j) { return V + (size_t)j * N; };
  // w = A v = E_s E_s* K* K v + alpha v
  auto apply_A = [&](const float* v, float* w) -> pat_status {
    PAT_TRY(wave_forward(p, v, p->d_ybuf, st));
    PAT_TRY(wave_adjoint(p, p->d_ybuf, p->d_img, st));
    PAT_TRY(apply_EsT(p, s, p->d_img, p->d_q, st));
    PAT_TRY(apply_Es(p, s, p->d_q, w, st));
    PAT_TRY_CUDA(axpy(w, v, alpha, N, st));
    return PAT_OK;
  };
  // x_k = sum_i z_i V_i, with J(E_s^{-1} x_k) when asked for
  auto assemble = [&](const std::vector<double>& z, int k) -> pat_status {
    PAT_TRY_CUDA(fill_launch(x, N, 0.f, st));
    for (int i = 0; i < k; ++i) PAT_TRY_CUDA(axpy(x, Vj(i), z[i], N, st));
    return PAT_OK;
  };
  auto objective_x = [&](double* Jk) -> pat_status {
    PAT_TRY(apply_EsT(p, -s, x, p->d_u, st));  // u = S_s^{-1} W x
    return objective(p, x, p->d_u, y, alpha, Jk, st);
  };
  // f = Gamma K* y (x_0 = 0, r_0 = f)
  PAT_TRY(wave_adjoint(p, y, p->d_img, st));
  PAT_TRY(apply_EsT(p, s, p->d_img, p->d_q, st));
  PAT_TRY(apply_Es(p, s, p->d_q, Vj(0), st));
  double beta = 0.0;
  PAT_TRY(dot_host(p, Vj(0), Vj(0), N, false, &beta, st));
  beta = std::sqrt(beta);
  if (res) res[0] = beta;
  PAT_TRY_CUDA(fill_launch(x, N, 0.f, st));
  if (J) PAT_TRY(objective_x(&J[0]));
  std::vector<double> H((size_t)(iters + 1) * (iters + 1), 0.0), cs(iters + 1, 0.0), sn(iters + 1, 0.0),
      g(iters + 2, 0.0);
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * (iters + 1) + j]; };
  g[0] = beta;
  int k = 0;  // basis vectors in use
  if (beta > 0.0) PAT_TRY_CUDA(scal(Vj(0), 1.0 / beta, N, st));
  auto solve_z = [&](int kk) {  // back substitution on the rotated upper triangle
    std::vector<double> z(kk, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
      double acc = g[i];
      for (int c = i + 1; c < kk; ++c) acc -= h(i, c) * z[c];
      z[i] = h(i, i) != 0.0 ? acc / h(i, i) : 0.0;
    }
    return z;
  };
  for (int j = 0; j < iters; ++j) {
    if (beta == 0.0 || (j > 0 && h(j, j - 1) == 0.0 && k == j)) {  // converged exactly: repeat the last values
      if (res) res[j + 1] = res[j];
      if (J) J[j + 1] = J[j];
      continue;
    }
    PAT_TRY(apply_A(Vj(j), Vj(j + 1)));
    // classical Gram-Schmidt applied twice (all projections of a pass in one launch, the second pass
    // restores the orthogonality a single classical pass loses); column j of H and the new norm come
    // back to the host in one copy
    const int kk = j + 1;
    double* hcol = dH;          // kk projection coefficients, accumulated over the two passes
    double* c = dH + kk_max;    // this pass's coefficients
    double* nrm = dH + 2 * kk_max;
    for (int pass = 0; pass < 2; ++pass) {
      mdot_partial_kernel<<<dim3(KB, kk), KT, 0, st>>>(V, Vj(j + 1), N, dP);
      mdot_final_kernel<<<kk, KT, 0, st>>>(dP, c, 0);
      maxpy_kernel<<<grid_of(N), 256, 0, st>>>(Vj(j + 1), V, c, kk, N);
      mdot_final_kernel<<<kk, KT, 0, st>>>(dP, hcol, pass);  // hcol (+)= c
    }
    mdot_partial_kernel<<<dim3(KB, 1), KT, 0, st>>>(Vj(j + 1), Vj(j + 1), N, dP);
    mdot_final_kernel<<<1, KT, 0, st>>>(dP, nrm, 0);
    normalize_kernel<<<grid_of(N), 256, 0, st>>>(Vj(j + 1), nrm, N);
    PAT_TRY_CUDA(cudaGetLastError());
    std::vector<double> hv(kk + 1);
    PAT_TRY_CUDA(cudaMemcpyAsync(hv.data(), hcol, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    PAT_TRY_CUDA(cudaMemcpyAsync(hv.data() + kk, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    PAT_TRY_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < kk; ++i) h(i, j) = hv[i];
    const double hn = std::sqrt(std::max(hv[kk], 0.0));
    // previous rotations on column j, then the one that zeroes h(j+1, j)
    for (int i = 0; i < j; ++i) {
      const double a = h(i, j), b = h(i + 1, j);
      h(i, j) = cs[i] * a + sn[i] * b;
      h(i + 1, j) = -sn[i] * a + cs[i] * b;
    }
    const double a = h(j, j), r = std::hypot(a, hn);
    cs[j] = r > 0.0 ? a / r : 1.0;
    sn[j] = r > 0.0 ? hn / r : 0.0;
    h(j, j) = r;
    h(j + 1, j) = hn;  // kept only to detect an exact (lucky) breakdown
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    if (res) res[j + 1] = std::fabs(g[j + 1]);
    if (J) {
      PAT_TRY(assemble(solve_z(k), k));
      PAT_TRY(objective_x(&J[j + 1]));
    }
  }
  PAT_TRY(assemble(solve_z(k), k));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

}  // namespace pat
