// Fused CG vector updates with FP64 device-resident scalars (paper Sec. 4:
// "iterative solution algorithms ... the conjugate gradient method", applied
// to the SPD system (E_s* K* K E_s + alpha I) u = E_s* K* y).
//
// Vectors are FP32; every inner product is accumulated in FP64 with a fixed
// summation order (grid-stride partial per thread, warp shuffles, fixed block
// tree, then the last block to finish sums the per-block partials in block
// order), so results are bit-reproducible run to run.  Step lengths live in
// device memory: the solve never waits for the host.
#include "internal.h"

namespace pat {
namespace {

constexpr int CG_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[CG_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < CG_THREADS / 32; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// Block partial -> partials[block]; the last block reduces them in order and
// calls fin(total) on thread 0.  Returns true in the last block.
template <typename Fin>
__device__ __forceinline__ void grid_sum(double v, double* partials, unsigned* counter, Fin fin) {
  const double bs = block_sum(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += CG_THREADS) s += __ldcg(partials + i);
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *counter = 0u;
    fin(s);
  }
}

__global__ void __launch_bounds__(CG_THREADS) cg_init_kernel(const float* __restrict__ b, float* __restrict__ r,
                                                             float* __restrict__ p, float* __restrict__ u, long long n,
                                                             int zero_u, double* partials, unsigned* counter,
                                                             CgScalars* sc) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS) {
    const float v = b[i];
    r[i] = v;
    p[i] = v;
    if (zero_u) u[i] = 0.f;
    acc += (double)v * (double)v;
  }
  grid_sum(acc, partials, counter, [&](double s) {
    sc->rr = s;
    sc->stopped = 0;
    sc->iter = 0;
  });
}

__global__ void __launch_bounds__(CG_THREADS) cg_sub_kernel(float* __restrict__ r, const float* __restrict__ q,
                                                            long long n) {
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS)
    r[i] -= q[i];
}

// p = r, rr = r.r  (restart after r = b - H u0)
__global__ void __launch_bounds__(CG_THREADS) cg_rr_kernel(const float* __restrict__ r, float* __restrict__ p,
                                                           long long n, double* partials, unsigned* counter,
                                                           CgScalars* sc) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS) {
    const float v = r[i];
    p[i] = v;
    acc += (double)v * (double)v;
  }
  grid_sum(acc, partials, counter, [&](double s) {
    sc->rr = s;
    sc->stopped = 0;
    sc->iter = 0;
  });
}

// q += alpha p ; pq = p.q
__global__ void __launch_bounds__(CG_THREADS) cg_pq_kernel(float* __restrict__ q, const float* __restrict__ p,
                                                           double alpha, long long n, double* partials,
                                                           unsigned* counter, CgScalars* sc) {
  const float af = (float)alpha;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS) {
    const float pv = p[i];
    const float qv = fmaf(af, pv, q[i]);
    q[i] = qv;
    acc += (double)pv * (double)qv;
  }
  grid_sum(acc, partials, counter, [&](double s) { sc->pq = s; });
}

// a = rr / pq ; u += a p ; r -= a q ; rr' = r.r ; beta = rr'/rr
__global__ void __launch_bounds__(CG_THREADS) cg_update_kernel(float* __restrict__ u, float* __restrict__ r,
                                                               const float* __restrict__ p,
                                                               const float* __restrict__ q, long long n,
                                                               double* partials, unsigned* counter, CgScalars* sc,
                                                               double* log, int* status) {
  const double rr = sc->rr, pq = sc->pq;
  const double a = rr / pq;
  const bool stop = sc->stopped != 0 || !(pq > 0.0) || !isfinite(pq) || !isfinite(a);
  if (stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && sc->stopped == 0) {
      sc->stopped = 1;
      atomicCAS(status, (int)PAT_OK, (int)PAT_ERR_BREAKDOWN);
    }
    return;  // every block takes the same decision: the reduction is skipped as a whole
  }
  const float af = (float)a;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS) {
    u[i] = fmaf(af, p[i], u[i]);
    const float rv = fmaf(-af, q[i], r[i]);
    r[i] = rv;
    acc += (double)rv * (double)rv;
  }
  grid_sum(acc, partials, counter, [&](double s) {
    const int k = sc->iter;
    if (log) {
      log[3 * k + 0] = rr;
      log[3 * k + 1] = pq;
      log[3 * k + 2] = a;
    }
    sc->a = a;
    sc->rr_new = s;
    sc->beta = s / rr;
    sc->rr = s;
    sc->iter = k + 1;
  });
}

// p = r + beta p
__global__ void __launch_bounds__(CG_THREADS) cg_direction_kernel(float* __restrict__ p, const float* __restrict__ r,
                                                                  long long n, const CgScalars* sc) {
  if (sc->stopped) return;
  const float b = (float)sc->beta;
  for (long long i = (long long)blockIdx.x * CG_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * CG_THREADS)
    p[i] = fmaf(b, p[i], r[i]);
}

int g_blocks = 0;

}  // namespace

int cg_grid_blocks() {
  if (g_blocks == 0) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_blocks = 2 * sms;
  }
  return g_blocks;
}

cudaError_t cg_init_launch(const float* b, float* r, float* p, float* u, long long n, bool zero_u, double* partials,
                           unsigned* counter, CgScalars* sc, cudaStream_t st) {
  cg_init_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(b, r, p, u, n, zero_u ? 1 : 0, partials, counter, sc);
  return cudaGetLastError();
}

cudaError_t cg_sub_launch(float* r, const float* q, long long n, cudaStream_t st) {
  cg_sub_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(r, q, n);
  return cudaGetLastError();
}

cudaError_t cg_rr_launch(const float* r, float* p, long long n, double* partials, unsigned* counter, CgScalars* sc,
                         cudaStream_t st) {
  cg_rr_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(r, p, n, partials, counter, sc);
  return cudaGetLastError();
}

cudaError_t cg_pq_launch(float* q, const float* p, double alpha, long long n, double* partials, unsigned* counter,
                         CgScalars* sc, cudaStream_t st) {
  cg_pq_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(q, p, alpha, n, partials, counter, sc);
  return cudaGetLastError();
}

cudaError_t cg_update_launch(float* u, float* r, const float* p, const float* q, long long n, double* partials,
                             unsigned* counter, CgScalars* sc, double* log, int* status, cudaStream_t st) {
  cg_update_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(u, r, p, q, n, partials, counter, sc, log, status);
  return cudaGetLastError();
}

cudaError_t cg_direction_launch(float* p, const float* r, long long n, const CgScalars* sc, cudaStream_t st) {
  cg_direction_kernel<<<cg_grid_blocks(), CG_THREADS, 0, st>>>(p, r, n, sc);
  return cudaGetLastError();
}

}  // namespace pat
