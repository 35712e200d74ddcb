// Batched 2D step kernel: one launch advances every running instance of a
// batch by one time step of the increment form (paper Sec. 2, Eq.
// wave_equation, eliminated to p only; constant or varying medium, kappa
// per cell read with the row when the instance has a varying medium):
//
//   forward, n = t:          D <- D + c_lap kappa L P^n,   P^{n+1} = P^n + D,   y[., n] = S P^n
//   adjoint, m = nt - 1 - t: G <- G + S^T r_m + c_lap L Z^{m+1},  Z^m = Z^{m+1} + kappa G
//                            (Z = kappa Q; m = 0: x = G + 1/2 L Z^1)
//
// The adjoint state Z integrates G over time and, in a closed box, grows far
// beyond the result: it is kept as a compensated pair Z + Z_lo (TwoSum), the
// stencil sees Z through the difference form and Z_lo through the sum form,
// as in the single-instance 2D step kernel.
//
// The tiles (64 columns x 64 or 32 rows) of all instances form one table,
// instances ordered by their number of time samples (longest first), so the
// tiles still running at global step t are a prefix of the table.  Persistent
// CTAs walk that prefix with the tile pipeline of the single-instance 2D step
// kernel: TMA halo boxes (P, or Z and Z_lo) in two shared-memory stages, D / G
// in registers, a sliding y window per thread.  Sampling and injection are
// fused per tile (each tile samples the sensors whose base cell it holds and
// injects into its own cells).  Each tile's descriptor (instance, origin, list
// ranges) is read two tiles ahead of its use, so the only loads left between
// the end of one tile and the stencil of the next are the tile's own D cells
// and the TMA boxes issued one tile ahead.
#include <algorithm>
#include <mutex>

#include "batch.h"
#include "stencil.cuh"
#include "tile2d.cuh"
#include "tma.cuh"

namespace pat {
namespace {

constexpr int TX = 64, XH = 8, BW = TX + 2 * XH;

// rows per thread: 8 for the forward; 4 for the adjoint, whose two stencils and two staged boxes
// per tile need more registers and shared memory per cell (twice the threads per tile keep the
// resident warps per SM up)
constexpr int run_rows(bool adj) { return adj ? 4 : 8; }

template <int R, int TY, bool ADJ>
struct GB {
  static constexpr int RUN = run_rows(ADJ);
  static constexpr int THREADS = (TX / 4) * (TY / RUN);
  static constexpr int PBOX = BW * (TY + 2 * R);  // floats (multiple of 32: 128-byte aligned stages)
  static constexpr int STAGE = (ADJ ? 2 : 1) * PBOX;
  static constexpr size_t SMEM = sizeof(float) * 2 * STAGE + 16;
};

// Grid-wide barrier of a cooperative launch: every CTA arrives once per
// barrier on a monotonic counter and waits (bounded) until all gridDim.x CTAs
// of barrier `round` (1, 2, ...) have arrived.  Thread 0 releases the CTA's
// global writes before arriving and, after the acquire, fences the async proxy
// so that the TMA loads it issues next see the other CTAs' writes.  False when
// the wait gave up (timeout, or another CTA recorded a failure in `status`).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned round, int* status, long long timeout_ns) {
  __syncthreads();
  int fail = 0;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = round * gridDim.x;
    const unsigned long long t0 = global_timer_ns();
    for (unsigned it = 0;; ++it) {
      if (ld_acquire_gpu_u(bar) >= target) break;
      if ((it & 63u) == 63u) {
        if (ld_relaxed_gpu(status) != (int)PAT_OK || (long long)(global_timer_ns() - t0) > timeout_ns ||
            it > (1u << 30)) {
          atomicCAS(status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
          fail = 1;
          break;
        }
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  return __syncthreads_or(fail) == 0;
}

template <int R, int TY, bool ADJ, bool RUNALL>
__global__ void __launch_bounds__(GB<R, TY, ADJ>::THREADS) batch_step_kernel(const BatchStepArgs a) {
  using G = GB<R, TY, ADJ>;
  constexpr int THREADS = G::THREADS, RUN = G::RUN;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage0 + 2 * G::STAGE);

  const int t = threadIdx.x;
  const int c0 = (t % (TX / 4)) * 4, r0 = (t / (TX / 4)) * RUN;
  float2 w2[R + 1];  // stencil weights, packed
#pragma unroll
  for (int m = 0; m <= R; ++m) w2[m] = dup2(a.w[m]);

  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  int k = 0, issued = 0;  // tiles processed (stage k & 1, phase (k >> 1) & 1) and TMA pairs issued, over all steps
  bool ok = true;
  const int t_end = RUNALL ? a.t_end : a.t + 1;
  for (int step = a.t; step < t_end && ok; ++step) {
  if (RUNALL && step > a.t && !grid_barrier(a.bar, (unsigned)(step - a.t), a.status, a.timeout_ns)) {
    ok = false;
    break;
  }
  const int active = RUNALL ? __ldg(a.active_dev + step) : a.active;

  // tile descriptor in registers: instance, origin and the list range of this direction
  // (an empty descriptor past the active prefix)
  struct Desc {
    int inst, gx0, gy0, e0, e1;
  };
  auto desc = [&](int tile) {
    Desc d{0, 0, 0, 0, 0};
    if (tile < active) {
      const int4* p = reinterpret_cast<const int4*>(a.tiles + tile);
      const int4 u = __ldg(p), v = __ldg(p + 1);
      d = Desc{u.x, u.y, u.z, ADJ ? v.z : v.x, ADJ ? v.w : v.y};
    }
    return d;
  };
  // halo boxes of the fields the tile's stencil reads at this step
  auto issue = [&](const Desc& d, int s) {
    const CUtensorMap* maps = a.maps + BATCH_MAPS * d.inst;
    float* st = stage0 + s * G::STAGE;
    mbar_expect_tx(&bars[s], (unsigned)G::STAGE * 4u);
    tma_load_2d(st, maps + ((!ADJ && step == 0) ? 2 : (step & 1)), d.gx0 - XH, d.gy0 - R, &bars[s]);
    if (ADJ) tma_load_2d(st + G::PBOX, maps + 3 + (step & 1), d.gx0 - XH, d.gy0 - R, &bars[s]);
  };
  Desc dc = desc(blockIdx.x), dn = desc(blockIdx.x + gridDim.x);
  if ((int)blockIdx.x < active) {
    if (t == 0) issue(dc, k & 1);
    ++issued;
  }

  for (int tile = blockIdx.x; tile < active; tile += gridDim.x, ++k) {
    const int s = k & 1;
    const int nxt = tile + gridDim.x;
    const Desc dnn = desc(nxt + gridDim.x);  // consumed two tiles from now
    if (t == 0) {
      fence_proxy_async_shared();  // the other stage was last read through the generic proxy
      if (nxt < active) {
        issue(dn, s ^ 1);
        ++issued;
      }
    }
    const BInst& I = a.inst[dc.inst];
    const int nx = I.nx, ny = I.ny, nt = I.nt;
    const int gx0 = dc.gx0, gy0 = dc.gy0;
    const int gx = gx0 + c0;
    const int n = ADJ ? nt - 1 - step : step;  // the instance's own time index
    const float* cur = (!ADJ && step == 0) ? I.img : I.P[step & 1];
    const bool final_step = ADJ && n == 0;
    const bool compute = ADJ || n < nt - 1;  // the forward's last index only samples
    float* out = final_step ? const_cast<float*>(I.img) : I.P[(step + 1) & 1];

    const bool load_d = !(!ADJ && n == 0);
    float4 d4[RUN];
    auto load_own_d = [&]() {
#pragma unroll
      for (int rr = 0; rr < RUN; ++rr) {
        const int gy = gy0 + r0 + rr;
        const bool in = compute && load_d && gy < ny && gx < nx;
        d4[rr] = in ? ld_stream4(I.D + (long long)gy * nx + gx) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    if (!ADJ) {  // y[s, n] = sum_k w_k P^n[cell_k] for the sensors based in this tile
      load_own_d();  // independent of the sampling: in flight while it runs
      for (int e = dc.e0 + t; e < dc.e1; e += THREADS) {
        const int sn = I.samp[e];
        float v = 0.f;
        for (int q = 0; q < I.corners; ++q)
          v = fmaf(I.sens_w[sn * I.corners + q], cur[I.sens_cell[sn * I.corners + q]], v);
        I.y[(long long)sn * nt + n] = v;
      }
    } else {  // G += S^T r_m on the tile's own cells
      if (dc.e1 > dc.e0) {  // uniform over the CTA
        for (int e = dc.e0 + t; e < dc.e1; e += THREADS) {
          const InjCell c = I.inj[e];
          float v = 0.f;
          for (int q = c.beg; q < c.end; ++q) v = fmaf(I.ent_w[q], I.y[(long long)I.ent_sensor[q] * nt + n], v);
          I.D[c.local] += v;
        }
        __syncthreads();  // the injected cells are read below by other threads of the CTA
      }
      load_own_d();
    }

    const bool good = mbar_wait(&bars[s], (k >> 1) & 1, a.timeout_ns);
    if (__syncthreads_or(!good)) {
      if (t == 0) atomicCAS(a.status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
      ok = false;
      break;
    }
    if (compute) {
      const float* P = stage0 + s * G::STAGE;  // P (forward) or Z (adjoint)
      const float* PL = P + G::PBOX;           // adjoint: Z_lo
      const float c_lap = (n == 0 || final_step) ? 0.5f : 1.f;
      const float ckh = c_lap * I.kappa0, ckl = c_lap * I.kappa0_lo;
      const bool varying = I.kappa != nullptr;  // uniform over the tile (one instance)
      float lo[RUN][4];  // adjoint: the Z_lo part of the stencil, first pass
      if (ADJ) stencil_run<R, RUN, BW, XH>(PL, r0, c0, a.w, lo);
      float4 win[2 * R + 1];
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) win[i] = *reinterpret_cast<const float4*>(P + (r0 + i) * BW + XH + c0);
#pragma unroll
      for (int rr = 0; rr < RUN; ++rr) {
        win[2 * R] = *reinterpret_cast<const float4*>(P + (r0 + rr + 2 * R) * BW + XH + c0);
        const int brow = r0 + rr + R;
        float f[20];
        load_row20(P + brow * BW + c0, f);
        float4 zl4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ADJ) zl4 = *reinterpret_cast<const float4*>(PL + brow * BW + XH + c0);
        // a varying medium's kappa (forward: hi and lo parts) for this row, in flight during the stencil
        const int gy = gy0 + r0 + rr;
        const bool own = gy < ny && gx < nx;
        float4 kh = make_float4(0.f, 0.f, 0.f, 0.f), kl = kh;
        if (varying && own) {
          kh = __ldg(reinterpret_cast<const float4*>(I.kappa + (long long)gy * nx + gx));
          if (!ADJ) kl = __ldg(reinterpret_cast<const float4*>(I.kappa_lo + (long long)gy * nx + gx));
        }
        float dn[4], pn[4], pl[4];
        float st4[4];
        stencil_cells2<R, ADJ>(win, f, w2, st4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float c = f[8 + j];
          if (!ADJ) {  // zero-sum pair form (a + b) - 2c per tap
            const float acc = st4[j];
            // D += c_lap (kappa_hi + kappa_lo) L, the product rounded once before it meets D
            const float inc = varying ? fmaf(c_lap * f4get(kh, j), acc, (c_lap * f4get(kl, j)) * acc)
                                      : fmaf(ckh, acc, ckl * acc);
            dn[j] = f4get(d4[rr], j) + inc;
            pn[j] = c + dn[j];
            pl[j] = 0.f;
          } else {
            const float acc = st4[j] + lo[rr][j];  // difference form on Z
            const float g = fmaf(c_lap, acc, f4get(d4[rr], j));
            dn[j] = g;
            float e = 0.f;
            const float u = varying ? f4get(kh, j) * g : fmaf(I.kappa0, g, I.kappa0_lo * g);  // kappa G
            pn[j] = final_step ? g : two_sum(c, u, e);                                          // Z += kappa G
            pl[j] = f4get(zl4, j) + e;
          }
        }
        if (own) {
          const long long gi = (long long)gy * nx + gx;
          *reinterpret_cast<float4*>(out + gi) = make_float4(pn[0], pn[1], pn[2], pn[3]);
          if (!final_step) {
            *reinterpret_cast<float4*>(I.D + gi) = make_float4(dn[0], dn[1], dn[2], dn[3]);
            if (ADJ) *reinterpret_cast<float4*>(I.P_lo[(step + 1) & 1] + gi) = make_float4(pl[0], pl[1], pl[2], pl[3]);
          }
        }
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) win[i] = win[i + 1];
      }
    }
    __syncthreads();  // this stage is refilled by the next iteration's TMA
    dc = dn;
    dn = dnn;
  }
  }  // steps
  // after a timed-out wait: give the copies in flight a bounded chance to land
  if (t == 0 && !ok)
    for (int j = max(0, issued - 2); j < issued; ++j) mbar_wait(&bars[j & 1], (j >> 1) & 1, a.timeout_ns);
}

template <int R, int TY>
const void* kernel_ptr(bool adj, bool runall) {
  if (runall)
    return adj ? reinterpret_cast<const void*>(&batch_step_kernel<R, TY, true, true>)
               : reinterpret_cast<const void*>(&batch_step_kernel<R, TY, false, true>);
  return adj ? reinterpret_cast<const void*>(&batch_step_kernel<R, TY, true, false>)
             : reinterpret_cast<const void*>(&batch_step_kernel<R, TY, false, false>);
}

const void* kernel_for(int R, int variant, bool adj, bool runall = false) {
  const bool tall = variant == 0;
  switch (R) {
    case 1: return tall ? kernel_ptr<1, 64>(adj, runall) : kernel_ptr<1, 32>(adj, runall);
    case 3: return tall ? kernel_ptr<3, 64>(adj, runall) : kernel_ptr<3, 32>(adj, runall);
    case 5: return tall ? kernel_ptr<5, 64>(adj, runall) : kernel_ptr<5, 32>(adj, runall);
    case 7: return tall ? kernel_ptr<7, 64>(adj, runall) : kernel_ptr<7, 32>(adj, runall);
    default: return nullptr;
  }
}

int threads_for(int variant, bool adj) { return (TX / 4) * (batch_tile_y(variant) / run_rows(adj)); }

}  // namespace

int batch_tile_y(int variant) { return variant == 0 ? 64 : 32; }

size_t batch_smem(int R, int variant, bool adj) {
  return sizeof(float) * 2 * (adj ? 2 : 1) * (size_t)BW * (batch_tile_y(variant) + 2 * R) + 16;
}

int batch_max_ctas(int R, int variant, bool adj) {
  // co-resident CTAs of the per-step and of the run-all kernel alike (the smaller of the two)
  int best = -1;
  for (int runall = 0; runall < 2; ++runall) {
    const void* fn = kernel_for(R, variant, adj, runall != 0);
    if (!fn) return 0;
    const size_t smem = batch_smem(R, variant, adj);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads_for(variant, adj), smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = best < 0 ? per * sms : std::min(best, per * sms);
  }
  return best;
}

cudaError_t batch_step_launch(int R, int variant, const BatchStepArgs& a, int nctas, cudaStream_t st) {
  if (a.active <= 0) return cudaSuccess;
  const bool adj = a.adjoint != 0;
  const void* fn = kernel_for(R, variant, adj);
  if (!fn) return cudaErrorInvalidValue;
  const int grid = nctas < a.active ? nctas : a.active;
  void* args[] = {const_cast<BatchStepArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads_for(variant, adj)), args, batch_smem(R, variant, adj), st);
}

cudaError_t batch_run_launch(int R, int variant, const BatchStepArgs& a, int nctas, cudaStream_t st) {
  if (a.t_end <= a.t) return cudaSuccess;
  const bool adj = a.adjoint != 0;
  const void* fn = kernel_for(R, variant, adj, true);
  if (!fn || nctas <= 0) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(threads_for(variant, adj));
  cfg.dynamicSmemBytes = batch_smem(R, variant, adj);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA co-resident: the grid barrier cannot deadlock
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<BatchStepArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t batch_encode(const float* base, int nx, int ny, int R, int variant, CUtensorMap* map) {
  auto fn = tma_encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t box[2] = {(cuuint32_t)BW, (cuuint32_t)(batch_tile_y(variant) + 2 * R)};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace pat
