// 2D wave step with TMA-fed tile pipelines: one launch per time step of the
// increment form (paper Sec. 2, Eq. wave_equation, eliminated to p only)
//
//   D^{n+1} = D^n + c_lap (kappa_hi + kappa_lo) L P^n,   P^{n+1} = P^n + D^{n+1}
//
// For a constant medium the adjoint recurrence has the same form,
// G^m = G^{m+1} + S^T r_m + kappa L Q^{m+1}, Q^m = Q^{m+1} + G^m, and runs
// through the same kernel (the injection S^T r_m is added to G beforehand;
// the final step writes x = G + c_lap kappa L Q^1).
//
// Persistent CTAs walk 64 x 64 tiles; one thread issues the TMA load of the
// next tile's P box (80 x (64+2R), halo included, zero outside the grid) into
// the second of two shared-memory stages while the CTA computes the current
// one.  Each thread owns 4 columns x 8 consecutive rows: y neighbours come
// from a sliding register window of 2R+1 rows, x neighbours from the
// shared-memory row; its own D (and kappa) cells are loaded straight into
// registers (coalesced 16-byte loads issued before the wait for the P box).
// Compulsory DRAM traffic per point-update: P and D read, P^{n+1} and D^{n+1}
// written (16 B), plus kappa hi/lo (8 B) for a varying medium.
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "internal.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace pat {
namespace {

constexpr int TX = 64, TY = 64, RUN = 8;
constexpr int TCOLS = TX / 4, TROWS = TY / RUN, THREADS = TCOLS * TROWS;  // 16 x 8 = 128
constexpr int XH = 8;            // box columns left of the tile (>= R, 16-byte aligned)
constexpr int BW = TX + 2 * XH;  // P box width, 80 floats

template <int R, int NBOX = 1>
struct G2 {
  static constexpr int BH = TY + 2 * R;
  static constexpr int PBOX = BW * BH;  // floats (multiple of 32: 128-byte aligned)
  static constexpr int STAGE = NBOX * PBOX;  // mode 3 stages the field and kappa
  static constexpr size_t SMEM = sizeof(float) * 2 * STAGE + 16;
};

__device__ __forceinline__ void fused_sample2(const StepArgs& a, long long gtid) {
  if (a.y == nullptr || gtid >= a.ns) return;
  const int s = (int)gtid;
  float v = 0.f;
  for (int k = 0; k < a.corners; ++k) v = fmaf(a.sens_w[s * a.corners + k], a.cur[a.sens_cell[s * a.corners + k]], v);
  a.y[(long long)s * a.nt + a.t_sample] = v;
}

// MODE 0: constant medium; 1: varying medium (forward); 2: constant medium with the adjoint's
// injection S^T r_m fused (a separate instance, so the other modes keep their code generation);
// 3: varying-medium adjoint, G' = G + c_lap L(kappa Q), Q' = Q + G': the stage holds boxes of Q and
// kappa, turned into W = kappa Q in shared memory before the stencil (uncompensated: FP32 emulation
// of the 512^2 / 1500-step order-8 workload gives 2.4e-6 against 1.5e-6 with TwoSum compensation).
// SP 0: no absorbing layer; 1: layer, forward update; 2: layer, adjoint update.  With the layer's
// per-cell factors a = (1-q)/(1+q), b = 1/(1+q), q = sigma dt/2:
//   forward  D' = a D + b inc (first step: D' = (a-1) P + b inc),  P' = P + D'
//   adjoint  G' = G + inc,  Q' = a Q + b G'  (final step: x = G' + ((a-1)/b) Q)
// Tiles that do not reach the layer use a = b = 1 without loading the factors.
template <int R, int MODE, int SP>
__global__ void __launch_bounds__(THREADS) step2d_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap mp,
                                                             const __grid_constant__ CUtensorMap mk, int* status,
                                                             long long timeout_ns) {
  constexpr bool VARC = MODE == 1, INJ = MODE == 2, WK = MODE == 3;
  using G = G2<R, WK ? 2 : 1>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage0 + 2 * G::STAGE);
  float* injt = stage0 + 2 * G::STAGE + 4;  // INJ: TX x TY injection tile after the barriers (16-byte aligned)

  const int t = threadIdx.x;
  fused_sample2(a, (long long)blockIdx.x * THREADS + t);
  if (INJ)
    for (int i = t; i < TX * TY / 4; i += THREADS) reinterpret_cast<float4*>(injt)[i] = make_float4(0.f, 0.f, 0.f, 0.f);

  const int nx = a.nx, ny = a.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int ntiles = tiles_x * ((ny + TY - 1) / TY);
  const int c0 = (t % TCOLS) * 4, r0 = (t / TCOLS) * RUN;
  const bool load_d = !a.d_zero;
  const unsigned stage_bytes = (unsigned)G::STAGE * 4u;

  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int tile, int s) {
    float* st = stage0 + s * G::STAGE;
    const int gx0 = (tile % tiles_x) * TX, gy0 = (tile / tiles_x) * TY;
    mbar_expect_tx(&bars[s], stage_bytes);
    tma_load_2d(st, &mp, gx0 - XH, gy0 - R, &bars[s]);
    if (WK) tma_load_2d(st + G::PBOX, &mk, gx0 - XH, gy0 - R, &bars[s]);
  };
  int first = blockIdx.x;
  if (t == 0 && first < ntiles) issue(first, 0);

  const float ckh = a.c_lap * a.kappa0, ckl = a.c_lap * a.kappa0_lo;
  int k = 0;
  bool ok = true;
  int issued = (first < ntiles) ? 1 : 0;
  for (int tile = first; tile < ntiles; tile += gridDim.x, ++k) {
    const int s = k & 1;
    if (t == 0) {
      fence_proxy_async_shared();  // the other stage was last read through the generic proxy
      const int nxt = tile + gridDim.x;
      if (nxt < ntiles) {
        issue(nxt, s ^ 1);
        ++issued;
      }
    }
    const int gx0 = (tile % tiles_x) * TX, gy0 = (tile / tiles_x) * TY;
    const int gx = gx0 + c0;
    // own-cell fields straight into registers, in flight while the P box lands
    float4 d4[RUN], kh4[RUN], kl4[RUN];
#pragma unroll
    for (int rr = 0; rr < RUN; ++rr) {
      const int gy = gy0 + r0 + rr;
      const bool in = gy < ny && gx < nx;
      const long long gi = (long long)gy * nx + gx;
      d4[rr] = (load_d && in) ? ld_stream4(a.dbuf + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (VARC) {
        kh4[rr] = in ? __ldg(reinterpret_cast<const float4*>(a.kappa + gi)) : make_float4(0.f, 0.f, 0.f, 0.f);
        kl4[rr] = in ? __ldg(reinterpret_cast<const float4*>(a.kappa_lo + gi)) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        kh4[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
        kl4[rr] = kh4[rr];
      }
    }
    int inj_b = 0, inj_e = 0;
    if (INJ) {  // adjoint: S^T r_m of the tile's injected cells into the shared tile (each cell listed once)
      inj_b = a.inj_tile_ptr[tile];
      inj_e = a.inj_tile_ptr[tile + 1];
      for (int e = inj_b + t; e < inj_e; e += THREADS) {
        const InjCell c = a.inj_tile[e];  // .local = ly * 64 + lx within the tile
        float v = 0.f;
        for (int q = c.beg; q < c.end; ++q)
          v = fmaf(a.ent_w[q], a.inj_r[(long long)a.ent_sensor[q] * a.nt + a.inj_t], v);
        injt[c.local] = v;
      }
    }
    const bool good = mbar_wait(&bars[s], (k >> 1) & 1, timeout_ns);
    if (__syncthreads_or(!good)) {
      if (t == 0) atomicCAS(status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
      ok = false;
      break;
    }
    float* Pw = stage0 + s * G::STAGE;
    const float* P = Pw;
    float4 qown[RUN];  // mode 3: this thread's own Q cells (the box becomes W = kappa Q)
    if (WK) {
#pragma unroll
      for (int rr = 0; rr < RUN; ++rr) qown[rr] = *reinterpret_cast<const float4*>(P + (r0 + rr + R) * BW + XH + c0);
      __syncthreads();
      float4* W4 = reinterpret_cast<float4*>(Pw);
      const float4* K4 = reinterpret_cast<const float4*>(Pw + G::PBOX);
      for (int i = t; i < G::PBOX / 4; i += THREADS) {
        const float4 q = W4[i], kk = K4[i];
        W4[i] = make_float4(kk.x * q.x, kk.y * q.y, kk.z * q.z, kk.w * q.w);
      }
      __syncthreads();
    }
    // absorbing layer: does the tile reach it (its factors are then loaded row by row)
    const bool layer = SP != 0 && (gx0 < a.sp_w || gx0 + TX > nx - a.sp_w || gy0 < a.sp_w || gy0 + TY > ny - a.sp_w);
    if (INJ && inj_e > inj_b) {  // G += S^T r_m in the owners' registers; the shared tile is cleared again
#pragma unroll
      for (int rr = 0; rr < RUN; ++rr) {
        float4* q = reinterpret_cast<float4*>(injt + (r0 + rr) * TX + c0);
        const float4 v = *q;
        d4[rr].x += v.x;
        d4[rr].y += v.y;
        d4[rr].z += v.z;
        d4[rr].w += v.w;
        *q = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }

    // the tile's update; instantiated separately for tiles inside and outside the layer, so that
    // tiles outside it run exactly the code of the kernel without a layer
    auto update = [&](auto in_layer) {
      constexpr bool LAYER = decltype(in_layer)::value;
      // sliding window over this thread's 4 columns: win[i] = box row (row - R + i)
      float4 win[2 * R + 1];
  #pragma unroll
      for (int i = 0; i < 2 * R; ++i) win[i] = *reinterpret_cast<const float4*>(P + (r0 + i) * BW + XH + c0);
  #pragma unroll
      for (int rr = 0; rr < RUN; ++rr) {
        win[2 * R] = *reinterpret_cast<const float4*>(P + (r0 + rr + 2 * R) * BW + XH + c0);
        const int brow = r0 + rr + R;
        float f[20];
  #pragma unroll
        for (int q = 0; q < 5; ++q) {
          const float4 v = *reinterpret_cast<const float4*>(P + brow * BW + c0 + 4 * q);
          f[4 * q + 0] = v.x;
          f[4 * q + 1] = v.y;
          f[4 * q + 2] = v.z;
          f[4 * q + 3] = v.w;
        }
        const int gy = gy0 + r0 + rr;
        const long long gi = (long long)gy * nx + gx;
        const bool in = gy < ny && gx < nx;
        float dn[4], pn[4];
        float4 sa4 = make_float4(1.f, 1.f, 1.f, 1.f), sb4 = sa4;
        if (LAYER && in) {
          sa4 = __ldg(reinterpret_cast<const float4*>(a.sp_a + gi));
          sb4 = __ldg(reinterpret_cast<const float4*>(a.sp_b + gi));
        }
  #pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float c = f[8 + j];
          const float c2 = c + c;
          float acc = 0.f;  // zero-sum pair form (a + b) - 2c per tap: 3 FP operations instead of 4
  #pragma unroll
          for (int m = 1; m <= R; ++m)
            acc = fmaf(a.w[m], pair_term<false>(f4get(win[R + m], j), f4get(win[R - m], j), c, c2), acc);
  #pragma unroll
          for (int m = 1; m <= R; ++m) acc = fmaf(a.w[m], pair_term<false>(f[8 + j + m], f[8 + j - m], c, c2), acc);
          float inc;
          if (WK)
            inc = a.c_lap * acc;  // kappa is inside the stencil field
          else if (VARC)
            inc = fmaf(a.c_lap * f4get(kh4[rr], j), acc, (a.c_lap * f4get(kl4[rr], j)) * acc);
          else
            inc = fmaf(ckh, acc, ckl * acc);
          const float qv = WK ? f4get(qown[rr], j) : c;  // the stepped field at this cell
          if (!LAYER) {
            dn[j] = f4get(d4[rr], j) + inc;
            pn[j] = a.final_step ? dn[j] : qv + dn[j];
          } else if (SP == 1) {  // forward in the layer
            const float fa = f4get(sa4, j), fb = f4get(sb4, j);
            dn[j] = load_d ? fmaf(fa, f4get(d4[rr], j), fb * inc) : fmaf(fa - 1.f, c, fb * inc);
            pn[j] = c + dn[j];
          } else {  // adjoint in the layer
            const float fa = f4get(sa4, j), fb = f4get(sb4, j);
            dn[j] = f4get(d4[rr], j) + inc;
            pn[j] = a.final_step ? fmaf((fa - 1.f) / fb, qv, dn[j]) : fmaf(fa, qv, fb * dn[j]);
          }
        }
        if (in) {
          *reinterpret_cast<float4*>(a.next + gi) = make_float4(pn[0], pn[1], pn[2], pn[3]);
          if (!a.final_step) *reinterpret_cast<float4*>(a.dbuf + gi) = make_float4(dn[0], dn[1], dn[2], dn[3]);
        }
  #pragma unroll
        for (int i = 0; i < 2 * R; ++i) win[i] = win[i + 1];
      }
    };
    if (SP != 0 && layer)
      update(std::true_type{});
    else
      update(std::false_type{});
    __syncthreads();  // this stage is refilled by the next iteration's TMA
  }
  // after a timed-out wait: give the copies in flight a bounded chance to land
  if (t == 0 && !ok)
    for (int j = max(0, issued - 2); j < issued; ++j) mbar_wait(&bars[j & 1], (j >> 1) & 1, timeout_ns);
}

template <int R, int MODE, int SP>
const void* kfn() {
  return reinterpret_cast<const void*>(&step2d_tma_kernel<R, MODE, SP>);
}

template <int R>
const void* kernel_r(int mode, int sp) {
  switch (mode * 3 + sp) {
    case 0: return kfn<R, 0, 0>();
    case 1: return kfn<R, 0, 1>();
    case 2: return kfn<R, 0, 2>();
    case 3: return kfn<R, 1, 0>();
    case 4: return kfn<R, 1, 1>();
    case 6: return kfn<R, 2, 0>();
    case 8: return kfn<R, 2, 2>();
    case 9: return kfn<R, 3, 0>();
    case 11: return kfn<R, 3, 2>();
    default: return nullptr;  // mismatched layer modes are not instantiated
  }
}

const void* kernel_for(int R, int mode, int sp) {
  switch (R) {
    case 1: return kernel_r<1>(mode, sp);
    case 3: return kernel_r<3>(mode, sp);
    case 5: return kernel_r<5>(mode, sp);
    case 7: return kernel_r<7>(mode, sp);
    default: return nullptr;
  }
}

size_t smem_for(int R, int mode) {
  const size_t base = mode == 3 ? (R == 1 ? G2<1, 2>::SMEM : R == 3 ? G2<3, 2>::SMEM : R == 5 ? G2<5, 2>::SMEM
                                                                                       : G2<7, 2>::SMEM)
                                : (R == 1 ? G2<1>::SMEM : R == 3 ? G2<3>::SMEM : R == 5 ? G2<5>::SMEM : G2<7>::SMEM);
  return base + (mode == 2 ? sizeof(float) * TX * TY : 0);
}

}  // namespace

bool tma2d_supported(int nx, int R) { return nx % 4 == 0 && (R == 1 || R == 3 || R == 5 || R == 7); }

// Descriptors of a 2D field: P boxes (80 x (64+2R)) and own-tile boxes (64 x 64, kept for
// kernels that stage own cells through shared memory).
cudaError_t tma2d_encode(const float* base, int nx, int ny, int R, CUtensorMap* halo, CUtensorMap* own) {
  auto fn = tma_encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t box_h[2] = {(cuuint32_t)BW, (cuuint32_t)(TY + 2 * R)};
  const cuuint32_t box_o[2] = {(cuuint32_t)TX, (cuuint32_t)TY};
  CUresult r1 = fn(halo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box_h, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = fn(own, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box_o, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

// Persistent grid: as many CTAs as fit on the device, at most one per tile.
int tma2d_ctas(int nx, int ny, int R, int mode, int sp) {
  static int cached[4][3][8] = {{{0}}};
  int& c = cached[mode][sp][R];
  if (!c) {
    int dev = 0, sms = 148, per = 1;
    const void* fn = kernel_for(R, mode, sp);
    const size_t smem = smem_for(R, mode);
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // mode 2 holds 16 KB more shared memory per CTA: ask for the largest carveout so that three CTAs
    // fit an SM (modes 0 and 1 run faster with the default split, which leaves L1 larger)
    if (mode == 2) cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, THREADS, smem) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    c = per * sms;
  }
  const int ntiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  return ntiles < c ? ntiles : c;
}

long long tma2d_threads(int nx, int ny, int R, int mode, int sp) {
  return (long long)tma2d_ctas(nx, ny, R, mode, sp) * THREADS;
}

cudaError_t step2d_tma_launch(int R, int mode, int sp, const StepArgs& a, const CUtensorMap& p, const CUtensorMap& k,
                              int* status, long long timeout_ns, cudaStream_t st) {
  const void* fn = kernel_for(R, mode, sp);
  if (!fn) return cudaErrorInvalidValue;
  const int nctas = tma2d_ctas(a.nx, a.ny, R, mode, sp);  // sets the kernel's attributes once
  CUtensorMap map = p, mapk = k;
  StepArgs args = a;
  void* params[] = {&args, &map, &mapk, &status, &timeout_ns};
  return cudaLaunchKernel(fn, dim3(nctas), dim3(THREADS), params, smem_for(R, mode), st);
}

}  // namespace pat
