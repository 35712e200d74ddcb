// 2D wave step with TMA-fed tile pipelines: one launch per time step of the
// increment form (paper Sec. 2, Eq. wave_equation, eliminated to p only)
//
//   forward:  D^{n+1} = D^n + c_lap (kappa_hi + kappa_lo) L P^n,   P^{n+1} = P^n + D^{n+1}
//   adjoint:  G^m = G^{m+1} + S^T r_m + c_lap L(kappa Q^{m+1}),    Q^m = Q^{m+1} + G^m
//             (final step: x = G^0 = G^1 + S^T r_0 + 1/2 L(kappa Q^1))
//
// The adjoint runs in the variable Z = kappa Q (constant or varying medium):
// Z^m = Z^{m+1} + kappa G^m, and the stencil acts on Z directly.  In a closed
// box Z integrates G over time and grows far beyond the result, so Z is kept
// as a compensated pair Z + Z_lo (TwoSum), the stencil sees both parts
// (Z through the difference form (a - c) + (b - c), whose rounding is relative
// to the differences, Z_lo through the cheapest sum form), and G is plain.
// FP32 emulation of the 512^2, 1500-step, order-8 adjoint with noisy data
// simulated from a phantom: 1.9e-5 for the plain pair-form recurrence
// (constant and varying medium), 1.5e-5 with the difference form alone,
// 7e-7 with the compensated Z.  The sensor injection S^T r_m is added to G by
// a separate launch before the step.
//
// Persistent CTAs walk 64 x 64 tiles; one thread issues the TMA load of the
// next tile's boxes (80 x (64+2R) floats, halo included, zero outside the
// grid: P for the forward, Z and Z_lo for the adjoint) into the second of two
// shared-memory stages while the CTA computes the current one.  Each thread
// owns 4 columns x 8 consecutive rows (4 rows in the adjoint, whose two boxes
// and two stencils per cell need more registers: 256 threads of at most 170
// registers per tile ran 6-19 % faster at 4096^2 than 128 threads of 238,
// and faster than 256 threads capped at 128 registers, which spilled).
// y neighbours come from a sliding register window of 2R+1 rows, x
// neighbours from the shared-memory row; its own D / G (and kappa) cells are
// loaded straight into registers (coalesced 16-byte loads issued before the
// wait for the boxes).
// Compulsory DRAM traffic per point-update: forward P and D read, P^{n+1} and
// D^{n+1} written (16 B), plus kappa hi/lo (8 B) for a varying medium;
// adjoint Z, Z_lo, G read and written (24 B), plus kappa (4 B) for a varying
// medium.
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "internal.h"
#include "stencil.cuh"
#include "tile2d.cuh"
#include "tma.cuh"

namespace pat {
namespace {

constexpr int TX = 64, TY = 64, TCOLS = TX / 4;
// rows per thread: 8 for the forward (128 threads per tile); 4 for the adjoint (256 threads), whose
// two stencils and two staged boxes need more registers and shared memory per cell
__host__ __device__ constexpr int run_rows(int mode) { return mode == 2 ? 4 : 8; }
__host__ __device__ constexpr int threads_of(int mode) { return TCOLS * (TY / run_rows(mode)); }
constexpr int XH = 8;            // box columns left of the tile (>= R, 16-byte aligned)
constexpr int BW = TX + 2 * XH;  // box width, 80 floats

template <int R, int NBOX = 1>
struct G2 {
  static constexpr int BH = TY + 2 * R;
  static constexpr int PBOX = BW * BH;       // floats (multiple of 32: 128-byte aligned)
  static constexpr int STAGE = NBOX * PBOX;  // the adjoint stages Z and Z_lo
  static constexpr size_t SMEM = sizeof(float) * 2 * STAGE + 16;
};

// Sensor s = b + t * gridDim.x is sampled by thread t of CTA b (the sensors spread over every CTA).
__device__ __forceinline__ void fused_sample2(const StepArgs& a, long long bid, int t) {
  const long long gs = bid + (long long)t * gridDim.x;
  if (a.y == nullptr || gs >= a.ns) return;
  const int s = (int)gs;
  float v = 0.f;
  for (int k = 0; k < a.corners; ++k) v = fmaf(a.sens_w[s * a.corners + k], a.cur[a.sens_cell[s * a.corners + k]], v);
  a.y[(long long)s * a.nt + a.t_sample] = v;
}

// MODE 0: constant medium, forward; 1: varying medium, forward; 2: adjoint (either medium) in
// Z = kappa Q with Z compensated.  SP 0: no absorbing layer; 1: layer, forward update; 2: layer,
// adjoint update.  With the layer's per-cell factors a = (1-q)/(1+q), b = 1/(1+q), q = sigma dt/2:
//   forward  D' = a D + b inc (first step: D' = (a-1) P + b inc),  P' = P + D'
//   adjoint  G' = G + inc,  Q' = a Q + b G', i.e. Z' = a Z + b kappa G'  (final step: x = G' + ((a-1)/b) Q)
// Tiles that do not reach the layer use a = b = 1 without loading the factors.
template <int R, int MODE, int SP>
__global__ void __launch_bounds__(threads_of(MODE)) step2d_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap mp,
                                                             const __grid_constant__ CUtensorMap ml, int* status,
                                                             long long timeout_ns) {
  constexpr bool VARC = MODE == 1, ADJ = MODE == 2;
  constexpr int RUN = run_rows(MODE), THREADS = threads_of(MODE);
  using G = G2<R, ADJ ? 2 : 1>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage0 + 2 * G::STAGE);

  const int t = threadIdx.x;

  const int nx = a.nx, ny = a.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int ntiles = tiles_x * ((ny + TY - 1) / TY);
  const int c0 = (t % TCOLS) * 4, r0 = (t / TCOLS) * RUN;
  const bool load_d = !a.d_zero;
  const bool kv = a.kappa != nullptr;  // adjoint: varying medium (per-cell kappa)
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
    if (ADJ) tma_load_2d(st + G::PBOX, &ml, gx0 - XH, gy0 - R, &bars[s]);
  };
  int first = blockIdx.x;
  if (t == 0 && first < ntiles) issue(first, 0);
  fused_sample2(a, blockIdx.x, t);  // while the first tile's boxes are in flight

  const float ckh = a.c_lap * a.kappa0, ckl = a.c_lap * a.kappa0_lo;
  float2 w2[R + 1];  // stencil weights, packed
#pragma unroll
  for (int m = 0; m <= R; ++m) w2[m] = dup2(a.w[m]);
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
    // own-cell fields straight into registers, in flight while the boxes land
    float4 d4[RUN], kh4[RUN], kl4[RUN];
#pragma unroll
    for (int rr = 0; rr < RUN; ++rr) {
      const int gy = gy0 + r0 + rr;
      const bool in = gy < ny && gx < nx;
      const long long gi = (long long)gy * nx + gx;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      d4[rr] = (load_d && in) ? ld_stream4(a.dbuf + gi) : z4;
      kh4[rr] = ((VARC || (ADJ && kv && !a.final_step)) && in) ? __ldg(reinterpret_cast<const float4*>(a.kappa + gi))
                                                               : z4;
      kl4[rr] = (VARC && in) ? __ldg(reinterpret_cast<const float4*>(a.kappa_lo + gi)) : z4;
    }
    const bool good = mbar_wait(&bars[s], (k >> 1) & 1, timeout_ns);
    if (__syncthreads_or(!good)) {
      if (t == 0) atomicCAS(status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
      ok = false;
      break;
    }
    const float* P = stage0 + s * G::STAGE;  // P (forward) or Z (adjoint)
    const float* PL = P + G::PBOX;           // adjoint: Z_lo
    // absorbing layer: does the tile reach it (its factors are then loaded row by row)
    const bool layer = SP != 0 && (gx0 < a.sp_w || gx0 + TX > nx - a.sp_w || gy0 < a.sp_w || gy0 + TY > ny - a.sp_w);

    // the tile's update; instantiated separately for tiles inside and outside the layer, so that
    // tiles outside it run exactly the code of the kernel without a layer
    auto update = [&](auto in_layer) {
      constexpr bool LAYER = decltype(in_layer)::value;
      float lo[RUN][4];  // adjoint: the Z_lo part of the stencil, first pass
      if (ADJ) stencil_run<R, RUN, BW, XH>(PL, r0, c0, a.w, lo);
      // sliding window over this thread's 4 columns: win[i] = box row (row - R + i)
      float4 win[2 * R + 1];
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) win[i] = *reinterpret_cast<const float4*>(P + (r0 + i) * BW + XH + c0);
#pragma unroll
      for (int rr = 0; rr < RUN; ++rr) {
        win[2 * R] = *reinterpret_cast<const float4*>(P + (r0 + rr + 2 * R) * BW + XH + c0);
        const int brow = r0 + rr + R;
        float f[20];
        load_row20(P + brow * BW + c0, f);
        const int gy = gy0 + r0 + rr;
        const long long gi = (long long)gy * nx + gx;
        const bool in = gy < ny && gx < nx;
        float dn[4], pn[4], pl[4];
        float4 sa4 = make_float4(1.f, 1.f, 1.f, 1.f), sb4 = sa4;
        if (LAYER && in) {
          sa4 = __ldg(reinterpret_cast<const float4*>(a.sp_a + gi));
          sb4 = __ldg(reinterpret_cast<const float4*>(a.sp_b + gi));
        }
        float4 zl4 = make_float4(0.f, 0.f, 0.f, 0.f);  // adjoint: own Z_lo cells
        if (ADJ) zl4 = *reinterpret_cast<const float4*>(PL + brow * BW + XH + c0);
        // forward: zero-sum pair form (a + b) - 2c per tap; adjoint: difference form on Z
        float st4[4];
        stencil_cells2<R, ADJ>(win, f, w2, st4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float c = f[8 + j];  // own P or Z
          if (!ADJ) {
            const float acc = st4[j];
            const float inc = VARC ? fmaf(a.c_lap * f4get(kh4[rr], j), acc, (a.c_lap * f4get(kl4[rr], j)) * acc)
                                   : fmaf(ckh, acc, ckl * acc);
            if (!LAYER) {
              dn[j] = f4get(d4[rr], j) + inc;
            } else {  // forward in the layer
              const float fa = f4get(sa4, j), fb = f4get(sb4, j);
              dn[j] = load_d ? fmaf(fa, f4get(d4[rr], j), fb * inc) : fmaf(fa - 1.f, c, fb * inc);
            }
            pn[j] = c + dn[j];
            pl[j] = 0.f;
          } else {
            const float acc = st4[j] + lo[rr][j];
            const float g = f4get(d4[rr], j) + a.c_lap * acc;  // G' (S^T r injected into G beforehand)
            const float zl = f4get(zl4, j);
            dn[j] = g;
            if (a.final_step) {
              pn[j] = g;
              if (LAYER) {  // x = G' + ((a-1)/b) Q,  Q = (Z + Z_lo) / kappa
                const float fa = f4get(sa4, j), fb = f4get(sb4, j);
                const float kap = kv ? a.kappa[gi + j] : a.kappa0;
                if (in && fa != 1.f) pn[j] = fmaf((fa - 1.f) / fb, (c + zl) / kap, g);
              }
              pl[j] = 0.f;
            } else {
              const float u = kv ? f4get(kh4[rr], j) * g : fmaf(a.kappa0, g, a.kappa0_lo * g);  // kappa G'
              if (LAYER && (f4get(sa4, j) != 1.f || f4get(sb4, j) != 1.f)) {  // Z' = a Z + b kappa G'
                const float fa = f4get(sa4, j), fb = f4get(sb4, j);
                pn[j] = fmaf(fa, c, fb * u);
                pl[j] = fa * zl;
              } else {
                float e;
                pn[j] = two_sum(c, u, e);
                pl[j] = zl + e;
              }
            }
          }
        }
        if (in) {
          *reinterpret_cast<float4*>(a.next + gi) = make_float4(pn[0], pn[1], pn[2], pn[3]);
          if (!a.final_step) {
            *reinterpret_cast<float4*>(a.dbuf + gi) = make_float4(dn[0], dn[1], dn[2], dn[3]);
            if (ADJ) *reinterpret_cast<float4*>(a.next_lo + gi) = make_float4(pl[0], pl[1], pl[2], pl[3]);
          }
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
    case 3: return kfn<R, 1, 0>();
    case 4: return kfn<R, 1, 1>();
    case 6: return kfn<R, 2, 0>();
    case 8: return kfn<R, 2, 2>();
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
  if (mode == 2) return R == 1 ? G2<1, 2>::SMEM : R == 3 ? G2<3, 2>::SMEM : R == 5 ? G2<5, 2>::SMEM : G2<7, 2>::SMEM;
  return R == 1 ? G2<1>::SMEM : R == 3 ? G2<3>::SMEM : R == 5 ? G2<5>::SMEM : G2<7>::SMEM;
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
  static int cached[3][3][8] = {{{0}}};
  int& c = cached[mode][sp][R];
  if (!c) {
    int dev = 0, sms = 148, per = 1;
    const void* fn = kernel_for(R, mode, sp);
    const size_t smem = smem_for(R, mode);
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads_of(mode), smem) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    c = per * sms;
  }
  const int ntiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  return ntiles < c ? ntiles : c;
}

long long tma2d_threads(int nx, int ny, int R, int mode, int sp) {
  return (long long)tma2d_ctas(nx, ny, R, mode, sp) * threads_of(mode);
}

cudaError_t step2d_tma_launch(int R, int mode, int sp, const StepArgs& a, const CUtensorMap& p, const CUtensorMap& lo,
                              int* status, long long timeout_ns, cudaStream_t st) {
  const void* fn = kernel_for(R, mode, sp);
  if (!fn) return cudaErrorInvalidValue;
  const int nctas = tma2d_ctas(a.nx, a.ny, R, mode, sp);  // sets the kernel's attributes once
  CUtensorMap map = p, mapl = lo;
  StepArgs args = a;
  void* params[] = {&args, &map, &mapl, &status, &timeout_ns};
  return cudaLaunchKernel(fn, dim3(nctas), dim3(threads_of(mode)), params, smem_for(R, mode), st);
}

}  // namespace pat
