// 3D wave step with TMA-fed plane pipelines (constant medium, the HBM-bound
// volumes): one launch per time step of the three-level recurrence
//
//   next = c_cur cur - c_prev prev + c_lap (kappa_hi + kappa_lo) L cur
//
// (paper Sec. 2, Eq. wave_equation; forward P^{n+1} = 2P^n - P^{n-1} +
// kappa L P^n and, because kappa is constant, the adjoint
// Q^n = 2Q^{n+1} - Q^{n+2} + kappa L Q^{n+1} have the same form).
//
// A CTA owns a 64 x 16 column of cells and marches through a range of z
// planes.  One thread issues TMA loads of each plane of `cur` as an
// (64+16) x (16+2R) box (x/y halo included, zero outside the grid) into a
// ring of shared-memory slots, PD planes ahead of the plane being computed,
// plus the own 64 x 16 tile of `prev`; completion is tracked by one mbarrier
// per slot.  Each thread owns 2 rows x 4 columns: x/y neighbours come from the
// centre plane's slot, z neighbours from a register ring of 2R+1 planes.
// Compulsory DRAM traffic per point-update: cur and prev read once, next
// written once (12 B); halo re-reads are served by L2.
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "internal.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace pat {
namespace {

constexpr int TX = 64, TY = 16, THREADS = (TX / 4) * (TY / 2);  // 128
constexpr int XH = 8;            // box columns left of the tile (>= R, 16-byte aligned)
constexpr int BW = TX + 2 * XH;  // box width, 80 floats
constexpr int PD = 2;            // prefetch distance in planes

template <int R>
struct G3 {
  static constexpr int BH = TY + 2 * R;
  static constexpr int PLANE = BW * BH;  // floats per cur slot (multiple of 32: 128-byte aligned slots)
  static constexpr int NS = R + 1 + PD;  // cur slots: centre plane .. queue plane + PD
  static constexpr int PREV = TX * TY;   // floats per prev slot
  static constexpr int NSP = PD + 1;
  static constexpr size_t SMEM = sizeof(float) * ((size_t)NS * PLANE + (size_t)NSP * PREV) + 8 * (NS + NSP);
};

// Sensor s = b + t * gridDim.x is sampled by thread t of CTA b: the sensors are spread over every CTA
// of the wave (a few per CTA) instead of loading the first CTAs with all of them.
__device__ __forceinline__ void fused_sample3(const StepArgs& a, long long bid, int t) {
  const long long gs = bid + (long long)t * gridDim.x;
  if (a.y == nullptr || gs >= a.ns) return;
  const int s = (int)gs;
  float v = 0.f;
  for (int k = 0; k < a.corners; ++k) v = fmaf(a.sens_w[s * a.corners + k], a.cur[a.sens_cell[s * a.corners + k]], v);
  a.y[(long long)s * a.nt + a.t_sample] = v;
}

// Runs f(S, i + S) for S = 0 .. Q-1 while i + S < n (S a compile-time constant in each call); false as
// soon as one call returns false.
template <int S, int Q, class F>
__device__ __forceinline__ bool march(F& f, int i, int n) {
  if constexpr (S == Q) {
    return true;
  } else {
    if (i + S >= n) return true;
    if (!f(std::integral_constant<int, S>{}, i + S)) return false;
    return march<S + 1, Q>(f, i, n);
  }
}

// The adjoint's injection S^T r_m into one cell: sum of w r_m over the cell's sensor entries.
__device__ __forceinline__ float inj_sum(const StepArgs& a, const InjCell& c) {
  float v = 0.f;
  for (int q = c.beg; q < c.end; ++q) v = fmaf(a.ent_w[q], a.inj_r[(long long)a.ent_sensor[q] * a.nt + a.inj_t], v);
  return v;
}

// INJ: the adjoint's injection S^T r_m into the CTA's own cells of `next` after the step (per-CTA lists)
// Work split (column-fastest): CTA b takes column b mod columns and the (b div columns)-th of
// nchunks equal z ranges, so CTAs that run together stream neighbouring columns of the same rows.
template <int R, bool INJ, bool RING>
__global__ void __launch_bounds__(THREADS) step3d_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap mcur,
                                                             const __grid_constant__ CUtensorMap mprev, int cols_x,
                                                             int nchunks, int* status, long long timeout_ns) {
  using G = G3<R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* pring = ring + G::NS * G::PLANE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(pring + G::NSP * G::PREV);
  uint64_t* pbars = bars + G::NS;

  const int t = threadIdx.x;
  const long long bid = blockIdx.x;

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  const int c0 = (t % (TX / 4)) * 4, r0 = (t / (TX / 4)) * 2;
  const long long ncols = (long long)cols_x * ((ny + TY - 1) / TY);
  const bool has_prev = a.prev != nullptr;
  const float ck = a.c_lap * a.kappa0, ckl = a.c_lap * a.kappa0_lo;
  const float2 ck2 = dup2(ck), ckl2 = dup2(ckl), ccur2 = dup2(a.c_cur), ncprev2 = dup2(-a.c_prev), m2 = dup2(-2.f);
  float2 w2[R + 1];
#pragma unroll
  for (int m = 0; m <= R; ++m) w2[m] = dup2(a.w[m]);

  bool ok_all = true;
  int issued = 0;       // cur planes issued (thread 0)
  int issued_prev = 0;  // prev planes issued
  const int col = (int)(bid % ncols);
  const long long zr = bid / ncols;
  const int z0 = (int)(zr * nz / nchunks);
  const int z1 = (int)((zr + 1) * nz / nchunks);
  const int gx0 = (col % cols_x) * TX, gy0 = (col / cols_x) * TY;
  const int nloc = z1 - z0;   // planes computed
  const int ncur = nloc + R;  // cur planes j = 0 .. ncur-1 (z = z0 + j) go through the ring
  if (t == 0) {
    for (int s = 0; s < G::NS + G::NSP; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue_cur = [&](int j) {
    issued = j + 1;
    const int s = j % G::NS;
    mbar_expect_tx(&bars[s], G::PLANE * 4);
    tma_load_3d(ring + s * G::PLANE, &mcur, gx0 - XH, gy0 - R, z0 + j, &bars[s]);
  };
  auto issue_prev = [&](int j) {
    issued_prev = j + 1;
    const int s = j % G::NSP;
    mbar_expect_tx(&pbars[s], G::PREV * 4);
    tma_load_3d(pring + s * G::PREV, &mprev, gx0, gy0, z0 + j, &pbars[s]);
  };
  if (t == 0) {
    for (int j = 0; j < min(R + PD, ncur); ++j) issue_cur(j);
    if (has_prev)
      for (int j = 0; j < min(PD, nloc); ++j) issue_prev(j);
  }
  fused_sample3(a, bid, t);  // the forward's sensor samples of cur, while the first copies are in flight

  // register ring of the own cells: at the first plane q[k] = plane z0 - R + k
  float4 q[2 * R + 1][2];
#pragma unroll
  for (int i = 0; i < R; ++i)  // planes z0-R .. z0-1 straight from global memory
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int z = z0 - R + i, gy = gy0 + r0 + rr, gx = gx0 + c0;
      q[i][rr] = (z >= 0 && gy < ny && gx < nx)
                     ? __ldg(reinterpret_cast<const float4*>(a.cur + z * plane + (long long)gy * nx + gx))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < R; ++i) {  // planes z0 .. z0+R-1 from the ring
    ok = ok && (i >= ncur || mbar_wait(&bars[i % G::NS], (i / G::NS) & 1, timeout_ns));
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
      q[R + i][rr] = *reinterpret_cast<const float4*>(ring + (i % G::NS) * G::PLANE + (r0 + rr + R) * BW + XH + c0);
  }

  // One plane of the march.  RING: the z queue is a ring in registers, logical entry k (plane z - R + k)
  // of plane i sitting in q[(k + i) % Q]; the loop is unrolled Q times, so S = i % Q is a compile-time
  // constant in every copy and no queue entry moves between registers (fewer instructions, a Q times
  // larger loop body).  Otherwise S = 0 and the queue shifts after every plane.
  constexpr int Q = 2 * R + 1;
  auto step = [&](auto sc, int i) -> bool {
    constexpr int S = decltype(sc)::value;
    if (t == 0) {
      fence_proxy_async_shared();  // the slots refilled below were last read through the generic proxy
      if (i + R + PD < ncur) issue_cur(i + R + PD);
      if (has_prev && i + PD < nloc) issue_prev(i + PD);
    }
    const int jq = i + R;  // queue plane
    bool good = ok && mbar_wait(&bars[jq % G::NS], (jq / G::NS) & 1, timeout_ns);
    if (has_prev) good = good && mbar_wait(&pbars[i % G::NSP], (i / G::NSP) & 1, timeout_ns);
    if (__syncthreads_or(!good)) {
      if (t == 0) atomicCAS(status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
      return false;
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
      q[(2 * R + S) % Q][rr] =
          *reinterpret_cast<const float4*>(ring + (jq % G::NS) * G::PLANE + (r0 + rr + R) * BW + XH + c0);

    const float* cen = ring + (i % G::NS) * G::PLANE;
    float2 L[2][2];  // packed pairs: cells (2p, 2p+1) of row rr
    lap_2x4_x2<R>(cen, BW, r0 + R, XH + c0, w2, L);
    const int z = z0 + i;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const float4 pv = has_prev ? *reinterpret_cast<const float4*>(pring + (i % G::NSP) * G::PREV + (r0 + rr) * TX + c0)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      float2 out[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const float2 c = p ? hi2(q[(R + S) % Q][rr]) : lo2(q[(R + S) % Q][rr]);
        float2 acc = L[rr][p];
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          const float2 up = p ? hi2(q[(R + m + S) % Q][rr]) : lo2(q[(R + m + S) % Q][rr]);
          const float2 dn = p ? hi2(q[(R - m + S) % Q][rr]) : lo2(q[(R - m + S) % Q][rr]);
          acc = __ffma2_rn(w2[m], __ffma2_rn(c, m2, __fadd2_rn(up, dn)), acc);
        }
        // c_cur c - c_prev prev + (ck + ckl) acc, the last product rounded once
        float2 v = __fmul2_rn(ccur2, c);
        if (has_prev) v = __ffma2_rn(ncprev2, p ? hi2(pv) : lo2(pv), v);
        out[p] = __fadd2_rn(v, __ffma2_rn(ck2, acc, __fmul2_rn(ckl2, acc)));
      }
      const int gy = gy0 + r0 + rr, gx = gx0 + c0;
      if (gy < ny && gx < nx)
        *reinterpret_cast<float4*>(a.next + z * plane + (long long)gy * nx + gx) =
            make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
    }
    __syncthreads();  // the centre slot is refilled by the next step's TMA
    return true;
  };
  if constexpr (RING) {
    for (int i = 0; i < nloc; i += Q)
      if (!march<0, Q>(step, i, nloc)) {
        ok_all = false;
        break;
      }
  } else {  // the queue shifts by one plane after every step (one copy of the loop body)
    for (int i = 0; i < nloc; ++i) {
      if (!step(std::integral_constant<int, 0>{}, i)) {
        ok_all = false;
        break;
      }
#pragma unroll
      for (int k = 0; k < 2 * R; ++k) {
        q[k][0] = q[k + 1][0];
        q[k][1] = q[k + 1][1];
      }
    }
  }
  if (INJ && ok_all) {  // every thread's stores to `next` precede the injection (same CTA)
    __syncthreads();
    for (int e = a.inj_tile_ptr[bid] + t; e < a.inj_tile_ptr[bid + 1]; e += THREADS)
      a.next[a.inj_tile[e].local] += inj_sum(a, a.inj_tile[e]);
  }
  // after a timed-out wait: give the copies still in flight (the last one of
  // each slot) a bounded chance to land before the CTA's shared memory goes away
  if (t == 0 && !ok_all) {
    for (int j = max(0, issued - G::NS); j < issued; ++j) mbar_wait(&bars[j % G::NS], (j / G::NS) & 1, timeout_ns);
    for (int j = max(0, issued_prev - G::NSP); j < issued_prev; ++j)
      mbar_wait(&pbars[j % G::NSP], (j / G::NSP) & 1, timeout_ns);
  }
}

template <int R, bool INJ, bool RING>
cudaError_t prepare_r() {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(step3d_tma_kernel<R, INJ, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G3<R>::SMEM);
  });
  return attr_err;
}

template <int R, bool INJ, bool RING>
cudaError_t launch_r(const StepArgs& a, const CUtensorMap& mc, const CUtensorMap& mp, int nctas, int nchunks,
                     int* status, long long timeout_ns, cudaStream_t st) {
  const cudaError_t attr_err = prepare_r<R, INJ, RING>();
  if (attr_err != cudaSuccess) return attr_err;
  step3d_tma_kernel<R, INJ, RING><<<nctas, THREADS, G3<R>::SMEM, st>>>(a, mc, mp, (a.nx + TX - 1) / TX, nchunks,
                                                                        status, timeout_ns);
  return cudaGetLastError();
}

template <int R, bool INJ, bool RING>
int blocks_per_sm() {
  int per = 0;
  if (prepare_r<R, INJ, RING>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step3d_tma_kernel<R, INJ, RING>, THREADS, G3<R>::SMEM) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per;
}

// Co-resident CTAs of the step kernel (every variant) on the current device.
template <int R>
int resident_r() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int v[4] = {blocks_per_sm<R, false, false>(), blocks_per_sm<R, true, false>(), blocks_per_sm<R, false, true>(),
                    blocks_per_sm<R, true, true>()};
  int per = v[0];
  for (int i = 1; i < 4; ++i) per = v[i] < per ? v[i] : per;
  return sms * per;
}

template <bool INJ, bool RING>
cudaError_t launch_i(int R, const StepArgs& a, const CUtensorMap& cur, const CUtensorMap& prev, int nctas,
                     int nchunks, int* status, long long timeout_ns, cudaStream_t st) {
  switch (R) {
    case 1: return launch_r<1, INJ, RING>(a, cur, prev, nctas, nchunks, status, timeout_ns, st);
    case 3: return launch_r<3, INJ, RING>(a, cur, prev, nctas, nchunks, status, timeout_ns, st);
    case 5: return launch_r<5, INJ, RING>(a, cur, prev, nctas, nchunks, status, timeout_ns, st);
    case 7: return launch_r<7, INJ, RING>(a, cur, prev, nctas, nchunks, status, timeout_ns, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link);
// nullptr when the driver does not provide it.
void* tma_encoder_raw() {
  static void* fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = p;
    else
      cudaGetLastError();
  });
  return fn;
}


bool tma3d_supported(int nx, int R, bool varc) { return !varc && nx % 4 == 0 && (R == 1 || R == 3 || R == 5 || R == 7); }

// Descriptors of a 3D field: `cur` boxes (80 x (16+2R) x 1) and `prev` boxes (64 x 16 x 1).
cudaError_t tma3d_encode(const float* base, int nx, int ny, int nz, int R, CUtensorMap* cur, CUtensorMap* prev) {
  auto fn = tma_encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_c[3] = {(cuuint32_t)BW, (cuuint32_t)(TY + 2 * R), 1};
  const cuuint32_t box_p[3] = {(cuuint32_t)TX, (cuuint32_t)TY, 1};
  CUresult r1 = fn(cur, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box_c, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = fn(prev, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box_p, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
}

// Work split of a step launch: columns (64 x 16 cells) x nchunks equal z ranges, column-fastest.  Few
// columns (fewer than a quarter of the co-resident CTAs; 64 at 256^3): as many z ranges as keep every
// CTA in one wave (9 at 256^3: 576 CTAs of 28-29 planes), so no second wave leaves SMs idle at the end
// of a step.  Many columns (256 at 512^3): ranges of at least 16 planes, doubled while the grid keeps
// >= 6 CTAs per SM.  Measured at 256^3: 41.0 / 40.0 us per K / K* step against 41.4 / 44.1 us with
// 16-plane ranges in 1024 CTAs (and 43.1 / 42.3 us with equal z-fastest shares of the (column, plane)
// work, whose concurrent CTAs no longer share x/y halos through L2).
Tma3dSplit tma3d_split(int R, int nx, int ny, int nz) {
  int cap = 0;
  switch (R) {
    case 1: cap = resident_r<1>(); break;
    case 3: cap = resident_r<3>(); break;
    case 5: cap = resident_r<5>(); break;
    case 7: cap = resident_r<7>(); break;
    default: return Tma3dSplit{0, 0};
  }
  if (cap <= 0) return Tma3dSplit{0, 0};
  const long long cols = (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  int chunks;
  if (cols * 4 < cap) {
    chunks = (int)(cap / cols);
  } else {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int zc = 16;
    while (zc < nz && cols * ((nz + zc * 2 - 1) / (zc * 2)) >= 6LL * sms) zc *= 2;
    chunks = (nz + zc - 1) / zc;
  }
  if (chunks > nz) chunks = nz;
  // the register-ring march saves the queue's register moves where issue is the bound (one-wave grids:
  // 38.7 / 40.3 us against 39.4 / 41.2 per K / K* step at 256^3), but its larger body costs where DRAM is
  // (many columns: 274.5 / 278.7 us against 264.8 / 268.9 at 512^3)
  return Tma3dSplit{(int)(cols * chunks), chunks, cols * 4 < cap};
}

// CTA holding cell (x, y, z) (the kernel's split: chunk zr holds z in [zr nz / k, (zr + 1) nz / k)).
int tma3d_cta_of(int nx, int ny, int nz, const Tma3dSplit& sp, int x, int y, int z) {
  const long long cols_x = (nx + TX - 1) / TX;
  const long long ncols = cols_x * ((ny + TY - 1) / TY);
  const long long col = (long long)(y / TY) * cols_x + x / TX;
  long long zr = (long long)z * sp.nchunks / nz;
  while (zr + 1 < sp.nchunks && (zr + 1) * nz / sp.nchunks <= z) ++zr;
  while (zr > 0 && zr * nz / sp.nchunks > z) --zr;
  return (int)(zr * ncols + col);
}

long long tma3d_threads(int nctas) { return (long long)nctas * THREADS; }

cudaError_t step3d_tma_launch(int R, const StepArgs& a, const CUtensorMap& cur, const CUtensorMap& prev,
                              const Tma3dSplit& sp, int* status, long long timeout_ns, cudaStream_t st) {
  if (sp.ring)
    return a.inj_r ? launch_i<true, true>(R, a, cur, prev, sp.nctas, sp.nchunks, status, timeout_ns, st)
                   : launch_i<false, true>(R, a, cur, prev, sp.nctas, sp.nchunks, status, timeout_ns, st);
  return a.inj_r ? launch_i<true, false>(R, a, cur, prev, sp.nctas, sp.nchunks, status, timeout_ns, st)
                 : launch_i<false, false>(R, a, cur, prev, sp.nctas, sp.nchunks, status, timeout_ns, st);
}

}  // namespace pat
