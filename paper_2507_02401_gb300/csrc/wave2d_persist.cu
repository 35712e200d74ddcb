// Persistent 2D wave kernel: one cooperative launch runs a whole time loop
// of K (forward) or K* (adjoint) with the wavefield held on chip.
//
// Method (paper Sec. 2, Eq. wave_equation, p_t(0) = 0, pressure zero outside
// the grid): the staggered leapfrog of order 2M, written without the velocity
// as a second-order recurrence in increment form
//
//   forward:  D^1 = kappa/2 L P^0,  D^{n+1} = D^n + kappa L P^n,  P^{n+1} = P^n + D^{n+1},
//             y[s, n] = S_s P^n  (bilinear sensor sampling), n = 0 .. nt-1;
//   adjoint:  G^{nt} = Q^{nt} = 0;  for n = nt-1 .. 1:
//             G^n = G^{n+1} + S^T r_n + L(kappa Q^{n+1}),  Q^n = Q^{n+1} + G^n;
//             x = S^T r_0 + G^1 + 1/2 L(kappa Q^1),
//
// which is the exact transpose of the forward program.  The increment form
// keeps FP32 rounding from being amplified in the low-frequency modes.
//
// GB300 mapping: the grid is cut into 64 x 32 tiles, one CTA per tile, all
// co-resident (cooperative launch).  Each thread keeps its 2 x 4 cells' state
// (P, D, kappa) in registers for the whole loop; the CTA keeps the current
// field plus an R-deep halo in shared memory (double buffered).  After each
// step a CTA publishes only its R-deep boundary strips to an L2-resident
// exchange buffer and bumps a per-tile flag (release); the four neighbours
// wait on that flag (acquire) and copy the strips into their halo.  No
// grid-wide barrier and no per-step launch.  Every wait is bounded by a
// global-timer limit and by a shared abort flag; a CTA that gives up records
// PAT_ERR_TIMEOUT, raises the abort flag and leaves the loop, so the launch
// always ends.
#include <cooperative_groups.h>

#include "internal.h"
#include "stencil.cuh"

namespace pat {
namespace {

constexpr int TX = 64;
constexpr int TY = 32;
constexpr int NTHREADS = (TX / 4) * (TY / 2);  // 256: each thread owns 2 rows x 4 columns
constexpr int XOFF = 8;                         // left halo columns in shared memory (>= R, multiple of 4)
constexpr int PITCH = TX + 16;                  // 8 halo columns each side
static_assert(NTHREADS % 128 == 0, "four halo regions need whole warps");

template <int R>
struct Geo {
  static constexpr int ROWS = TY + 2 * R;
  static constexpr int SBUF = ROWS * PITCH;         // one shared-memory field buffer
  static constexpr int STRIP = 2 * R * (TX + TY);   // floats published per tile per slot
};

// Bounded wait until *flag >= target (wrap-safe).  Executed by a whole warp.
__device__ __forceinline__ bool wait_flag(const int* flag, int target, const int* abort, long long timeout_ns) {
  if (__all_sync(0xffffffffu, (int)(ld_acquire_gpu(flag) - target) >= 0)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (unsigned it = 0; it < (1u << 28); ++it) {
    if (__all_sync(0xffffffffu, (int)(ld_acquire_gpu(flag) - target) >= 0)) return true;
    if ((it & 31u) == 31u) {
      if (ld_relaxed_gpu(abort) != 0) return false;
      if ((long long)(global_timer_ns() - t0) > timeout_ns) return false;
    }
  }
  return false;
}

// Write the thread's 2x4 block of the new state into a shared buffer and the
// boundary strips of the exchange slot X: [top R x TX][bottom R x TX]
// [left TY x R][right TY x R].
template <int R>
__device__ __forceinline__ void store_state(float* Sn, float* X, const float V[2][4], int r0, int c0) {
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int row = r0 + rr;
    const float4 v = make_float4(V[rr][0], V[rr][1], V[rr][2], V[rr][3]);
    *reinterpret_cast<float4*>(Sn + (row + R) * PITCH + XOFF + c0) = v;
    if (row < R) *reinterpret_cast<float4*>(X + row * TX + c0) = v;
    if (row >= TY - R) *reinterpret_cast<float4*>(X + R * TX + (row - (TY - R)) * TX + c0) = v;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + j;
      if (col < R) X[2 * R * TX + row * R + col] = V[rr][j];
      if (col >= TX - R) X[2 * R * TX + TY * R + row * R + (col - (TX - R))] = V[rr][j];
    }
  }
}

template <int R, bool ADJ, bool VARC>
__global__ void __launch_bounds__(NTHREADS, 1) wave2d_persist_kernel(const Persist2DArgs a) {
  using G = Geo<R>;
  extern __shared__ float4 smem4[];
  float* S0 = reinterpret_cast<float*>(smem4);
  float* J = S0 + 2 * G::SBUF;  // adjoint injection accumulator, TY x TX
  __shared__ int s_abort;

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  const int tile = blockIdx.x;
  const int tix = tile % a.tiles_x;
  const int tiy = tile / a.tiles_x;
  const int gx0 = tix * TX, gy0 = tiy * TY;
  const int c0 = (t % (TX / 4)) * 4;
  const int r0 = (t / (TX / 4)) * 2;
  const int nx = a.nx, ny = a.ny, nt = a.nt;

  const unsigned ep = ld_acquire_gpu_u(a.epoch);
  const int base = (int)(ep << 20);

  // halo duty of this warp: 0 = north, 1 = south, 2 = west, 3 = east neighbour
  const int region = warp & 3;
  const int rrank = (warp >> 2) * 32 + lane;
  constexpr int RCOUNT = NTHREADS / 4;
  int nb = -1;
  if (region == 0 && tiy > 0) nb = tile - a.tiles_x;
  if (region == 1 && tiy < a.tiles_y - 1) nb = tile + a.tiles_x;
  if (region == 2 && tix > 0) nb = tile - 1;
  if (region == 3 && tix < a.tiles_x - 1) nb = tile + 1;

  float P[2][4], D[2][4], K[2][4];
  bool valid[2][4];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gx = gx0 + c0 + j, gy = gy0 + r0 + rr;
      const bool v = gx < nx && gy < ny;
      valid[rr][j] = v;
      const long long gi = (long long)gy * nx + gx;
      K[rr][j] = v ? (VARC ? a.kappa[gi] : a.kappa0) : 0.f;
      P[rr][j] = (!ADJ && v) ? a.in[gi] : 0.f;
      D[rr][j] = 0.f;
    }
  for (int i = t; i < 2 * G::SBUF; i += NTHREADS) S0[i] = 0.f;
  if (ADJ)
    for (int i = t; i < TX * TY; i += NTHREADS) J[i] = 0.f;
  if (t == 0) s_abort = 0;
  __syncthreads();

  {  // publish state 0
    float V[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int j = 0; j < 4; ++j) V[rr][j] = ADJ ? K[rr][j] * P[rr][j] : P[rr][j];
    store_state<R>(S0, a.xbuf + (size_t)tile * 2 * G::STRIP, V, r0, c0);
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release_gpu(&a.flags[tile], base);
    }
  }

  for (int k = 0; k < nt; ++k) {
    float* Sc = S0 + (k & 1) * G::SBUF;
    // ---- halo of state k from the neighbours' slot (k & 1)
    if (nb >= 0) {
      if (!wait_flag(&a.flags[nb], base + k, a.abort, a.timeout_ns)) {
        if (lane == 0) {
          s_abort = 1;
          atomicCAS(a.status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
          atomicExch(a.abort, 1);
        }
      } else {
        const float* X = a.xbuf + ((size_t)nb * 2 + (k & 1)) * G::STRIP;
        if (region == 0) {  // north tile's bottom strip -> my rows -R .. -1
          for (int i = rrank; i < R * TX / 4; i += RCOUNT) {
            const int row = i / (TX / 4), cq = (i % (TX / 4)) * 4;
            *reinterpret_cast<float4*>(Sc + row * PITCH + XOFF + cq) =
                __ldcg(reinterpret_cast<const float4*>(X + R * TX + row * TX + cq));
          }
        } else if (region == 1) {  // south tile's top strip -> my rows TY .. TY+R-1
          for (int i = rrank; i < R * TX / 4; i += RCOUNT) {
            const int row = i / (TX / 4), cq = (i % (TX / 4)) * 4;
            *reinterpret_cast<float4*>(Sc + (TY + R + row) * PITCH + XOFF + cq) =
                __ldcg(reinterpret_cast<const float4*>(X + row * TX + cq));
          }
        } else if (region == 2) {  // west tile's right strip -> my columns -R .. -1
          for (int i = rrank; i < TY * R; i += RCOUNT) {
            const int row = i / R, j = i % R;
            Sc[(row + R) * PITCH + XOFF - R + j] = __ldcg(X + 2 * R * TX + TY * R + i);
          }
        } else {  // east tile's left strip -> my columns TX .. TX+R-1
          for (int i = rrank; i < TY * R; i += RCOUNT) {
            const int row = i / R, j = i % R;
            Sc[(row + R) * PITCH + XOFF + TX + j] = __ldcg(X + 2 * R * TX + i);
          }
        }
      }
    }
    if (ADJ) {  // S^T r_n for this tile's injected cells, n = nt-1-k
      const int n = nt - 1 - k;
      const int e1 = a.tile_inj_ptr[tile + 1];
      for (int e = a.tile_inj_ptr[tile] + t; e < e1; e += NTHREADS) {
        const InjCell ic = a.inj[e];
        float s = 0.f;
        for (int q = ic.beg; q < ic.end; ++q) s = fmaf(a.ent_w[q], a.in[(long long)a.ent_sensor[q] * nt + n], s);
        J[ic.local] = s;
      }
    }
    __syncthreads();
    if (s_abort) break;

    if (!ADJ) {  // y[:, k] = S P^k
      const int e1 = a.tile_samp_ptr[tile + 1];
      for (int e = a.tile_samp_ptr[tile] + t; e < e1; e += NTHREADS) {
        const SampEntry se = a.samp[e];
        const float* b = Sc + (se.ly + R) * PITCH + XOFF + se.lx;
        const float v = se.w[0] * b[0] + se.w[1] * b[1] + se.w[2] * b[PITCH] + se.w[3] * b[PITCH + 1];
        a.out[(long long)se.sensor * nt + k] = v;
      }
    }

    float L[2][4];
    lap_2x4<R>(Sc, PITCH, r0 + R, XOFF + c0, a.w, L);

    if (k == nt - 1) {
      if (ADJ) {  // x = S^T r_0 + G^1 + 1/2 L(kappa Q^1)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (!valid[rr][j]) continue;
            const int lr = r0 + rr, lc = c0 + j;
            const float xv = J[lr * TX + lc] + D[rr][j] + 0.5f * L[rr][j];
            a.out[(long long)(gy0 + lr) * nx + gx0 + lc] = xv;
          }
      }
      break;
    }

    float V[2][4];
    if (!ADJ) {
      const float cf = (k == 0) ? 0.5f : 1.0f;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          D[rr][j] = fmaf(cf * K[rr][j], L[rr][j], D[rr][j]);
          P[rr][j] += D[rr][j];
          V[rr][j] = P[rr][j];
        }
    } else {
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int li = (r0 + rr) * TX + c0 + j;
          const float g = valid[rr][j] ? (D[rr][j] + J[li]) + L[rr][j] : 0.f;
          J[li] = 0.f;
          D[rr][j] = g;
          P[rr][j] = valid[rr][j] ? P[rr][j] + g : 0.f;
          V[rr][j] = K[rr][j] * P[rr][j];
        }
    }
    store_state<R>(S0 + ((k + 1) & 1) * G::SBUF, a.xbuf + ((size_t)tile * 2 + ((k + 1) & 1)) * G::STRIP, V, r0,
                   c0);
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release_gpu(&a.flags[tile], base + k + 1);
    }
  }

  // launch accounting: the last CTA to finish advances the epoch and clears abort
  __syncthreads();
  if (t == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(a.done, 1u);
    if (prev == gridDim.x - 1) {
      *a.done = 0u;
      atomicExch(a.abort, 0);
      __threadfence();
      atomicAdd(a.epoch, 1u);
    }
  }
}

template <int R, bool ADJ, bool VARC>
constexpr void* kfn() {
  return (void*)wave2d_persist_kernel<R, ADJ, VARC>;
}

void* pick(int R, bool adj, bool varc) {
#define PAT_P2D(RR)                                                           \
  if (R == RR) {                                                              \
    if (adj) return varc ? kfn<RR, true, true>() : kfn<RR, true, false>();    \
    return varc ? kfn<RR, false, true>() : kfn<RR, false, false>();           \
  }
  PAT_P2D(1)
  PAT_P2D(3)
  PAT_P2D(5)
  PAT_P2D(7)
#undef PAT_P2D
  return nullptr;
}

size_t smem_bytes(int R, bool adj) {
  const size_t sbuf = (size_t)(TY + 2 * R) * PITCH;
  return (2 * sbuf + (adj ? (size_t)TX * TY : 0)) * sizeof(float);
}

}  // namespace

bool persist2d_supported(int R, bool) { return R == 1 || R == 3 || R == 5 || R == 7; }
int persist2d_tile_x() { return TX; }
int persist2d_tile_y() { return TY; }
size_t persist2d_smem_bytes(int R, bool adj) { return smem_bytes(R, adj); }

int persist2d_max_ctas(int R, bool adj, bool varc) {
  void* f = pick(R, adj, varc);
  if (!f) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, NTHREADS, smem_bytes(R, adj)) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

cudaError_t persist2d_launch(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st) {
  void* f = pick(R, adj, varc);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(f, dim3(nctas), dim3(NTHREADS), args, smem_bytes(R, adj), st);
}

}  // namespace pat
