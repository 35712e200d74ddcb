// Periodic orthonormal Daubechies DWT levels with fused level scaling
// (paper Sec. 4: the fast wavelet transform W, W^{-1} = W^T, and the diagonal
// scaling D of the detail blocks, Prop. 4.2).
//
// One analysis level along an axis of even length n with filters h, g
// (g_j = (-1)^j h_{L-1-j}):
//   a_k = sum_j h_j x[(2k+j) mod n],  d_k = sum_j g_j x[(2k+j) mod n];
// synthesis is the transpose: x[(2k+j) mod n] += h_j a_k + g_j d_k.
//
// 2D levels are fused: one CTA stages a periodic input window in shared
// memory, filters along x, then along y, and writes the four bands (details
// times the level weight).  Levels whose width is a multiple of 8 take the
// HBM-rate kernels (16-byte cp.async staging with the periodic wrap computed
// per 16-byte chunk, float4 band stores); narrower levels take the generic
// kernels.  3D levels with width a multiple of 8 run as one fused pass
// (x/y in shared memory, z in registers while marching through z, or all
// planes of an output plane at once on levels that fit one wave of CTAs);
// other 3D levels run as separable 1D passes.
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "stencil.cuh"
#include "tma.cuh"

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


// ------------------------------------------- 2D levels at HBM rate (nx % 8 == 0)
// 16-byte asynchronous copy global -> shared, cached in L2 only
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


// Four consecutive values as two packed FP32x2 pairs (FFMA2 / FMUL2: one
// instruction per pair, each lane rounded as the scalar instruction would).
struct F4x2 {
  float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
  __device__ __forceinline__ static F4x2 ld(const float* s) {
    const float4 v = *reinterpret_cast<const float4*>(s);
    F4x2 r;
    r.p0 = make_float2(v.x, v.y);
    r.p1 = make_float2(v.z, v.w);
    return r;
  }
  __device__ __forceinline__ void fma(float2 w, const F4x2& v) {
    p0 = __ffma2_rn(w, v.p0, p0);
    p1 = __ffma2_rn(w, v.p1, p1);
  }
  __device__ __forceinline__ F4x2 scale(float2 w) const {
    F4x2 r;
    r.p0 = __fmul2_rn(w, p0);
    r.p1 = __fmul2_rn(w, p1);
    return r;
  }
  __device__ __forceinline__ float4 f4() const { return make_float4(p0.x, p0.y, p1.x, p1.y); }
  __device__ __forceinline__ void st(float* d) const { *reinterpret_cast<float4*>(d) = f4(); }
};

// Programmatic dependent launch: a level's grid may start while the previous
// level's grid drains; griddepcontrol.wait (before any read of the previous
// level's output) blocks until that grid has completed and its writes are
// visible.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Row stride of a staged 3D window: an odd number of 16-byte units.  The x
// pass has each thread read 16 bytes every 32 bytes of a row, a warp spanning
// four rows; with an even stride every row of the warp starts on the same
// bank and each 16-byte load takes twice the minimum shared-memory wavefronts.
__host__ __device__ constexpr int pad_row(int w) { return (w / 4) % 2 == 0 ? w + 4 : w; }

// Analysis: tile (kx0, ky0) gives OX x OY coefficients of each band from the
// input window rows [2 ky0, 2 ky0 + 2 OY + L - 2) x columns [2 kx0, 2 kx0 +
// 2 OX + HX) (periodic).  Persistent CTAs walk the tiles, staging the next
// tile's window (cp.async, second buffer) while filtering the current one.
template <int L>
struct A2F {
  static constexpr int OX = 64, OY = 16, THREADS = 256;
  static constexpr int HX = (L - 2 + 3) / 4 * 4;  // right halo, rounded up to whole float4
  static constexpr int WX = 2 * OX + HX;
  static constexpr int WY = 2 * OY + L - 2;
  static constexpr int NQ = WX / 4;
  static constexpr int NCH = (WY * NQ + THREADS - 1) / THREADS;  // 16-byte chunks per thread and window
  static constexpr int WIN = WY * WX;  // floats per window buffer (multiple of 4)
  static constexpr int LOHI = WY * OX;
  static constexpr int SMEM = (2 * WIN + 2 * LOHI) * 4;
};

template <int L>
__global__ void __launch_bounds__(256) dwt2d_analysis_fast_kernel(const float* __restrict__ in, int nx, int ny,
                                                                  float* __restrict__ A, float* __restrict__ Hb,
                                                                  float* __restrict__ Vb, float* __restrict__ Db,
                                                                  float wdet, const Filt f, int tiles_x,
                                                                  int ntiles) {
  using G = A2F<L>;
  extern __shared__ __align__(16) unsigned char dsm[];
  float* win0 = reinterpret_cast<float*>(dsm);          // two window buffers
  auto lo = reinterpret_cast<float(*)[G::OX]>(win0 + 2 * G::WIN);
  auto hi = reinterpret_cast<float(*)[G::OX]>(win0 + 2 * G::WIN + G::LOHI);
  const int t = threadIdx.x;
  griddep_wait();
  griddep_trigger();
  // this thread's 16-byte chunks of a window: shared offset and (interior windows) source offset from the
  // window corner are the same for every tile, so they are computed once
  int soff[G::NCH], roff[G::NCH];
#pragma unroll
  for (int c = 0; c < G::NCH; ++c) {
    const int i = t + c * G::THREADS;
    const int r = i / G::NQ, q = i - r * G::NQ;
    soff[c] = i < G::WY * G::NQ ? r * G::WX + 4 * q : -1;
    roff[c] = r * nx + 4 * q;
  }
  auto stage = [&](int tile, float* w) {
    const int kx0 = (tile % tiles_x) * G::OX, ky0 = (tile / tiles_x) * G::OY;
    if (2 * kx0 + G::WX <= nx && 2 * ky0 + G::WY <= ny) {  // interior window: no wrap
      const float* src = in + (long long)(2 * ky0) * nx + 2 * kx0;
#pragma unroll
      for (int c = 0; c < G::NCH; ++c)
        if (soff[c] >= 0) cp_async16(w + soff[c], src + roff[c]);
    } else {
      for (int i = t; i < G::WY * G::NQ; i += G::THREADS) {
        const int r = i / G::NQ, q = i - r * G::NQ;
        const int gy = (2 * ky0 + r) % ny, gx = (2 * kx0 + 4 * q) % nx;  // nx % 4 == 0: a chunk never straddles
        cp_async16(w + r * G::WX + 4 * q, in + (long long)gy * nx + gx);  // the wrap
      }
    }
  };
  int tile = blockIdx.x;
  if (tile < ntiles) stage(tile, win0);
  cp_async_commit();
  const int qx = t % (G::OX / 4), ky = t / (G::OX / 4);
  const int nx2 = nx >> 1, ny2 = ny >> 1;
  const float2 w2 = dup2(wdet);
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) stage(nxt, win0 + ((k + 1) & 1) * G::WIN);  // read two barriers ago: free
    cp_async_commit();
    cp_async_wait_group<1>();  // this tile's window has landed (this thread's copies)
    __syncthreads();           // ... and every thread's
    const float(*win)[G::WX] = reinterpret_cast<const float(*)[G::WX]>(win0 + (k & 1) * G::WIN);
    // along x: outputs 4q .. 4q+3 of window row r read window columns 8q .. 8q + 6 + L - 1
    for (int i = t; i < G::WY * (G::OX / 4); i += G::THREADS) {
      const int r = i / (G::OX / 4), q = i % (G::OX / 4);
      float v[8 + G::HX];
#pragma unroll
      for (int c = 0; c < (8 + G::HX) / 4; ++c) {
        const float4 w4 = *reinterpret_cast<const float4*>(&win[r][8 * q + 4 * c]);
        v[4 * c] = w4.x;
        v[4 * c + 1] = w4.y;
        v[4 * c + 2] = w4.z;
        v[4 * c + 3] = w4.w;
      }
      float sl[4], sh[4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        sl[kk] = 0.f;
        sh[kk] = 0.f;
#pragma unroll
        for (int j = 0; j < L; ++j) {
          sl[kk] = fmaf(f.h[j], v[2 * kk + j], sl[kk]);
          sh[kk] = fmaf(f.g[j], v[2 * kk + j], sh[kk]);
        }
      }
      *reinterpret_cast<float4*>(&lo[r][4 * q]) = make_float4(sl[0], sl[1], sl[2], sl[3]);
      *reinterpret_cast<float4*>(&hi[r][4 * q]) = make_float4(sh[0], sh[1], sh[2], sh[3]);
    }
    __syncthreads();
    // along y: 4 consecutive coefficients of one output row per thread
    F4x2 a, hh, vv, dd;  // packed pairs (columns 0-1, 2-3)
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const F4x2 l = F4x2::ld(&lo[2 * ky + j][4 * qx]);
      const F4x2 h = F4x2::ld(&hi[2 * ky + j][4 * qx]);
      const float2 hj = dup2(f.h[j]), gj = dup2(f.g[j]);
      a.fma(hj, l);
      hh.fma(gj, l);  // x low, y high
      vv.fma(hj, h);  // x high, y low
      dd.fma(gj, h);
    }
    const int oy = (tile / tiles_x) * G::OY + ky, ox = (tile % tiles_x) * G::OX + 4 * qx;
    if (oy < ny2 && ox < nx2) {  // nx2 % 4 == 0: the four coefficients are all in or all out
      const long long o = (long long)oy * nx2 + ox;
      a.st(A + o);
      hh.scale(w2).st(Hb + o);
      vv.scale(w2).st(Vb + o);
      dd.scale(w2).st(Db + o);
    }
  }
}

// Synthesis: tile (kx0, ky0) gives the 2 OX x 2 OY pixels of coefficient block
// (kx0 .. kx0+OX-1, ky0 .. ky0+OY-1) from the coefficient window rows
// [ky0 - LH, ky0 + OY) x columns [kx0 - CX, kx0 + OX) of each band
// (periodic); persistent CTAs, next window staged while filtering.
template <int L>
struct S2F {
  static constexpr int OX = 64, OY = 16, THREADS = 256;
  static constexpr int LH = L / 2 - 1;             // coefficients left of / above the block that reach it
  static constexpr int CX = (LH + 3) / 4 * 4;      // left halo, rounded up to whole float4
  static constexpr int WX = OX + CX;
  static constexpr int WY = OY + LH;
  static constexpr int NQ = WX / 4;
  static constexpr int K0 = (CX - LH) & ~1;        // first (even) window column a pixel quad reads
  static constexpr int NK2 = (CX + 2 - K0) / 2;    // float2 loads per pixel quad
  static constexpr int NCH = (4 * WY * NQ + THREADS - 1) / THREADS;  // 16-byte chunks per thread and window
  static constexpr int WIN = 4 * WY * WX;          // floats per window buffer (four bands)
  static constexpr int LOHI = 2 * OY * WX;
  static constexpr int SMEM = (2 * WIN + 2 * LOHI) * 4;
};

template <int L>
__global__ void __launch_bounds__(256, 4) dwt2d_synthesis_fast_kernel(const float* __restrict__ A,
                                                                   const float* __restrict__ Hb,
                                                                   const float* __restrict__ Vb,
                                                                   const float* __restrict__ Db, float wdet, int nx,
                                                                   int ny, float* __restrict__ out, const Filt f,
                                                                   int tiles_x, int ntiles) {
  using G = S2F<L>;
  extern __shared__ __align__(16) unsigned char dsm[];
  float* cw0 = reinterpret_cast<float*>(dsm);  // two window buffers [4][WY][WX]
  auto lo = reinterpret_cast<float(*)[G::WX]>(cw0 + 2 * G::WIN);
  auto hi = reinterpret_cast<float(*)[G::WX]>(cw0 + 2 * G::WIN + G::LOHI);
  const int t = threadIdx.x;
  const int nx2 = nx >> 1, ny2 = ny >> 1;
  griddep_wait();
  griddep_trigger();
  // this thread's 16-byte chunks of the four band windows: shared offset, and band (bits 28-29) with source
  // offset from the window corner (interior windows), the same for every tile, so computed once
  int soff[G::NCH], code[G::NCH];
#pragma unroll
  for (int c = 0; c < G::NCH; ++c) {
    const int i = t + c * G::THREADS;
    const int b = i / (G::WY * G::NQ), rq = i - b * (G::WY * G::NQ);
    const int r = rq / G::NQ, q = rq - r * G::NQ;
    soff[c] = i < 4 * G::WY * G::NQ ? (b * G::WY + r) * G::WX + 4 * q : -1;
    code[c] = (b << 28) | (r * nx2 + 4 * q);
  }
  auto stage = [&](int tile, float* w) {
    const int kx0 = (tile % tiles_x) * G::OX, ky0 = (tile / tiles_x) * G::OY;
    const bool interior = kx0 >= G::CX && ky0 >= G::LH && kx0 + G::OX <= nx2 && ky0 + G::OY <= ny2;
    if (interior) {
      const long long corner = (long long)(ky0 - G::LH) * nx2 + kx0 - G::CX;
#pragma unroll
      for (int c = 0; c < G::NCH; ++c) {
        if (soff[c] < 0) continue;
        const int b = code[c] >> 28;
        const float* src = b == 0 ? A : (b == 1 ? Hb : (b == 2 ? Vb : Db));
        cp_async16(w + soff[c], src + corner + (code[c] & 0x0fffffff));
      }
      return;
    }
    for (int i = t; i < 4 * G::WY * G::NQ; i += G::THREADS) {
      const int b = i / (G::WY * G::NQ), rq = i - b * (G::WY * G::NQ);
      const int r = rq / G::NQ, q = rq - r * G::NQ;
      // periodic (a coarse level may be shorter than the halo: wrap repeatedly); nx2 % 4 == 0
      const int ky = pmod(ky0 - G::LH + r, ny2);
      const int kx = pmod(kx0 - G::CX + 4 * q, nx2);
      const float* src = b == 0 ? A : (b == 1 ? Hb : (b == 2 ? Vb : Db));
      cp_async16(w + (b * G::WY + r) * G::WX + 4 * q, src + (long long)ky * nx2 + kx);
    }
  };
  int tile = blockIdx.x;
  if (tile < ntiles) stage(tile, cw0);
  cp_async_commit();
  const float2 w2 = dup2(wdet);
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) stage(nxt, cw0 + ((k + 1) & 1) * G::WIN);
    cp_async_commit();
    cp_async_wait_group<1>();
    __syncthreads();
    const float(*cw)[G::WY][G::WX] = reinterpret_cast<const float(*)[G::WY][G::WX]>(cw0 + (k & 1) * G::WIN);
    // along y: pixel row r of the block at every window column; x[2k + j] gets h_j a_k + g_j d_k, so
    // row r reads window rows (r - j)/2 + LH, j = r mod 2, r mod 2 + 2, ... (each item is a row pair,
    // so the filter taps of both parities are compile-time indices)
    for (int i = t; i < G::OY * G::NQ; i += G::THREADS) {
      const int rp = i / G::NQ, q = i % G::NQ;
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        const int r = 2 * rp + par;
        F4x2 sa, sg, sv, sd;
#pragma unroll
        for (int jj = 0; jj < L / 2; ++jj) {
          const int j = 2 * jj + par;
          const int kr = rp - jj + G::LH;  // (r - j) / 2 + LH
          const float2 hj = dup2(f.h[j]), gj = dup2(f.g[j]);
          sa.fma(hj, F4x2::ld(&cw[0][kr][4 * q]));
          sg.fma(gj, F4x2::ld(&cw[1][kr][4 * q]));
          sv.fma(hj, F4x2::ld(&cw[2][kr][4 * q]));
          sd.fma(gj, F4x2::ld(&cw[3][kr][4 * q]));
        }
        // lo = sum h A + wdet sum g H;  hi = wdet (sum h V + sum g D)
        F4x2 l2, h2;
        l2.p0 = __ffma2_rn(w2, sg.p0, sa.p0);
        l2.p1 = __ffma2_rn(w2, sg.p1, sa.p1);
        h2.p0 = __fmul2_rn(w2, __fadd2_rn(sv.p0, sd.p0));
        h2.p1 = __fmul2_rn(w2, __fadd2_rn(sv.p1, sd.p1));
        l2.st(&lo[r][4 * q]);
        h2.st(&hi[r][4 * q]);
      }
    }
    __syncthreads();
    // along x: pixels 4p .. 4p+3 of row r; pixel i reads window columns (i - j)/2 + CX
    const int ky0 = (tile / tiles_x) * G::OY, kx0 = (tile % tiles_x) * G::OX;
    for (int i = t; i < 2 * G::OY * (2 * G::OX / 4); i += G::THREADS) {
      const int r = i / (2 * G::OX / 4), p = i % (2 * G::OX / 4);
      float l[2 * G::NK2], h[2 * G::NK2];  // window columns 2p + K0 ..
#pragma unroll
      for (int c = 0; c < G::NK2; ++c) {
        const float2 l2 = *reinterpret_cast<const float2*>(&lo[r][2 * p + G::K0 + 2 * c]);
        const float2 h2 = *reinterpret_cast<const float2*>(&hi[r][2 * p + G::K0 + 2 * c]);
        l[2 * c] = l2.x;
        l[2 * c + 1] = l2.y;
        h[2 * c] = h2.x;
        h[2 * c + 1] = h2.y;
      }
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[e] = 0.f;
#pragma unroll
        for (int jj = 0; jj < L / 2; ++jj) {
          const int j = 2 * jj + (e & 1);
          const int kk = ((e - j) >> 1) + G::CX - G::K0;  // index into l/h (window column - 2p - K0)
          v[e] = fmaf(f.h[j], l[kk], v[e]);
          v[e] = fmaf(f.g[j], h[kk], v[e]);
        }
      }
      const int iy = 2 * ky0 + r, ix = 2 * kx0 + 4 * p;
      if (iy < ny && ix < nx)
        *reinterpret_cast<float4*>(out + (long long)iy * nx + ix) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// Resident CTAs of a 256-thread kernel with `smem` bytes of dynamic shared
// memory on the current device (the attribute set once per kernel).
int resident_ctas(const void* fn, int smem) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * sms;
}

// CTAs for `work` (column, plane) units of a 3D level: every resident CTA,
// down to one output plane each on the small levels (a CTA walks its planes
// one after the other, so short runs on many CTAs beat long runs on few).
int grid3d(long long work, int cap) {
  return (int)(work < cap ? (work < 1 ? 1 : work) : cap);
}

// Launch with programmatic stream serialization (the kernel waits on the
// previous grid itself, griddep_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int L>
cudaError_t launch_a2(cudaStream_t st, const float* in, int nx, int ny, float* A, float* H, float* V, float* D,
                      float wdet, const Filt& f) {
  static std::once_flag once;
  static int cap = 0;
  std::call_once(once, [] { cap = resident_ctas((const void*)dwt2d_analysis_fast_kernel<L>, A2F<L>::SMEM); });
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const int tx = ((nx >> 1) + A2F<L>::OX - 1) / A2F<L>::OX, ty = ((ny >> 1) + A2F<L>::OY - 1) / A2F<L>::OY;
  const int ntiles = tx * ty;
  return launch_pdl(dwt2d_analysis_fast_kernel<L>, ntiles < cap ? ntiles : cap, A2F<L>::SMEM, st, in, nx, ny, A, H, V,
                    D, wdet, f, tx, ntiles);
}

template <int L>
cudaError_t launch_s2(cudaStream_t st, const float* A, const float* H, const float* V, const float* D, float wdet,
                      int nx, int ny, float* out, const Filt& f) {
  static std::once_flag once;
  static int cap = 0;
  std::call_once(once, [] { cap = resident_ctas((const void*)dwt2d_synthesis_fast_kernel<L>, S2F<L>::SMEM); });
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const int tx = ((nx >> 1) + S2F<L>::OX - 1) / S2F<L>::OX, ty = ((ny >> 1) + S2F<L>::OY - 1) / S2F<L>::OY;
  const int ntiles = tx * ty;
  return launch_pdl(dwt2d_synthesis_fast_kernel<L>, ntiles < cap ? ntiles : cap, S2F<L>::SMEM, st, A, H, V, D, wdet,
                    nx, ny, out, f, tx, ntiles);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


// ----------------------------------------- 3D levels at HBM rate (nx % 8 == 0)
// One pass per level: a CTA owns an OX x OY block of coefficient columns and
// marches through a chunk of z planes.  Each input plane's window is staged
// by cp.async (NSLOT - 1 planes ahead), filtered along x and y in shared
// memory into the four (x, y) quarters; each thread folds its quarter values
// of every plane into register accumulators of the L/2 output planes that
// plane reaches (low and high along z, taps in tap order) and writes the
// finished output plane after every second input plane: the eight bands
// (code = zb << 2 | yb << 1 | xb; code 0 is the approximation) with float4
// stores.  The staging chunks' offsets are computed once per run of planes.
struct Bands8 {
  float* p[8];
};
struct CBands8 {
  const float* p[8];
};
__device__ __forceinline__ const float* band_sel(const CBands8& b, int c) {
  return c == 0 ? b.p[0] : c == 1 ? b.p[1] : c == 2 ? b.p[2] : c == 3 ? b.p[3]
       : c == 4 ? b.p[4] : c == 5 ? b.p[5] : c == 6 ? b.p[6] : b.p[7];
}

template <int L>
struct A3F {
  static constexpr int OX = 32, OY = 8, THREADS = 256, NSLOT = 4;
  static constexpr int HX = (L - 2 + 3) / 4 * 4;
  static constexpr int WX = 2 * OX + HX;
  static constexpr int WXP = pad_row(WX);  // row stride in shared memory
  static constexpr int WY = 2 * OY + L - 2;
  static constexpr int NQ = WX / 4;
  static constexpr int NCH = (WY * NQ + THREADS - 1) / THREADS;  // 16-byte chunks per thread and plane
  static constexpr int SLAB_BYTES = NSLOT * WY * WXP * 4;  // multiple of 16
  static constexpr int X_BYTES = WY * OX * 4;
  static constexpr int SMEM = SLAB_BYTES + 2 * X_BYTES;
};

template <int L>
__global__ void __launch_bounds__(256, 2) dwt3d_analysis_fast_kernel(const float* __restrict__ in, int nx, int ny, int nz,
                                                                  const Bands8 out, float wdet, const Filt f,
                                                                  int cols_x, int ncols) {
  using G = A3F<L>;
  extern __shared__ __align__(16) unsigned char dsm[];  // G::SMEM bytes (more than the static 48 KB)
  auto slab = reinterpret_cast<float(*)[G::WY][G::WXP]>(dsm);
  auto xl = reinterpret_cast<float(*)[G::OX]>(dsm + G::SLAB_BYTES);
  auto xh = reinterpret_cast<float(*)[G::OX]>(dsm + G::SLAB_BYTES + G::X_BYTES);
  const int t = threadIdx.x;
  const int nx2 = nx >> 1, ny2 = ny >> 1, nz2 = nz >> 1;
  griddep_wait();
  griddep_trigger();
  // this thread's y-pass output: quarter qq (xb = qq & 1, yb = qq >> 1), row ky, columns 4 qx .. 4 qx + 3
  const int qq = t / 64, ky = (t / 8) % 8, qx = t % 8;
  const int xb = qq & 1, yb = qq >> 1;
  const float(*src)[G::OX] = xb ? xh : xl;
  float2 fy[L];  // the y filter of this quarter, packed
#pragma unroll
  for (int j = 0; j < L; ++j) fy[j] = dup2(yb ? f.g[j] : f.h[j]);
  float* plo = qq == 0 ? out.p[0] : qq == 1 ? out.p[1] : qq == 2 ? out.p[2] : out.p[3];
  float* phi = qq == 0 ? out.p[4] : qq == 1 ? out.p[5] : qq == 2 ? out.p[6] : out.p[7];
  const float2 wlo = dup2(qq == 0 ? 1.f : wdet), whi = dup2(wdet);
  // this CTA's share of the (column, output plane) work, z fastest: whole runs of one column, so a
  // z halo is staged again only where the share crosses into the next column
  const long long W = (long long)ncols * nz2;
  const long long w_end = W * (blockIdx.x + 1) / gridDim.x;
  for (long long w = W * blockIdx.x / gridDim.x; w < w_end;) {
  const int colid = (int)(w / nz2);
  const int kz0 = (int)(w - (long long)colid * nz2);
  const int kz1 = (int)(w_end - w < (long long)(nz2 - kz0) ? kz0 + (w_end - w) : nz2);
  w += kz1 - kz0;
  const int kx0 = (colid % cols_x) * G::OX, ky0 = (colid / cols_x) * G::OY;
  __syncthreads();  // the previous run is done with the shared buffers
  const int nplanes = 2 * (kz1 - kz0) + L - 2;  // input planes 2 kz0 .. 2 kz1 + L - 3 (periodic)
  // this thread's 16-byte chunks of a plane's window: shared offset and in-plane source offset (with the
  // periodic wrap) are the same for every plane of the run, so they are computed once here
  int soff[G::NCH], goff[G::NCH];
#pragma unroll
  for (int c = 0; c < G::NCH; ++c) {
    const int i = t + c * G::THREADS;
    const int r = i / G::NQ, q = i - r * G::NQ;
    soff[c] = i < G::WY * G::NQ ? r * G::WXP + 4 * q : -1;
    goff[c] = ((2 * ky0 + r) % ny) * nx + (2 * kx0 + 4 * q) % nx;  // nx % 4 == 0: a chunk never straddles the wrap
  }
  auto load = [&](int pl) {
    if (pl < nplanes) {
      int z = 2 * kz0 + pl;
      while (z >= nz) z -= nz;
      float* dst = &slab[pl % G::NSLOT][0][0];
      const float* src = in + (long long)z * ny * nx;
#pragma unroll
      for (int c = 0; c < G::NCH; ++c)
        if (soff[c] >= 0) cp_async16(dst + soff[c], src + goff[c]);
    }
    cp_async_commit();  // one group per plane (possibly empty) keeps the group count uniform
  };
#pragma unroll
  for (int pl = 0; pl < G::NSLOT - 1; ++pl) load(pl);
  const int oy = ky0 + ky, ox = kx0 + 4 * qx;
  const bool store = oy < ny2 && ox < nx2;
  // x and y passes of input plane pl: this thread's quarter values of the plane
  auto plane = [&](int pl) -> F4x2 {
    load(pl + G::NSLOT - 1);
    cp_async_wait_group<G::NSLOT - 1>();  // this thread's copies of plane pl have landed
    __syncthreads();                      // ... and every other thread's
    const float(*w)[G::WXP] = slab[pl % G::NSLOT];
    for (int i = t; i < G::WY * (G::OX / 4); i += G::THREADS) {  // along x
      const int r = i / (G::OX / 4), q = i - r * (G::OX / 4);
      float v[8 + G::HX];
#pragma unroll
      for (int c = 0; c < (8 + G::HX) / 4; ++c) {
        const float4 w4 = *reinterpret_cast<const float4*>(&w[r][8 * q + 4 * c]);
        v[4 * c] = w4.x;
        v[4 * c + 1] = w4.y;
        v[4 * c + 2] = w4.z;
        v[4 * c + 3] = w4.w;
      }
      float sl[4], sh[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sl[k] = 0.f;
        sh[k] = 0.f;
#pragma unroll
        for (int j = 0; j < L; ++j) {
          sl[k] = fmaf(f.h[j], v[2 * k + j], sl[k]);
          sh[k] = fmaf(f.g[j], v[2 * k + j], sh[k]);
        }
      }
      *reinterpret_cast<float4*>(&xl[r][4 * q]) = make_float4(sl[0], sl[1], sl[2], sl[3]);
      *reinterpret_cast<float4*>(&xh[r][4 * q]) = make_float4(sh[0], sh[1], sh[2], sh[3]);
    }
    __syncthreads();
    F4x2 v4;  // along y
#pragma unroll
    for (int j = 0; j < L; ++j) v4.fma(fy[j], F4x2::ld(&src[2 * ky + j][4 * qx]));
    return v4;
  };
  // along z in registers: acc[i] accumulates output plane m = k - (NA - 1) + i while the pair of input
  // planes 2k, 2k + 1 passes (taps 2 (NA - 1 - i) and 2 (NA - 1 - i) + 1, in tap order)
  constexpr int NA = L / 2;
  F4x2 alo[NA], ahi[NA];
  for (int k = 0; 2 * k < nplanes; ++k) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const F4x2 v = plane(2 * k + e);
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        alo[i].fma(dup2(f.h[2 * (NA - 1 - i) + e]), v);
        ahi[i].fma(dup2(f.g[2 * (NA - 1 - i) + e]), v);
      }
    }
    if (k >= NA - 1 && store) {  // output plane kz0 + k - (NA - 1) has all its L taps
      const long long o = ((long long)(kz0 + k - (NA - 1)) * ny2 + oy) * nx2 + ox;
      alo[0].scale(wlo).st(plo + o);
      ahi[0].scale(whi).st(phi + o);
    }
#pragma unroll
    for (int i = 0; i < NA - 1; ++i) {
      alo[i] = alo[i + 1];
      ahi[i] = ahi[i + 1];
    }
    alo[NA - 1] = F4x2();
    ahi[NA - 1] = F4x2();
  }
  }  // runs
}

// Plane-parallel form of a 3D analysis level, for levels whose (column,
// output plane) items fit in one wave of CTAs: a CTA makes one output plane
// m of one column, staging all L input planes 2m .. 2m + L - 1 (periodic) at
// once and filtering them along x, then y, then z.  One staging round trip
// and two barriers instead of L serial plane steps; the passes are the
// marching kernel's, in the same tap order, so the bands are identical.
template <int L>
struct A3P {
  static constexpr int OX = 32, OY = 8, THREADS = 256;
  static constexpr int HX = (L - 2 + 3) / 4 * 4;
  static constexpr int WX = 2 * OX + HX;
  static constexpr int WXP = pad_row(WX);
  static constexpr int WY = 2 * OY + L - 2;
  static constexpr int NQ = WX / 4;
  static constexpr int NCH = (WY * NQ + THREADS - 1) / THREADS;
  static constexpr int SLAB_BYTES = L * WY * WXP * 4;
  static constexpr int X_BYTES = WY * OX * 4;
  static constexpr int SMEM = SLAB_BYTES + 2 * L * X_BYTES;  // L staged planes; x-low and x-high of each
};

template <int L>
__global__ void __launch_bounds__(256) dwt3d_analysis_pp_kernel(const float* __restrict__ in, int nx, int ny, int nz,
                                                                const Bands8 out, float wdet, const Filt f,
                                                                int cols_x, int ncols) {
  using G = A3P<L>;
  extern __shared__ __align__(16) unsigned char dsm[];
  auto slab = reinterpret_cast<float(*)[G::WY][G::WXP]>(dsm);                 // [plane]
  auto xbuf = reinterpret_cast<float(*)[G::WY][G::OX]>(dsm + G::SLAB_BYTES);  // [2 plane + xb]
  const int t = threadIdx.x;
  const int nx2 = nx >> 1, ny2 = ny >> 1;
  const int col = (int)(blockIdx.x % ncols), m = (int)(blockIdx.x / ncols);
  const int kx0 = (col % cols_x) * G::OX, ky0 = (col / cols_x) * G::OY;
  griddep_wait();
  griddep_trigger();
#pragma unroll
  for (int c = 0; c < G::NCH; ++c) {
    const int i = t + c * G::THREADS;
    if (i >= G::WY * G::NQ) break;
    const int r = i / G::NQ, q = i - r * G::NQ;
    const int soff = r * G::WXP + 4 * q;
    const int goff = ((2 * ky0 + r) % ny) * nx + (2 * kx0 + 4 * q) % nx;  // nx % 4 == 0: no chunk straddles the wrap
#pragma unroll
    for (int p = 0; p < L; ++p) {
      int z = 2 * m + p;
      while (z >= nz) z -= nz;
      cp_async16(&slab[p][0][0] + soff, in + (long long)z * ny * nx + goff);
    }
  }
  cp_async_commit();
  cp_async_wait_group<0>();
  __syncthreads();
  for (int i = t; i < L * G::WY * (G::OX / 4); i += G::THREADS) {  // along x, every plane
    const int p = i / (G::WY * (G::OX / 4)), ri = i - p * (G::WY * (G::OX / 4));
    const int r = ri / (G::OX / 4), q = ri - r * (G::OX / 4);
    float v[8 + G::HX];
#pragma unroll
    for (int c = 0; c < (8 + G::HX) / 4; ++c) {
      const float4 w4 = *reinterpret_cast<const float4*>(&slab[p][r][8 * q + 4 * c]);
      v[4 * c] = w4.x;
      v[4 * c + 1] = w4.y;
      v[4 * c + 2] = w4.z;
      v[4 * c + 3] = w4.w;
    }
    float sl[4], sh[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sl[k] = 0.f;
      sh[k] = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        sl[k] = fmaf(f.h[j], v[2 * k + j], sl[k]);
        sh[k] = fmaf(f.g[j], v[2 * k + j], sh[k]);
      }
    }
    *reinterpret_cast<float4*>(&xbuf[2 * p][r][4 * q]) = make_float4(sl[0], sl[1], sl[2], sl[3]);
    *reinterpret_cast<float4*>(&xbuf[2 * p + 1][r][4 * q]) = make_float4(sh[0], sh[1], sh[2], sh[3]);
  }
  __syncthreads();
  // along y (this thread's quarter qq, row ky, columns 4 qx ..), then along z over the L planes
  const int qq = t / 64, ky = (t / 8) % 8, qx = t % 8;
  const int xb = qq & 1, yb = qq >> 1;
  F4x2 lo, hi;
#pragma unroll
  for (int p = 0; p < L; ++p) {
    F4x2 v;
#pragma unroll
    for (int j = 0; j < L; ++j) v.fma(dup2(yb ? f.g[j] : f.h[j]), F4x2::ld(&xbuf[2 * p + xb][2 * ky + j][4 * qx]));
    lo.fma(dup2(f.h[p]), v);
    hi.fma(dup2(f.g[p]), v);
  }
  const int oy = ky0 + ky, ox = kx0 + 4 * qx;
  if (oy < ny2 && ox < nx2) {
    float* plo = qq == 0 ? out.p[0] : qq == 1 ? out.p[1] : qq == 2 ? out.p[2] : out.p[3];
    float* phi = qq == 0 ? out.p[4] : qq == 1 ? out.p[5] : qq == 2 ? out.p[6] : out.p[7];
    const long long o = ((long long)m * ny2 + oy) * nx2 + ox;
    lo.scale(dup2(qq == 0 ? 1.f : wdet)).st(plo + o);
    hi.scale(dup2(wdet)).st(phi + o);
  }
}

// Runs f(S, i + S) for S = 0 .. Q-1 while i + S < n (S a compile-time constant in each call).
template <int S, int Q, class F>
__device__ __forceinline__ bool march3(F& f, int i, int n) {
  if constexpr (S == Q) {
    return true;
  } else {
    if (i + S >= n) return true;
    if (!f(std::integral_constant<int, S>{}, i + S)) return false;
    return march3<S + 1, Q>(f, i, n);
  }
}

template <int L>
struct S3F {
  static constexpr int OX = 32, OY = 8, THREADS = 256, NSLOT = 3;  // coefficient block; 2 OX x 2 OY pixels
  static constexpr int LH = L / 2 - 1;
  static constexpr int CX = (LH + 3) / 4 * 4;
  static constexpr int WX = OX + CX;
  static constexpr int WY = OY + LH;
  static constexpr int NQ = WX / 4;
  static constexpr int K0 = (CX - LH) & ~1;
  static constexpr int NK2 = (CX + 2 - K0) / 2;
  static constexpr int NCH = (8 * WY * NQ + THREADS - 1) / THREADS;  // 16-byte chunks per thread and plane
};

// Synthesis of one 3D level: coefficient extents (nx/2, ny/2, nz/2) -> (nx, ny, nz).
// Per coefficient plane m the x/y synthesis of the four zb = 0 bands and of the
// four zb = 1 bands gives two full-resolution planes P_lo(m), P_hi(m); output
// plane 2m + e is then sum_jj h_{2jj+e} P_lo(m - jj) + g_{2jj+e} P_hi(m - jj).
template <int L>
__global__ void __launch_bounds__(256, 2) dwt3d_synthesis_fast_kernel(const CBands8 in, float wdet, int nx, int ny,
                                                                   int nz, float* __restrict__ out, const Filt f,
                                                                   int cols_x, int ncols) {
  using G = S3F<L>;
  __shared__ __align__(16) float cw[G::NSLOT][8][G::WY][G::WX];
  __shared__ __align__(16) float yl[2][2 * G::OY][G::WX];
  __shared__ __align__(16) float yh[2][2 * G::OY][G::WX];
  const int t = threadIdx.x;
  const int cx = nx >> 1, cy = ny >> 1, cz2 = nz >> 1;
  griddep_wait();
  griddep_trigger();
  const int pr = t / 16, pq = t % 16;  // this thread's pixel row and quad (x-pass, z-pass, store)
  // this CTA's share of the (column, coefficient plane) work, z fastest (as in the analysis)
  const long long W = (long long)ncols * cz2;
  const long long w_end = W * (blockIdx.x + 1) / gridDim.x;
  for (long long w = W * blockIdx.x / gridDim.x; w < w_end;) {
  const int colid = (int)(w / cz2);
  const int kz0 = (int)(w - (long long)colid * cz2);
  const int kz1 = (int)(w_end - w < (long long)(cz2 - kz0) ? kz0 + (w_end - w) : cz2);
  w += kz1 - kz0;
  const int kx0 = (colid % cols_x) * G::OX, ky0 = (colid / cols_x) * G::OY;
  __syncthreads();  // the previous run is done with the shared buffers
  const int nplanes = kz1 - kz0 + G::LH;  // coefficient planes kz0 - LH .. kz1 - 1 (periodic)
  // this thread's 16-byte chunks of a plane's eight band windows: shared offset and source (band, periodic
  // in-plane position) are the same for every coefficient plane of the run, so they are computed once here
  int soff[G::NCH];
  const float* gsrc[G::NCH];
#pragma unroll
  for (int c = 0; c < G::NCH; ++c) {
    const int i = t + c * G::THREADS;
    const int b = i / (G::WY * G::NQ), rq = i - b * (G::WY * G::NQ);
    const int r = rq / G::NQ, q = rq - r * G::NQ;
    const bool ok = i < 8 * G::WY * G::NQ;
    soff[c] = ok ? (b * G::WY + r) * G::WX + 4 * q : -1;
    gsrc[c] = ok ? band_sel(in, b) + pmod(ky0 - G::LH + r, cy) * cx + pmod(kx0 - G::CX + 4 * q, cx) : nullptr;
  }
  auto load = [&](int pl) {
    if (pl < nplanes) {
      const long long zoff = (long long)pmod(kz0 - G::LH + pl, cz2) * cy * cx;
      float* dst = &cw[pl % G::NSLOT][0][0][0];
#pragma unroll
      for (int c = 0; c < G::NCH; ++c)
        if (soff[c] >= 0) cp_async16(dst + soff[c], gsrc[c] + zoff);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int pl = 0; pl < G::NSLOT - 1; ++pl) load(pl);
  float4 rlo[L / 2], rhi[L / 2];  // P_lo, P_hi of the last L/2 coefficient planes, oldest first
#pragma unroll
  for (int j = 0; j < L / 2; ++j) rlo[j] = rhi[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  // one coefficient plane; the z ring is rotated, not shifted: logical entry k (k = 0 oldest) of plane pl
  // sits in rlo/rhi[(k + pl) % NRG], and the loop below is unrolled NRG times so that S = pl % NRG is a
  // compile-time constant in every copy
  constexpr int NRG = L / 2;
  auto plane_step = [&](auto sc, int pl) -> bool {
    constexpr int S = decltype(sc)::value;
    load(pl + G::NSLOT - 1);
    cp_async_wait_group<G::NSLOT - 1>();
    __syncthreads();
    const float(*W)[G::WY][G::WX] = cw[pl % G::NSLOT];
    // along y, both z halves: item = (half, row pair, quad)
    for (int i = t; i < 2 * G::OY * G::NQ; i += G::THREADS) {
      const int zb = i / (G::OY * G::NQ), rq = i % (G::OY * G::NQ);
      const int rp = rq / G::NQ, q = rq % G::NQ;
      const int c0 = zb << 2;
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        F4x2 s0, s1, s2, s3;  // codes c0 | 0, 1, 2, 3
#pragma unroll
        for (int jj = 0; jj < L / 2; ++jj) {
          const int j = 2 * jj + par;
          const int k = rp - jj + G::LH;
          const float2 hj = dup2(f.h[j]), gj = dup2(f.g[j]);
          s0.fma(hj, F4x2::ld(&W[c0 | 0][k][4 * q]));
          s2.fma(gj, F4x2::ld(&W[c0 | 2][k][4 * q]));
          s1.fma(hj, F4x2::ld(&W[c0 | 1][k][4 * q]));
          s3.fma(gj, F4x2::ld(&W[c0 | 3][k][4 * q]));
        }
        const int r = 2 * rp + par;
        // x-low rows: code c0 (weight 1 only for the approximation) + code c0|2; x-high rows: codes c0|1, c0|3
        const float2 w0 = dup2(zb ? wdet : 1.f), w2 = dup2(wdet);
        F4x2 l2, h2;
        l2.p0 = __ffma2_rn(w2, s2.p0, __fmul2_rn(w0, s0.p0));
        l2.p1 = __ffma2_rn(w2, s2.p1, __fmul2_rn(w0, s0.p1));
        h2.p0 = __fmul2_rn(w2, __fadd2_rn(s1.p0, s3.p0));
        h2.p1 = __fmul2_rn(w2, __fadd2_rn(s1.p1, s3.p1));
        l2.st(&yl[zb][r][4 * q]);
        h2.st(&yh[zb][r][4 * q]);
      }
    }
    __syncthreads();
    float4 P[2];  // along x: this thread's pixel quad of P_lo (zb = 0) and P_hi (zb = 1)
#pragma unroll
    for (int zb = 0; zb < 2; ++zb) {
      float l[2 * G::NK2], h[2 * G::NK2];
#pragma unroll
      for (int c = 0; c < G::NK2; ++c) {
        const float2 l2 = *reinterpret_cast<const float2*>(&yl[zb][pr][2 * pq + G::K0 + 2 * c]);
        const float2 h2 = *reinterpret_cast<const float2*>(&yh[zb][pr][2 * pq + G::K0 + 2 * c]);
        l[2 * c] = l2.x;
        l[2 * c + 1] = l2.y;
        h[2 * c] = h2.x;
        h[2 * c + 1] = h2.y;
      }
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[e] = 0.f;
#pragma unroll
        for (int jj = 0; jj < L / 2; ++jj) {
          const int j = 2 * jj + (e & 1);
          const int k = ((e - j) >> 1) + G::CX - G::K0;
          v[e] = fmaf(f.h[j], l[k], v[e]);
          v[e] = fmaf(f.g[j], h[k], v[e]);
        }
      }
      P[zb] = make_float4(v[0], v[1], v[2], v[3]);
    }
    rlo[(NRG - 1 + S) % NRG] = P[0];  // the newest plane replaces the oldest
    rhi[(NRG - 1 + S) % NRG] = P[1];
    if (pl >= G::LH) {  // rings hold coefficient planes m - LH .. m: output planes 2m, 2m + 1
      const int m = kz0 + pl - G::LH;
      const int iy = 2 * ky0 + pr, ix = 2 * kx0 + 4 * pq;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        F4x2 v;
#pragma unroll
        for (int jj = 0; jj < L / 2; ++jj) {
          const int j = 2 * jj + e;
          F4x2 a, b;
          a.p0 = make_float2(rlo[(NRG - 1 - jj + S) % NRG].x, rlo[(NRG - 1 - jj + S) % NRG].y);
          a.p1 = make_float2(rlo[(NRG - 1 - jj + S) % NRG].z, rlo[(NRG - 1 - jj + S) % NRG].w);
          b.p0 = make_float2(rhi[(NRG - 1 - jj + S) % NRG].x, rhi[(NRG - 1 - jj + S) % NRG].y);
          b.p1 = make_float2(rhi[(NRG - 1 - jj + S) % NRG].z, rhi[(NRG - 1 - jj + S) % NRG].w);
          v.fma(dup2(f.h[j]), a);
          v.fma(dup2(f.g[j]), b);
        }
        if (iy < ny && ix < nx) v.st(out + ((long long)(2 * m + e) * ny + iy) * nx + ix);
      }
    }
    return true;
  };
  for (int pl = 0; pl < nplanes; pl += NRG) march3<0, NRG>(plane_step, pl, nplanes);
  }  // runs
}

template <int L>
cudaError_t launch_a3(cudaStream_t st, const float* in, int nx, int ny, int nz, const Bands8& b, float wdet,
                      const Filt& f) {
  static std::once_flag once;
  static int cap = 0;
  static int cap_pp = 0;
  std::call_once(once, [] {
    cap = resident_ctas((const void*)dwt3d_analysis_fast_kernel<L>, A3F<L>::SMEM);
    cap_pp = resident_ctas((const void*)dwt3d_analysis_pp_kernel<L>, A3P<L>::SMEM);
  });
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const int cols_x = ((nx >> 1) + A3F<L>::OX - 1) / A3F<L>::OX;
  const int ncols = cols_x * (((ny >> 1) + A3F<L>::OY - 1) / A3F<L>::OY);
  const long long work = (long long)ncols * (nz >> 1);
  if (work <= cap_pp)  // every (column, output plane) item in one wave: no serial plane march
    return launch_pdl(dwt3d_analysis_pp_kernel<L>, (int)work, A3P<L>::SMEM, st, in, nx, ny, nz, b, wdet, f, cols_x,
                      ncols);
  return launch_pdl(dwt3d_analysis_fast_kernel<L>, grid3d(work, cap), A3F<L>::SMEM, st, in, nx, ny, nz, b, wdet, f,
                    cols_x, ncols);
}

template <int L>
cudaError_t launch_s3(cudaStream_t st, const CBands8& b, float wdet, int nx, int ny, int nz, float* out,
                      const Filt& f) {
  static std::once_flag once;
  static int cap = 0;
  std::call_once(once, [] { cap = resident_ctas((const void*)dwt3d_synthesis_fast_kernel<L>, 0); });
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const int cols_x = ((nx >> 1) + S3F<L>::OX - 1) / S3F<L>::OX;
  const int ncols = cols_x * (((ny >> 1) + S3F<L>::OY - 1) / S3F<L>::OY);
  const long long work = (long long)ncols * (nz >> 1);
  return launch_pdl(dwt3d_synthesis_fast_kernel<L>, grid3d(work, cap), 0, st, b, wdet, nx, ny, nz, out, f, cols_x,
                    ncols);
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
  // (nx bounded: the fast kernels keep in-window source offsets as int)
  if (nx % 8 == 0 && nx <= (1 << 24) && ny % 2 == 0 && aligned16(in) && aligned16(approx) && aligned16(bandH) &&
      aligned16(bandV) && aligned16(bandD) && (L == 2 || L == 4 || L == 8)) {
    if (L == 2) return launch_a2<2>(st, in, nx, ny, approx, bandH, bandV, bandD, wdet, f);
    if (L == 4) return launch_a2<4>(st, in, nx, ny, approx, bandH, bandV, bandD, wdet, f);
    return launch_a2<8>(st, in, nx, ny, approx, bandH, bandV, bandD, wdet, f);
  }
  dim3 grid(((nx >> 1) + A_OX - 1) / A_OX, ((ny >> 1) + A_OY - 1) / A_OY);
  dwt2d_analysis_kernel<<<grid, A_THREADS, 0, st>>>(in, nx, ny, approx, bandH, bandV, bandD, wdet, f);
  return cudaGetLastError();
}

cudaError_t dwt2d_synthesis_level(const float* approx, const float* bandH, const float* bandV, const float* bandD,
                                  float wdet, int nx, int ny, float* out, const float* h, const float* g, int L,
                                  cudaStream_t st) {
  const Filt f = make_filt(h, g, L);
  // (nx bounded: the fast kernels keep in-window source offsets as int, the band in bits 28-29)
  if (nx % 8 == 0 && nx <= (1 << 24) && ny % 2 == 0 && aligned16(approx) && aligned16(bandH) && aligned16(bandV) &&
      aligned16(bandD) && aligned16(out) && (L == 2 || L == 4 || L == 8)) {
    if (L == 2) return launch_s2<2>(st, approx, bandH, bandV, bandD, wdet, nx, ny, out, f);
    if (L == 4) return launch_s2<4>(st, approx, bandH, bandV, bandD, wdet, nx, ny, out, f);
    return launch_s2<8>(st, approx, bandH, bandV, bandD, wdet, nx, ny, out, f);
  }
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

cudaError_t dwt3d_analysis_level(const float* in, int nx, int ny, int nz, float* const bands[8], float wdet,
                                 const float* h, const float* g, int L, cudaStream_t st) {
  if (nx % 8 != 0 || ny % 2 != 0 || nz % 2 != 0 || !(L == 2 || L == 4 || L == 8) || !aligned16(in))
    return cudaErrorNotSupported;
  if ((long long)nx * ny > 0x7fffffffLL) return cudaErrorNotSupported;  // in-plane offsets are int
  Bands8 b;
  for (int c = 0; c < 8; ++c) {
    if (!aligned16(bands[c])) return cudaErrorNotSupported;
    b.p[c] = bands[c];
  }
  const Filt f = make_filt(h, g, L);
  if (L == 2) return launch_a3<2>(st, in, nx, ny, nz, b, wdet, f);
  if (L == 4) return launch_a3<4>(st, in, nx, ny, nz, b, wdet, f);
  return launch_a3<8>(st, in, nx, ny, nz, b, wdet, f);
}

cudaError_t dwt3d_synthesis_level(const float* const bands[8], float wdet, int nx, int ny, int nz, float* out,
                                  const float* h, const float* g, int L, cudaStream_t st) {
  if (nx % 8 != 0 || ny % 2 != 0 || nz % 2 != 0 || !(L == 2 || L == 4 || L == 8) || !aligned16(out))
    return cudaErrorNotSupported;
  if ((long long)nx * ny > 0x7fffffffLL) return cudaErrorNotSupported;  // in-plane offsets are int
  CBands8 b;
  for (int c = 0; c < 8; ++c) {
    if (!aligned16(bands[c])) return cudaErrorNotSupported;
    b.p[c] = bands[c];
  }
  const Filt f = make_filt(h, g, L);
  if (L == 2) return launch_s3<2>(st, b, wdet, nx, ny, nz, out, f);
  if (L == 4) return launch_s3<4>(st, b, wdet, nx, ny, nz, out, f);
  return launch_s3<8>(st, b, wdet, nx, ny, nz, out, f);
}

cudaError_t scale_copy_launch(float* dst, const float* src, long long n, float w, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scale_copy_kernel<<<grid1d(n), 256, 0, st>>>(dst, src, n, w);
  return cudaGetLastError();
}

}  // namespace pat
