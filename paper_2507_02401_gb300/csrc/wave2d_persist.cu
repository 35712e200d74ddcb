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
// Precision.  kappa is applied as an unevaluated pair kappa_hi + kappa_lo:
// with a constant medium a rounded kappa is the same everywhere and shifts
// the phase of every mode coherently, step after step.  In the adjoint the
// state Q integrates G over time and, in a closed (reflecting) box, grows far
// beyond the result.  The adjoint therefore runs in Z = kappa Q,
//   G^n = G^{n+1} + S^T r_n + L Z^{n+1},  Z^n = Z^{n+1} + kappa G^n,
// with Z kept as a compensated pair Z + Z_lo (TwoSum) that is exchanged and
// fed to the stencil as two FP32 fields (Z through the difference form, whose
// rounding is relative to the differences, Z_lo through the cheap form); G is
// plain.
//
// GB300 mapping.  The grid is cut into 64 x 32 tiles, one CTA per tile, all
// co-resident (cooperative launch).  Each thread keeps its 2 x 4 cells' state
// in registers for the whole loop; the CTA keeps the current field plus an
// R-deep halo in shared memory (double buffered).  After each step the
// threads that own boundary cells write the R-deep strips straight to an
// L2-resident exchange buffer (relaxed GPU-scope stores; 93.4 against 92.3
// reconstruction iterations/s at 512^2 when they were staged in shared memory
// and handed to the TMA engine), every value packed with the step it belongs
// to into one 64-bit word; an aligned
// 64-bit access is single-copy atomic, so a neighbour that reads a word with
// the expected tag has the right value: no flags, no fences, one L2 round
// trip per exchange and one CTA barrier per step.  Every wait is bounded by a
// global-timer limit and a shared abort flag; a CTA that gives up records
// PAT_ERR_TIMEOUT, raises the abort flag and leaves the loop, so the launch
// always ends.
#include "internal.h"
#include "stencil.cuh"

namespace pat {
namespace {

using u64 = unsigned long long;

constexpr int TX = 64;
constexpr int TY = 32;
constexpr int NTHREADS = (TX / 4) * (TY / 2);  // 256: each thread owns 2 rows x 4 columns
constexpr int XOFF = 8;                         // left halo columns in shared memory (>= R, multiple of 4)
constexpr int PITCH = TX + 16;                  // 8 halo columns each side
constexpr int RCOUNT = NTHREADS / 4;            // threads serving one neighbour
static_assert(NTHREADS % 128 == 0, "four halo regions need whole warps");

template <int R, bool ADJ>
struct Geo {
  static constexpr int NF = ADJ ? 2 : 1;           // shared-memory fields: P, or (W_hi, W_lo)
  static constexpr int ROWS = TY + 2 * R;
  static constexpr int SBUF = ROWS * PITCH;        // one shared-memory field buffer
  static constexpr int STRIP = 2 * R * (TX + TY);  // exchanged words per tile per slot
  static constexpr int SLOT = STRIP;
  static constexpr int NPAIR = R * TX / 2;         // word pairs of a north/south strip
  static constexpr int NSIDE = TY * R;             // words of a west/east strip
  static constexpr int PER_NS = (NPAIR + RCOUNT - 1) / RCOUNT;
  static constexpr int PER_WE = (NSIDE + RCOUNT - 1) / RCOUNT;
};

// Exchange words.  The buffer is filled with 0xff bytes before every launch,
// so no stale word can carry a valid tag.
//   forward: [step (32 bits)][P (32 bits)]
//   adjoint: [W_lo with its low 8 mantissa bits replaced by step mod 128][W_hi]
//            (W_lo is a correction ~2^-24 of W_hi; dropping 8 of its bits is
//            far below FP32 rounding of W)
template <bool ADJ>
__device__ __forceinline__ u64 pack(float hi, float lo, unsigned step) {
  if (!ADJ) return ((u64)step << 32) | (u64)__float_as_uint(hi);
  const unsigned l = (__float_as_uint(lo) & ~0xffu) | (step & 0x7fu);
  return ((u64)l << 32) | (u64)__float_as_uint(hi);
}
template <bool ADJ>
__device__ __forceinline__ bool tag_ok(u64 w, unsigned step) {
  const unsigned h = (unsigned)(w >> 32);
  return ADJ ? (h & 0xffu) == (step & 0x7fu) : h == step;
}
__device__ __forceinline__ float word_hi(u64 w) { return __uint_as_float((unsigned)(w & 0xffffffffull)); }
__device__ __forceinline__ float word_lo(u64 w) { return __uint_as_float((unsigned)(w >> 32) & ~0xffu); }

// Exchange words are written with relaxed GPU-scope stores straight from the
// owning threads (aligned 64-bit elements: single-copy atomic) and read with
// relaxed GPU-scope loads.
__device__ __forceinline__ void st_word2(u64* p, u64 a, u64 b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void st_word(u64* p, u64 a) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}
__device__ __forceinline__ void ld_word2(const u64* p, u64& a, u64& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ u64 ld_word(const u64* p) {
  u64 a;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(a) : "l"(p) : "memory");
  return a;
}

// Write the thread's 2x4 block of the new state into the shared field
// buffer(s) Sn (second field at Sn + SBUF) and, packed and tagged, its
// boundary cells into the tile's exchange slot X in global memory, laid out
// as the boundary strips [top R x TX][bottom R x TX][left TY x R][right TY x R].
template <int R, bool ADJ>
__device__ __forceinline__ void store_state(float* Sn, u64* X, const float V[2][4], const float Vl[2][4], int r0,
                                            int c0, unsigned step) {
  constexpr int SBUF = Geo<R, ADJ>::SBUF;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int row = r0 + rr;
    *reinterpret_cast<float4*>(Sn + (row + R) * PITCH + XOFF + c0) =
        make_float4(V[rr][0], V[rr][1], V[rr][2], V[rr][3]);
    if (ADJ)
      *reinterpret_cast<float4*>(Sn + SBUF + (row + R) * PITCH + XOFF + c0) =
          make_float4(Vl[rr][0], Vl[rr][1], Vl[rr][2], Vl[rr][3]);
    u64 w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = pack<ADJ>(V[rr][j], Vl[rr][j], step);
    u64* dst = nullptr;
    if (row < R) dst = X + row * TX + c0;
    if (row >= TY - R) dst = X + R * TX + (row - (TY - R)) * TX + c0;
    if (dst) {  // TY >= 2R: a row is in at most one of the two strips
      st_word2(dst, w[0], w[1]);
      st_word2(dst + 2, w[2], w[3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + j;
      if (col < R) st_word(X + 2 * R * TX + row * R + col, w[j]);
      if (col >= TX - R) st_word(X + 2 * R * TX + TY * R + row * R + (col - (TX - R)), w[j]);
    }
  }
}

// Copy the halo of state `step` of NR fields from the neighbour's strips X[r]
// into the shared buffers Sc[r] (second field at Sc[r] + SBUF).  Executed by
// the RCOUNT threads of one region; returns false if the wait ran out.  Each
// poll first issues the loads of every word still pending (all fields), then
// checks their tags, so the L2 round trips of one poll overlap instead of
// following one another.
template <int R, bool ADJ, int NR>
__device__ bool load_halo(float* const (&Sc)[NR], const u64* const (&X)[NR], int region, int rrank, unsigned step,
                          const int* abort, long long timeout_ns, int poll_ns) {
  using G = Geo<R, ADJ>;
  constexpr int PMAX = G::PER_NS > G::PER_WE ? G::PER_NS : G::PER_WE;
  static_assert(NR * PMAX <= 32, "pending bits");
  const bool ns = region < 2;
  const int per = ns ? G::PER_NS : G::PER_WE;
  const int count = ns ? G::NPAIR : G::NSIDE;
  unsigned pending = 0;  // bit r * PMAX + j
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
      if (j < per && rrank + j * RCOUNT < count) pending |= 1u << (r * PMAX + j);
  unsigned long long t0 = 0;
  for (unsigned it = 0; it < (1u << 28); ++it) {
    u64 wa[NR][PMAX], wb[NR][PMAX];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < PMAX; ++j) {
        wa[r][j] = wb[r][j] = 0ull;
        if (!(pending & (1u << (r * PMAX + j)))) continue;
        const int i = rrank + j * RCOUNT;
        if (ns)
          ld_word2(X[r] + (region == 0 ? R * TX : 0) + 2 * i, wa[r][j], wb[r][j]);
        else
          wa[r][j] = ld_word(X[r] + 2 * R * TX + (region == 2 ? TY * R : 0) + i);
      }
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < PMAX; ++j) {
        const unsigned bit = 1u << (r * PMAX + j);
        if (!(pending & bit)) continue;
        const int i = rrank + j * RCOUNT;
        if (ns) {
          if (tag_ok<ADJ>(wa[r][j], step) && tag_ok<ADJ>(wb[r][j], step)) {
            const int row = (2 * i) / TX, col = (2 * i) % TX;
            const int o = (region == 0 ? row : TY + R + row) * PITCH + XOFF + col;
            *reinterpret_cast<float2*>(Sc[r] + o) = make_float2(word_hi(wa[r][j]), word_hi(wb[r][j]));
            if (ADJ) *reinterpret_cast<float2*>(Sc[r] + G::SBUF + o) = make_float2(word_lo(wa[r][j]), word_lo(wb[r][j]));
            pending &= ~bit;
          }
        } else {
          if (tag_ok<ADJ>(wa[r][j], step)) {
            const int row = i / R, jj = i % R;
            const int o = (row + R) * PITCH + (region == 2 ? XOFF - R + jj : XOFF + TX + jj);
            Sc[r][o] = word_hi(wa[r][j]);
            if (ADJ) Sc[r][G::SBUF + o] = word_lo(wa[r][j]);
            pending &= ~bit;
          }
        }
      }
    if (__all_sync(0xffffffffu, pending == 0)) return true;
    if (it == 0) t0 = global_timer_ns();
    if (poll_ns > 0) __nanosleep(poll_ns);
    if ((it & 31u) == 31u) {
      if (ld_relaxed_gpu(abort) != 0) return false;
      if ((long long)(global_timer_ns() - t0) > timeout_ns) return false;
    }
  }
  return false;
}

// SP: absorbing layer.  With per-cell factors a, b (1 outside the layer):
//   forward  D' = a D + b inc (first step D' = (a-1) P + b inc), P' = P + D'
//   adjoint  G' = G + inc, Q' = a Q + b G', i.e. Z' = a Z + b kappa G' (final x = ... + ((a-1)/b) Q);
//   inside the layer Z_lo is only damped (the fields are being damped there).
// NR right-hand sides advance together (NR = 2: two independent fields of the same plan, e.g. two CG
// solves of one medium): every step exchanges both fields' strips in the same round trip and runs both
// updates between the same barriers.  Inputs / outputs of field r are a.in / a.out (r = 0) and a.in1 /
// a.out1 (r = 1); field r's exchange words follow field 0's in each slot.
template <int R, bool ADJ, bool VARC, bool SP, int NR>
__global__ void __launch_bounds__(NTHREADS, 1) wave2d_persist_kernel(const Persist2DArgs a) {
  using G = Geo<R, ADJ>;
  static_assert(NR == 1 || !SP, "several right-hand sides run without the absorbing layer");
  extern __shared__ float4 smem4[];
  float* S0 = reinterpret_cast<float*>(smem4);   // [slot][rhs][field] buffers
  float* J0 = S0 + 2 * NR * G::NF * G::SBUF;     // adjoint injection accumulators, [rhs][slot] x TY x TX
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
  u64* xbuf = reinterpret_cast<u64*>(a.xbuf);
  float2 w2[R + 1];  // stencil weights, packed
#pragma unroll
  for (int m = 0; m <= R; ++m) w2[m] = dup2(a.w[m]);
  const float* IN[2] = {a.in, a.in1};
  float* OUT[2] = {a.out, a.out1};
  float* PART[2] = {a.part, a.part1};

  // halo duty of this warp: 0 = north, 1 = south, 2 = west, 3 = east neighbour
  const int region = warp & 3;
  const int rrank = (warp >> 2) * 32 + lane;
  int nb = -1;
  if (region == 0 && tiy > 0) nb = tile - a.tiles_x;
  if (region == 1 && tiy < a.tiles_y - 1) nb = tile + a.tiles_x;
  if (region == 2 && tix > 0) nb = tile - 1;
  if (region == 3 && tix < a.tiles_x - 1) nb = tile + 1;

  // forward: P, D ; adjoint: Z (in P, with Z_lo in Pl), G (in D); per right-hand side
  float P[NR][2][4], D[NR][2][4], Pl[NR][2][4];
  float K[2][4], Kl[2][4];
  float SA[2][4], SB[2][4];  // layer factors (SP only)
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
      Kl[rr][j] = v ? (VARC ? a.kappa_lo[gi] : a.kappa0_lo) : 0.f;
      SA[rr][j] = (SP && v) ? a.sp_a[gi] : 1.f;
      SB[rr][j] = (SP && v) ? a.sp_b[gi] : 1.f;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        P[r][rr][j] = (!ADJ && v) ? IN[r][gi] : 0.f;
        D[r][rr][j] = 0.f;
        Pl[r][rr][j] = 0.f;
      }
    }
  for (int i = t; i < 2 * NR * G::NF * G::SBUF; i += NTHREADS) S0[i] = 0.f;
  if (ADJ)
    for (int i = t; i < NR * 2 * TX * TY; i += NTHREADS) J0[i] = 0.f;
  if (t == 0) s_abort = 0;
  __syncthreads();

  auto Sbuf = [&](int slot, int r) { return S0 + (slot * NR + r) * G::NF * G::SBUF; };
  auto Jbuf = [&](int r, int slot) { return J0 + (r * 2 + slot) * TX * TY; };
  auto Xslot = [&](int tl, int slot, int r) { return xbuf + ((size_t)tl * 2 + slot) * NR * G::SLOT + r * G::SLOT; };
#pragma unroll
  for (int r = 0; r < NR; ++r)  // publish state 0 (forward: x; adjoint: zero)
    store_state<R, ADJ>(Sbuf(0, r), Xslot(tile, 0, r), P[r], Pl[r], r0, c0, 0u);

  for (int k = 0; k < nt; ++k) {
    if (ADJ) {  // S^T r_n for this tile's injected cells, n = nt-1-k (independent of the halo: these
                //  dependent loads overlap the neighbours' exchange)
      const int n = nt - 1 - k;
      const int e1 = a.tile_inj_ptr[tile + 1];
      for (int e = a.tile_inj_ptr[tile] + t; e < e1; e += NTHREADS) {
        const InjCell ic = a.inj[e];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          float s = 0.f;
          for (int q = ic.beg; q < ic.end; ++q) s = fmaf(a.ent_w[q], IN[r][(long long)a.ent_sensor[q] * nt + n], s);
          Jbuf(r, k & 1)[ic.local] = s;
        }
      }
    }
    // ---- halo of state k from the neighbour's slot (k & 1)
    if (nb >= 0) {
      float* sc[NR];
      const u64* xs[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        sc[r] = Sbuf(k & 1, r);
        xs[r] = Xslot(nb, k & 1, r);
      }
      if (!load_halo<R, ADJ, NR>(sc, xs, region, rrank, (unsigned)k, a.abort, a.timeout_ns, a.poll_ns)) {
        if (lane == 0) {
          s_abort = 1;
          atomicCAS(a.status, (int)PAT_OK, (int)PAT_ERR_TIMEOUT);
          atomicExch(a.abort, 1);
        }
      }
    }
    __syncthreads();
    if (s_abort) break;

    if (!ADJ) {  // y[:, k] = S P^k
      const int e1 = a.tile_samp_ptr[tile + 1];
      for (int e = a.tile_samp_ptr[tile] + t; e < e1; e += NTHREADS) {
        const SampEntry se = a.samp[e];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float* b = Sbuf(k & 1, r) + (se.ly + R) * PITCH + XOFF + se.lx;
          if (se.part < 0) {
            const float v = se.w[0] * b[0] + se.w[1] * b[1] + se.w[2] * b[PITCH] + se.w[3] * b[PITCH + 1];
            OUT[r][(long long)se.sensor * nt + k] = v;
          } else {
            PART[r][(long long)se.part * nt + k] = se.w[0] * b[0];
          }
        }
      }
    }

#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float* Sc = Sbuf(k & 1, r);
      const float* Jc = Jbuf(r, k & 1);
      float L[2][4];
      lap_2x4_p<R, true, false>(Sc, PITCH, r0 + R, XOFF + c0, w2, L);
      if (ADJ) lap_2x4_p<R, false, true>(Sc + G::SBUF, PITCH, r0 + R, XOFF + c0, w2, L);

      if (k == nt - 1) {
        if (ADJ) {  // x = S^T r_0 + G^1 + 1/2 L Z^1
#pragma unroll
          for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (!valid[rr][j]) continue;
              const int lr = r0 + rr, lc = c0 + j;
              float xv = Jc[lr * TX + lc] + D[r][rr][j] + 0.5f * L[rr][j];
              if (SP && SA[rr][j] != 1.f)  // + ((a-1)/b) Q,  Q = (Z + Z_lo) / kappa
                xv = fmaf((SA[rr][j] - 1.f) / SB[rr][j], (P[r][rr][j] + Pl[r][rr][j]) / (K[rr][j] + Kl[rr][j]), xv);
              OUT[r][(long long)(gy0 + lr) * nx + gx0 + lc] = xv;
            }
        }
        continue;
      }

      float V[2][4], Vl[2][4];
      if (!ADJ) {
        const float cf = (k == 0) ? 0.5f : 1.0f;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // D += cf (kappa_hi + kappa_lo) L, the product rounded once before it meets D
            const float inc = fmaf(cf * K[rr][j], L[rr][j], (cf * Kl[rr][j]) * L[rr][j]);
            if (SP)
              D[r][rr][j] = k == 0 ? fmaf(SA[rr][j] - 1.f, P[r][rr][j], SB[rr][j] * inc)
                                   : fmaf(SA[rr][j], D[r][rr][j], SB[rr][j] * inc);
            else
              D[r][rr][j] += inc;
            P[r][rr][j] += D[r][rr][j];
            V[rr][j] = P[r][rr][j];
            Vl[rr][j] = 0.f;
          }
      } else {
        float* Jw = Jbuf(r, k & 1);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int li = (r0 + rr) * TX + c0 + j;
            const float inc = Jw[li] + L[rr][j];
            Jw[li] = 0.f;
            float g = D[r][rr][j] + inc;                         // G += S^T r + L Z
            const float u = fmaf(K[rr][j], g, Kl[rr][j] * g);    // (kappa_hi + kappa_lo) G, rounded once
            float z, zl;
            if (SP && (SA[rr][j] != 1.f || SB[rr][j] != 1.f)) {  // Z = a Z + b kappa G inside the layer
              z = fmaf(SA[rr][j], P[r][rr][j], SB[rr][j] * u);
              zl = SA[rr][j] * Pl[r][rr][j];
            } else {
              float e;
              z = two_sum(P[r][rr][j], u, e);  // Z += kappa G (compensated)
              zl = Pl[r][rr][j] + e;
            }
            if (!valid[rr][j]) g = z = zl = 0.f;
            D[r][rr][j] = g;
            P[r][rr][j] = z;
            Pl[r][rr][j] = zl;
            V[rr][j] = z;
            Vl[rr][j] = zl;
          }
      }
      store_state<R, ADJ>(Sbuf((k + 1) & 1, r), Xslot(tile, (k + 1) & 1, r), V, Vl, r0, c0, (unsigned)(k + 1));
    }
    if (k == nt - 1) break;
  }

}

__global__ void split_combine_kernel(const float* __restrict__ part, const int* __restrict__ split_sensor,
                                     int nsplit, int nt, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nsplit * nt) return;
  const int q = (int)(i / nt), t = (int)(i % nt);
  const float* p = part + (long long)4 * q * nt + t;
  y[(long long)split_sensor[q] * nt + t] = ((p[0] + p[nt]) + p[2 * nt]) + p[3 * nt];
}

template <int R, bool ADJ, bool VARC, bool SP, int NR = 1>
void* kfn() {
  return (void*)wave2d_persist_kernel<R, ADJ, VARC, SP, NR>;
}

template <bool SP>
void* pick_sp(int R, bool adj, bool varc) {
#define PAT_P2D(RR)                                                               \
  if (R == RR) {                                                                  \
    if (adj) return varc ? kfn<RR, true, true, SP>() : kfn<RR, true, false, SP>(); \
    return varc ? kfn<RR, false, true, SP>() : kfn<RR, false, false, SP>();       \
  }
  PAT_P2D(1)
  PAT_P2D(3)
  PAT_P2D(5)
  PAT_P2D(7)
#undef PAT_P2D
  return nullptr;
}

void* pick(int R, bool adj, bool varc) { return pick_sp<false>(R, adj, varc); }

// two right-hand sides, no absorbing layer
void* pick2(int R, bool adj, bool varc) {
#define PAT_P2D2(RR)                                                                              \
  if (R == RR) {                                                                                  \
    if (adj) return varc ? kfn<RR, true, true, false, 2>() : kfn<RR, true, false, false, 2>();    \
    return varc ? kfn<RR, false, true, false, 2>() : kfn<RR, false, false, false, 2>();           \
  }
  PAT_P2D2(1)
  PAT_P2D2(3)
  PAT_P2D2(5)
  PAT_P2D2(7)
#undef PAT_P2D2
  return nullptr;
}

size_t smem_bytes(int R, bool adj, int nr = 1) {
  const size_t sbuf = (size_t)(TY + 2 * R) * PITCH;
  const size_t nf = adj ? 2 : 1;
  return (size_t)nr * (2 * nf * sbuf + (adj ? 2 * (size_t)TX * TY : 0)) * sizeof(float);
}

cudaError_t prepare(void* f, int R, bool adj, int nr = 1) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(R, adj, nr));
}

}  // namespace

cudaError_t persist2d_split_combine(const float* part, const int* split_sensor, int nsplit, int nt, float* y,
                                    cudaStream_t st) {
  if (nsplit <= 0) return cudaSuccess;
  const long long n = (long long)nsplit * nt;
  split_combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, split_sensor, nsplit, nt, y);
  return cudaGetLastError();
}

bool persist2d_supported(int R, bool) { return R == 1 || R == 3 || R == 5 || R == 7; }
int persist2d_tile_x() { return TX; }
int persist2d_tile_y() { return TY; }
size_t persist2d_smem_bytes(int R, bool adj) { return smem_bytes(R, adj); }
size_t persist2d_xbuf_words(int R, bool, int ntiles, int nr) { return (size_t)nr * ntiles * 2 * 2 * R * (TX + TY); }

int persist2d_max_ctas(int R, bool adj, bool varc) {
  void* f = pick(R, adj, varc);
  if (!f) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (prepare(f, R, adj) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, NTHREADS, smem_bytes(R, adj)) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

cudaError_t persist2d_launch_layer(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st) {
  void* f = pick_sp<true>(R, adj, varc);
  if (!f) return cudaErrorInvalidValue;
  int per_sm = 0, dev = 0, sms = 0;  // the layer variant must fit as many CTAs as the plan's tiles
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorUnknown;
  cudaError_t e = prepare(f, R, adj);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, NTHREADS, smem_bytes(R, adj));
  if (e != cudaSuccess) return e;
  if (per_sm * sms < nctas) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(f, dim3(nctas), dim3(NTHREADS), args, smem_bytes(R, adj), st);
}

int persist2d_max_ctas2(int R, bool adj, bool varc) {
  void* f = pick2(R, adj, varc);
  if (!f) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (prepare(f, R, adj, 2) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, NTHREADS, smem_bytes(R, adj, 2)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per_sm;
}

cudaError_t persist2d_launch2(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st) {
  void* f = pick2(R, adj, varc);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare(f, R, adj, 2);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(f, dim3(nctas), dim3(NTHREADS), args, smem_bytes(R, adj, 2), st);
}

cudaError_t persist2d_launch(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st) {
  void* f = pick(R, adj, varc);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare(f, R, adj);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(f, dim3(nctas), dim3(NTHREADS), args, smem_bytes(R, adj), st);
}

}  // namespace pat
