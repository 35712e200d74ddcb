// Internal declarations of the GB300 PAT library (not part of the C ABI).
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pat.h"

namespace pat {

constexpr int kMaxR = 7;       // composed stencil radius of order 8
constexpr int kMaxTaps = 8;    // db4 filter length
constexpr int kMaxLevels = 20;

// Orthonormal Daubechies scaling filter with nv vanishing moments (2 nv taps);
// false if its orthonormality self-check fails.  Host code, no allocation
// on the device.
bool daubechies_filter(int nv, double* h);

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
pat_status cuda_fail(cudaError_t e, const char* what);

#define PAT_TRY_CUDA(expr)                                       \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return ::pat::cuda_fail(_e, #expr);   \
  } while (0)

#define PAT_TRY(expr)                       \
  do {                                      \
    pat_status _s = (expr);                 \
    if (_s != PAT_OK) return _s;            \
  } while (0)

// ------------------------------------------------------- device structs
// One sensor's bilinear sampling entry inside a persistent 2D tile.
// A sensor whose 2x2 interpolation block straddles four tiles (its base cell
// is a tile's last row and column) cannot be read from one tile's cross-shaped
// halo; each of its four cells is then sampled by the tile that owns it into
// part[(4*q + corner)*nt + t] and a small kernel sums the four afterwards.
struct SampEntry {
  int sensor;
  int part;      // -1: whole sensor sampled here; else 4*q + corner of a split sensor
  short lx, ly;  // base cell (or the split corner's cell) in tile-local coordinates
  float w[4];    // weights of (lx,ly), (lx+1,ly), (lx,ly+1), (lx+1,ly+1); split: w[0] only
};

// One injected cell inside a persistent 2D tile: entries [beg, end) of the
// plan's (sensor, weight) list, summed in that order.
struct InjCell {
  int local;  // ly * TX + lx
  int beg, end;
};

// Arguments of the persistent 2D wave kernel.
struct Persist2DArgs {
  int nx, ny, nt;
  int tiles_x, tiles_y;
  float w[kMaxR + 1];  // composed stencil weights, w[1..R]
  float kappa0;        // (c dt / h)^2 when the medium is constant
  float kappa0_lo;     // kappa0 - fl(kappa0) (rounding residual)
  const float* kappa;  // per-cell kappa, or nullptr
  const float* kappa_lo;  // per-cell rounding residual of kappa, or nullptr
  const float* in;     // forward: x (N);  adjoint: y (ns*nt)
  float* out;          // forward: y;      adjoint: x
  const int* tile_samp_ptr;
  const SampEntry* samp;
  float* part;  // split-sensor partial samples (4 x nt per split sensor)
  const int* tile_inj_ptr;
  const InjCell* inj;
  const int* ent_sensor;
  const float* ent_w;
  void* xbuf;            // tagged boundary strips (64-bit words), 2 slots per tile
  int* abort;            // set when any CTA gives up
  int* status;           // sticky plan status
  long long timeout_ns;  // bound on any single wait
  int poll_ns;           // back-off between polls of the exchange (0 = spin)
  const float* sp_a;     // absorbing layer: per-cell factors a, b of the damped update (nullptr = none)
  const float* sp_b;
  // second right-hand side (the two-field kernel only)
  const float* in1;
  float* out1;
  float* part1;
};

// Arguments of the per-step kernels.
//   2D (increment form): d = (d_zero ? 0 : dbuf) + c_lap kappa L cur, dbuf = d,
//      next = cur + d; with final = 1 (adjoint's last step) next = dbuf + c_lap L(kappa cur).
//   3D (three-level form): next = c_cur cur - c_prev prev + c_lap kappa L cur
//      (adjoint: L(kappa cur)).
//   2D adjoint carries compensation terms in cur_lo/next_lo (and dbuf_lo): the TMA kernel keeps
//      the state Z = kappa Q with its low part in cur_lo/next_lo (G plain); the plain kernel keeps
//      Q with Q_lo there and G_lo in dbuf_lo, feeding the stencil kappa*Q as a hi + lo pair.
struct StepArgs {
  int nx, ny, nz;
  float w[kMaxR + 1];
  float kappa0, kappa0_lo;
  const float* kappa;     // or nullptr
  const float* kappa_lo;  // rounding residual of kappa, or nullptr
  const float* cur;    // P^n (forward) or Q^{n+1} (adjoint)
  const float* cur_lo;  // 2D adjoint: compensation of Q^{n+1} (Z^{n+1} on the TMA kernel)
  float* next_lo;       // 2D adjoint: compensation of Q^n (Z^n on the TMA kernel)
  float* dbuf_lo;       // 2D adjoint, plain kernel: compensation of G
  const float* prev;   // 3D: P^{n-1} or Q^{n+2}   (nullptr = 0)
  float* dbuf;         // 2D: increment D (forward) / G (adjoint), updated in place
  int d_zero;          // 2D: treat the incoming increment as 0
  int final_step;      // 2D adjoint: next = dbuf + c_lap L(kappa cur)
  float* next;         // P^{n+1} or Q^n (or the adjoint's result)
  float c_lap;         // coefficient of kappa*L (1, or 0.5 for the first/last step)
  float c_cur;         // 3D: coefficient of the current field (2, or 1)
  float c_prev;        // 3D: coefficient of the previous field (1, or 0)
  // fused sampling of `cur` (forward): y[s*nt + t_sample] for s in [0, ns)
  int ns, nt, t_sample;
  const int* sens_cell;
  const float* sens_w;
  int corners;
  float* y;
  // Adjoint injection S^T r_{inj_t} (nullptr = none): 2D, into dbuf by a separate injection launch
  // before the step; 3D, fused after the step through per-CTA lists (inj_tile_ptr / inj_tile).
  // 2D absorbing layer (nullptr = none): per-cell factors a, b of the damped update and the layer
  // width in cells (tiles farther than that from every face skip the factors)
  const float* sp_a;
  const float* sp_b;
  int sp_w;
  const float* inj_r;
  int inj_t;
  const int* inj_tile_ptr;
  const InjCell* inj_tile;
  const int* ent_sensor;
  const float* ent_w;
};

// ------------------------------------------------------------ launchers
// wave2d_persist.cu
bool persist2d_supported(int R, bool varc);
int persist2d_tile_x();
int persist2d_tile_y();
size_t persist2d_smem_bytes(int R, bool adj);
size_t persist2d_xbuf_words(int R, bool adj, int ntiles, int nr = 1);  // 64-bit exchange words, nr fields
int persist2d_max_ctas(int R, bool adj, bool varc);  // co-resident CTA limit on this device
cudaError_t persist2d_launch(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st);
// Two right-hand sides per launch (no absorbing layer): a.in / a.out and a.in1 / a.out1.
int persist2d_max_ctas2(int R, bool adj, bool varc);
cudaError_t persist2d_launch2(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st);
// the same with the absorbing layer (a.sp_a, a.sp_b set)
cudaError_t persist2d_launch_layer(int R, bool adj, bool varc, const Persist2DArgs& a, int nctas, cudaStream_t st);
cudaError_t persist2d_split_combine(const float* part, const int* split_sensor, int nsplit, int nt, float* y,
                                    cudaStream_t st);

// wave3d_tma.cu: constant-medium 3D step with TMA plane pipelines
bool tma3d_supported(int nx, int R, bool varc);
// `cur` (80 x (16+2R) x 1 boxes) and `prev` (64 x 16 x 1) descriptors of an nx x ny x nz float field
cudaError_t tma3d_encode(const float* base, int nx, int ny, int nz, int R, CUtensorMap* cur, CUtensorMap* prev);
// Work split of a 3D TMA step launch: nctas = columns x nchunks CTAs, column-fastest, each a z range
// of nz / nchunks planes; ring: the kernel form whose z queue is a register ring (one-wave grids).
struct Tma3dSplit {
  int nctas, nchunks;
  bool ring;
};
Tma3dSplit tma3d_split(int R, int nx, int ny, int nz);
int tma3d_cta_of(int nx, int ny, int nz, const Tma3dSplit& sp, int x, int y, int z);  // CTA holding a cell
long long tma3d_threads(int nctas);  // threads of one launch (fused sampling)
cudaError_t step3d_tma_launch(int R, const StepArgs& a, const CUtensorMap& cur, const CUtensorMap& prev, const Tma3dSplit& sp,
                              int* status, long long timeout_ns, cudaStream_t st);

// wave2d_tma.cu: 2D increment-form step with TMA tile pipelines (forward; constant-medium adjoint)
bool tma2d_supported(int nx, int R);
// P boxes (80 x (64+2R)) and own-tile boxes (64 x 64) of an nx x ny float field
cudaError_t tma2d_encode(const float* base, int nx, int ny, int R, CUtensorMap* halo, CUtensorMap* own);
// mode 0: constant medium, 1: varying medium (forward), 2: constant medium with fused injection (adjoint),
// 3: varying-medium adjoint (k: kappa's halo-box descriptor, unused by the other modes);
// sp 0: no absorbing layer, 1: layer with the forward update, 2: layer with the adjoint update
long long tma2d_threads(int nx, int ny, int R, int mode, int sp);  // threads of one launch (fused sampling)
cudaError_t step2d_tma_launch(int R, int mode, int sp, const StepArgs& a, const CUtensorMap& p, const CUtensorMap& k,
                              int* status, long long timeout_ns, cudaStream_t st);

// wave_step.cu
cudaError_t step2d_launch(int R, bool adj, const StepArgs& a, cudaStream_t st);
cudaError_t step3d_launch(int R, bool adj, const StepArgs& a, cudaStream_t st);
cudaError_t sample_launch(const float* P, int ns, int nt, int t, const int* cell, const float* w, int corners,
                          float* y, cudaStream_t st);
cudaError_t inject_launch(float* Q, int n_inj, const int* inj_cell, const int* inj_ptr, const int* ent_sensor,
                          const float* ent_w, const float* r, int nt, int t, float scale, cudaStream_t st);
// zform: the adjoint state holds Z = kappa Q (2D TMA engine); the accumulator divides by kappa
cudaError_t grad_acc_launch(int R, double* gacc, const float* Q, const float* Qlo, const float* P, float coef,
                            const StepArgs& a, int dim, bool zform, cudaStream_t st);
cudaError_t d2f_launch(float* out, const double* in, long long n, cudaStream_t st);
cudaError_t dfill_launch(double* p, long long n, cudaStream_t st);
cudaError_t fill_launch(float* p, long long n, float v, cudaStream_t st);
cudaError_t copy_launch(float* dst, const float* src, long long n, cudaStream_t st);

// dwt.cu
cudaError_t dwt2d_analysis_level(const float* in, int nx, int ny, float* approx, float* bandH, float* bandV,
                                 float* bandD, float wdet, const float* h, const float* g, int L, cudaStream_t st);
cudaError_t dwt2d_synthesis_level(const float* approx, const float* bandH, const float* bandV, const float* bandD,
                                  float wdet, int nx, int ny, float* out, const float* h, const float* g, int L,
                                  cudaStream_t st);
cudaError_t dwt1d_analysis_axis(const float* in, int n0, int n1, int n2, int axis, float* lo, float* hi, float wlo,
                                float whi, const float* h, const float* g, int L, cudaStream_t st);
cudaError_t dwt1d_synthesis_axis(const float* lo, const float* hi, float wlo, float whi, int n0, int n1, int n2,
                                 int axis, float* out, const float* h, const float* g, int L, cudaStream_t st);
// One fused 3D level (band pointers in code order zb << 2 | yb << 1 | xb, code 0 =
// approximation); cudaErrorNotSupported (nothing launched) when nx % 8 != 0 or
// an address is not 16-byte aligned, for the separable passes to take over.
cudaError_t dwt3d_analysis_level(const float* in, int nx, int ny, int nz, float* const bands[8], float wdet,
                                 const float* h, const float* g, int L, cudaStream_t st);
cudaError_t dwt3d_synthesis_level(const float* const bands[8], float wdet, int nx, int ny, int nz, float* out,
                                  const float* h, const float* g, int L, cudaStream_t st);
cudaError_t scale_copy_launch(float* dst, const float* src, long long n, float w, cudaStream_t st);

// cg.cu
struct CgScalars {
  double rr, pq, a, rr_new, beta;
  int stopped;
  int iter;
};
int cg_grid_blocks();
cudaError_t cg_init_launch(const float* b, float* r, float* p, float* u, long long n, bool zero_u, double* partials,
                           unsigned* counter, CgScalars* sc, cudaStream_t st);
cudaError_t cg_sub_launch(float* r, const float* q, long long n, cudaStream_t st);  // r -= q
cudaError_t cg_pq_launch(float* q, const float* p, double alpha, long long n, double* partials, unsigned* counter,
                         CgScalars* sc, cudaStream_t st);
cudaError_t cg_update_launch(float* u, float* r, const float* p, const float* q, long long n, double* partials,
                             unsigned* counter, CgScalars* sc, double* log, int* status, cudaStream_t st);
cudaError_t cg_direction_launch(float* p, const float* r, long long n, const CgScalars* sc, cudaStream_t st);
cudaError_t cg_rr_launch(const float* r, float* p, long long n, double* partials, unsigned* counter, CgScalars* sc,
                         cudaStream_t st);  // p = r, rr = r.r

}  // namespace pat
