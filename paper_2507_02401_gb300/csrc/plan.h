// Definition of the opaque plan object behind the C ABI.
#pragma once

#include <vector>

#include "internal.h"

struct pat_plan {
  // ---- problem
  int dim = 2;
  int n[3] = {1, 1, 1};  // nx, ny, nz
  long long N = 0;
  double h = 0, dt = 0;
  int nt = 0, order = 2, M = 1, R = 1, ns = 0, corners = 4;
  double c_max = 0;
  bool varc = false;
  float kappa0 = 0.f;
  float kappa0_lo = 0.f;  // rounding residual of kappa0
  float* d_kappa = nullptr;
  float* d_kappa_lo = nullptr;  // rounding residual of kappa (varying medium)
  float w[pat::kMaxR + 1] = {0};  // composed stencil weights w[1..R]

  // ---- sensors: sampling (ns x corners) and the transposed injection CSR
  int* d_sens_cell = nullptr;
  float* d_sens_w = nullptr;
  std::vector<int> h_sens_cell;
  std::vector<float> h_sens_w;
  int n_inj = 0;
  int* d_inj_cell = nullptr;
  int* d_inj_ptr = nullptr;
  int* d_ent_sensor = nullptr;
  float* d_ent_w = nullptr;
  std::vector<int> h_inj_cell, h_inj_ptr;

  // ---- wavelet
  int family = 1, L = 2, levels = 1, level_offset = 0;
  float hf[pat::kMaxTaps] = {0}, gf[pat::kMaxTaps] = {0};

  // ---- wave engine
  int path = PAT_PATH_STEP;       // engine in use
  bool persist_ok = false;        // persistent engine available for this plan
  int tiles_x = 0, tiles_y = 0, ntiles = 0;
  int* d_tile_samp_ptr = nullptr;
  pat::SampEntry* d_samp = nullptr;
  int nsplit = 0;                 // sensors sampled as four per-tile parts
  int* d_split_sensor = nullptr;
  float* d_part = nullptr;
  int* d_tile_inj_ptr = nullptr;
  pat::InjCell* d_tinj = nullptr;
  void* d_xbuf = nullptr;  // tagged 64-bit exchange words
  size_t xbuf_bytes = 0;
  int* d_abort = nullptr;
  long long timeout_ns = 2000000000LL;
  int poll_ns = 0;  // exchange polling back-off
  float* d_wv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // per-step engine fields
  // absorbing layer (2D): width in cells (0 = none), damping rate at the faces [1/s], per-cell factors
  int sponge_w = 0;
  double sponge_sigma_max = 0.0;
  float* d_sp_a = nullptr;
  float* d_sp_b = nullptr;
  bool tma3d = false;  // 3D steps through the TMA plane-pipeline kernel
  pat::Tma3dSplit tma3d_split{0, 0};  // work split of a 3D TMA step launch
  bool tma2d = false;  // 2D steps through the TMA tile-pipeline kernel (where it applies)
  int* d_tinj3_ptr = nullptr;       // 3D TMA kernel: injection lists per CTA (64 x 16 columns x z chunk)
  pat::InjCell* d_tinj3 = nullptr;  // .local = linear cell index
  struct TmaDesc {
    const float* base;
    CUtensorMap halo, own;  // stencil-input boxes with halo, own-tile boxes
  };
  std::vector<TmaDesc> tma_desc;  // descriptors by field address (small, most recent last)

  // ---- Fourier-form prior (kind 1 of pat_plan_set_prior): lengths in units of fourier_lc cells
  int prior = 0;
  double fourier_lc = 1.0;
  float2* d_fc = nullptr;  // two complex N-buffers (spectrum and its transpose)
  float2* d_tw = nullptr;  // twiddle tables of the x and y transforms

  // ---- wavelet scratch
  float* d_dwt_a = nullptr;  // approximation ping-pong (2 x N/2^dim)
  float* d_dwt_b = nullptr;
  float* d_dwt_t1 = nullptr;  // 3D separable-pass intermediates (N each)
  float* d_dwt_t2 = nullptr;

  // ---- solver workspace
  float *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_img = nullptr, *d_u = nullptr, *d_ybuf = nullptr;
  pat::CgScalars* d_sc = nullptr;
  // second right-hand side of pat_solve_multi (allocated on first use): CG vectors, data and image
  // buffers, split-sensor parts and the two-field exchange strips
  struct Rhs2 {
    float *r = nullptr, *p = nullptr, *q = nullptr, *img = nullptr, *u = nullptr, *ybuf = nullptr, *part = nullptr;
    pat::CgScalars* sc = nullptr;
    double* partials = nullptr;
    unsigned* counter = nullptr;
    void* xbuf = nullptr;
    size_t xbuf_bytes = 0;
    bool ready = false;
    bool two_field = false;  // the two-field persistent kernel fits (both directions)
  } m2;
  double* d_partials = nullptr;
  unsigned* d_counter = nullptr;
  int* d_status = nullptr;
  double* d_kr = nullptr;  // GMRES / Landweber reduction partials (allocated on first use)

  // ---- staging for host arrays
  float* d_stage[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t stage_bytes[4] = {0, 0, 0, 0};

  // ---- medium-gradient workspace (allocated by the first pat_grad_kappa call)
  int kg_segment = 0;           // checkpoint interval the buffers were sized for
  float* kg_ckpt = nullptr;     // per checkpoint: two fields (P and D, or P and P^{n-1})
  float* kg_seg = nullptr;      // one segment of recomputed fields
  float* kg_work = nullptr;     // forward-pass fields (3 x N)
  double* kg_acc = nullptr;     // FP64 gradient accumulator

  // ---- measurement hooks
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // start/stop pairs
  int prof_used = 0;                 // events used (2 per wave application)
  long long prof_kernels = 0;
  long long prof_points = 0;

  std::vector<void*> allocations;
};

namespace pat {
pat_status plan_alloc(pat_plan* p, void** ptr, size_t bytes, const char* what);
pat_status wave_forward(pat_plan* p, const float* x, float* y, cudaStream_t st);
pat_status wave_adjoint(pat_plan* p, const float* y, float* x, cudaStream_t st);
pat_status apply_Es(pat_plan* p, double s, const float* u, float* x, cudaStream_t st);
pat_status apply_EsT(pat_plan* p, double s, const float* x, float* u, cudaStream_t st);
pat_status solve_device(pat_plan* p, const float* y, double alpha, double s, int iters, const float* u0, float* u,
                        float* x, double* log, cudaStream_t st);
pat_status kappa_grad_device(pat_plan* p, const float* x, const float* r, float* g, int segment, cudaStream_t st);
bool fourier_supported(int dim, int nx, int ny);
pat_status fourier_setup(pat_plan* p, double length_cells, cudaStream_t st);
pat_status fourier_apply(pat_plan* p, double s, const float* in, float* out, cudaStream_t st);
// J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 into *J (host) and, if grad, its gradient (device, N).
pat_status objective_device(pat_plan* p, const float* y, double alpha, double s, const float* u, double* J,
                            float* grad, cudaStream_t st);
// CG of nrhs problems on one plan (own data, alpha, s), two at a time per wave launch on the persistent engine.
pat_status solve_multi_device(pat_plan* p, int nrhs, const float* const* ys, const double* alphas, const double* ss,
                              int iters, float* const* xs, cudaStream_t st);
pat_status landweber_device(pat_plan* p, const float* y, double alpha, double s, int iters, double omega, float* u,
                            float* x, double* J, cudaStream_t st);
pat_status gmres_device(pat_plan* p, const float* y, double alpha, double s, int iters, float* x, double* res,
                        double* J, cudaStream_t st);
}  // namespace pat
