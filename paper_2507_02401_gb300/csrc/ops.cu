// Operators and solver behind the C ABI: K, K*, E_s, E_s*, CG.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch.h"
#include "plan.h"

namespace pat {

// ------------------------------------------------------------------- K, K*
static Persist2DArgs persist_args(pat_plan* p) {
  Persist2DArgs a{};
  a.nx = p->n[0];
  a.ny = p->n[1];
  a.nt = p->nt;
  a.tiles_x = p->tiles_x;
  a.tiles_y = p->tiles_y;
  for (int m = 0; m <= kMaxR; ++m) a.w[m] = p->w[m];
  a.kappa0 = p->kappa0;
  a.kappa0_lo = p->kappa0_lo;
  a.kappa = p->varc ? p->d_kappa : nullptr;
  a.kappa_lo = p->varc ? p->d_kappa_lo : nullptr;
  a.tile_samp_ptr = p->d_tile_samp_ptr;
  a.samp = p->d_samp;
  a.part = p->d_part;
  a.tile_inj_ptr = p->d_tile_inj_ptr;
  a.inj = p->d_tinj;
  a.ent_sensor = p->d_ent_sensor;
  a.ent_w = p->d_ent_w;
  a.xbuf = p->d_xbuf;
  a.abort = p->d_abort;
  a.status = p->d_status;
  a.timeout_ns = p->timeout_ns;
  a.poll_ns = p->poll_ns;
  if (p->sponge_w > 0) {
    a.sp_a = p->d_sp_a;
    a.sp_b = p->d_sp_b;
  }
  return a;
}

// One persistent launch: the exchange words are invalidated (no valid tag) and
// the abort flag cleared on the stream first.
static pat_status persist_launch(pat_plan* p, bool adj, const Persist2DArgs& a, cudaStream_t st) {
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_xbuf, 0xff, p->xbuf_bytes, st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_abort, 0, sizeof(int), st));
  if (p->sponge_w > 0)
    PAT_TRY_CUDA(persist2d_launch_layer(p->R, adj, p->varc, a, p->ntiles, st));
  else
    PAT_TRY_CUDA(persist2d_launch(p->R, adj, p->varc, a, p->ntiles, st));
  return PAT_OK;
}

static StepArgs step_args(pat_plan* p) {
  StepArgs a{};
  a.nx = p->n[0];
  a.ny = p->n[1];
  a.nz = p->n[2];
  for (int m = 0; m <= kMaxR; ++m) a.w[m] = p->w[m];
  a.kappa0 = p->kappa0;
  a.kappa0_lo = p->kappa0_lo;
  a.kappa = p->varc ? p->d_kappa : nullptr;
  a.kappa_lo = p->varc ? p->d_kappa_lo : nullptr;
  a.ns = p->ns;
  a.nt = p->nt;
  a.sens_cell = p->d_sens_cell;
  a.sens_w = p->d_sens_w;
  a.corners = p->corners;
  if (p->sponge_w > 0) {
    a.sp_a = p->d_sp_a;
    a.sp_b = p->d_sp_b;
    a.sp_w = p->sponge_w;
  }
  return a;
}

// Tensor-map descriptors of a field, encoded on first use and kept per address.
static const pat_plan::TmaDesc* tma_desc(pat_plan* p, const float* base) {
  for (auto& d : p->tma_desc)
    if (d.base == base) return &d;
  pat_plan::TmaDesc d;
  d.base = base;
  const cudaError_t e = p->dim == 3 ? tma3d_encode(base, p->n[0], p->n[1], p->n[2], p->R, &d.halo, &d.own)
                                     : tma2d_encode(base, p->n[0], p->n[1], p->R, &d.halo, &d.own);
  if (e != cudaSuccess) return nullptr;
  if (p->tma_desc.size() >= 16) p->tma_desc.erase(p->tma_desc.begin());
  p->tma_desc.push_back(d);
  return &p->tma_desc.back();
}

// The TMA kernels take 16-byte aligned fields (descriptor bases, float4 stores).
static bool tma_ready(pat_plan* p, const StepArgs& a) {
  auto al = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
  return al(a.cur) && al(a.prev) && al(a.next) && (p->dim == 3 || (al(a.dbuf) && al(a.cur_lo) && al(a.next_lo)));
}

static cudaError_t step_launch(pat_plan* p, bool adj, StepArgs& a, cudaStream_t st) {
  // sample separately when the step grid has fewer threads than sensors
  float* y = a.y;
  cudaError_t e;
  if (p->dim == 2 && p->tma2d && tma_ready(p, a)) {
    // TMA tile pipelines: forward (constant or varying medium); adjoint in Z = kappa Q with Z
    // compensated (boxes of Z and Z_lo), its injection S^T r_m added to G by a launch just before
    const int mode = adj ? 2 : (p->varc ? 1 : 0);
    const int sp = p->sponge_w > 0 ? (adj ? 2 : 1) : 0;
    const long long nthr = tma2d_threads(p->n[0], p->n[1], p->R, mode, sp);
    if (y && a.ns > nthr) a.y = nullptr;
    // copies: a second lookup may move the cached descriptors
    const pat_plan::TmaDesc* dp = tma_desc(p, a.cur);
    if (!dp) return cudaErrorInvalidValue;
    const CUtensorMap mcur = dp->halo;
    CUtensorMap mlo = mcur;
    if (adj) {
      const pat_plan::TmaDesc* dl = tma_desc(p, a.cur_lo);
      if (!dl) return cudaErrorInvalidValue;
      mlo = dl->halo;
    }
    StepArgs b = a;
    if (!p->varc) b.kappa = b.kappa_lo = nullptr;
    if (a.inj_r) {
      e = inject_launch(a.dbuf, p->n_inj, p->d_inj_cell, p->d_inj_ptr, p->d_ent_sensor, p->d_ent_w, a.inj_r, p->nt,
                        a.inj_t, 1.f, st);
      if (e != cudaSuccess) return e;
      b.inj_r = nullptr;
    }
    e = step2d_tma_launch(p->R, mode, sp, b, mcur, mlo, p->d_status, p->timeout_ns, st);
  } else if (p->dim == 2) {
    const long long nthr = (long long)((p->n[0] + 63) / 64) * ((p->n[1] + 31) / 32) * 256;
    if (y && a.ns > nthr) a.y = nullptr;
    if (a.inj_r) {
      e = inject_launch(a.dbuf, p->n_inj, p->d_inj_cell, p->d_inj_ptr, p->d_ent_sensor, p->d_ent_w, a.inj_r, p->nt,
                        a.inj_t, 1.f, st);
      if (e != cudaSuccess) return e;
    }
    StepArgs b = a;
    b.inj_r = nullptr;
    e = step2d_launch(p->R, adj, b, st);
  } else if (p->tma3d && tma_ready(p, a)) {
    const long long nthr = tma3d_threads(p->tma3d_split.nctas);
    if (y && a.ns > nthr) a.y = nullptr;
    if (a.inj_r) {  // the adjoint's post-step injection, fused per CTA
      a.inj_tile_ptr = p->d_tinj3_ptr;
      a.inj_tile = p->d_tinj3;
      a.ent_sensor = p->d_ent_sensor;
      a.ent_w = p->d_ent_w;
    }
    CUtensorMap mc, mp;
    const pat_plan::TmaDesc* dc = tma_desc(p, a.cur);
    if (!dc) return cudaErrorInvalidValue;
    mc = dc->halo;
    mp = dc->own;  // unused when there is no previous field
    if (a.prev) {
      const pat_plan::TmaDesc* dp = tma_desc(p, a.prev);
      if (!dp) return cudaErrorInvalidValue;
      mp = dp->own;
    }
    e = step3d_tma_launch(p->R, a, mc, mp, p->tma3d_split, p->d_status, p->timeout_ns, st);
  } else {
    const long long nthr =
        (long long)((p->n[0] + 31) / 32) * ((p->n[1] + 15) / 16) * ((p->n[2] + 31) / 32) * 128;
    if (y && a.ns > nthr) a.y = nullptr;
    StepArgs b = a;
    b.inj_r = nullptr;
    e = step3d_launch(p->R, adj, b, st);
    if (e == cudaSuccess && a.inj_r)  // the adjoint's injection after the step
      e = inject_launch(a.next, p->n_inj, p->d_inj_cell, p->d_inj_ptr, p->d_ent_sensor, p->d_ent_w, a.inj_r, p->nt,
                        a.inj_t, 1.f, st);
  }
  if (e == cudaSuccess && y && !a.y)
    e = sample_launch(a.cur, p->ns, p->nt, a.t_sample, p->d_sens_cell, p->d_sens_w, p->corners, y, st);
  a.y = y;
  return e;
}

static pat_status wave_forward_impl(pat_plan* p, const float* x, float* y, cudaStream_t st) {
  if (p->path == PAT_PATH_PERSISTENT) {
    Persist2DArgs a = persist_args(p);
    a.in = x;
    a.out = y;
    PAT_TRY(persist_launch(p, false, a, st));
    PAT_TRY_CUDA(persist2d_split_combine(p->d_part, p->d_split_sensor, p->nsplit, p->nt, y, st));
    return PAT_OK;
  }
  const int nt = p->nt;
  if (nt == 1) {
    PAT_TRY_CUDA(sample_launch(x, p->ns, nt, 0, p->d_sens_cell, p->d_sens_w, p->corners, y, st));
    return PAT_OK;
  }
  StepArgs a = step_args(p);
  a.y = y;
  if (p->dim == 2) {
    // increment form: F_0 = x, F_n = wv[(n-1) % 2], D = wv[2]; step n makes F_{n+1}, samples F_n
    a.dbuf = p->d_wv[2];
    for (int n = 0; n < nt - 1; ++n) {
      a.cur = (n == 0) ? x : p->d_wv[(n - 1) % 2];
      a.next = p->d_wv[n % 2];
      a.d_zero = (n == 0);
      a.c_lap = (n == 0) ? 0.5f : 1.f;
      a.t_sample = n;
      PAT_TRY_CUDA(step_launch(p, false, a, st));
    }
    PAT_TRY_CUDA(sample_launch(p->d_wv[(nt - 2) % 2], p->ns, nt, nt - 1, p->d_sens_cell, p->d_sens_w, p->corners,
                               y, st));
    return PAT_OK;
  }
  // three-level form: F_0 = x, F_n = wv[(n-1) % 3]
  for (int n = 0; n < nt - 1; ++n) {
    a.cur = (n == 0) ? x : p->d_wv[(n - 1) % 3];
    a.prev = (n == 0) ? nullptr : (n == 1 ? x : p->d_wv[(n - 2) % 3]);
    a.next = p->d_wv[n % 3];
    a.c_cur = (n == 0) ? 1.f : 2.f;
    a.c_prev = (n == 0) ? 0.f : 1.f;
    a.c_lap = (n == 0) ? 0.5f : 1.f;
    a.t_sample = n;
    PAT_TRY_CUDA(step_launch(p, false, a, st));
  }
  PAT_TRY_CUDA(sample_launch(p->d_wv[(nt - 2) % 3], p->ns, nt, nt - 1, p->d_sens_cell, p->d_sens_w, p->corners, y, st));
  return PAT_OK;
}

static pat_status wave_adjoint_impl(pat_plan* p, const float* y, float* x, cudaStream_t st) {
  if (p->path == PAT_PATH_PERSISTENT) {
    Persist2DArgs a = persist_args(p);
    a.in = y;
    a.out = x;
    PAT_TRY(persist_launch(p, true, a, st));
    return PAT_OK;
  }
  const int nt = p->nt;
  auto inject = [&](float* Q, int t) {
    return inject_launch(Q, p->n_inj, p->d_inj_cell, p->d_inj_ptr, p->d_ent_sensor, p->d_ent_w, y, nt, t, 1.f, st);
  };
  if (nt == 1) {
    PAT_TRY_CUDA(fill_launch(x, p->N, 0.f, st));
    PAT_TRY_CUDA(inject(x, 0));
    return PAT_OK;
  }
  StepArgs a = step_args(p);
  a.y = nullptr;
  if (p->dim == 2) {
    // increment form with compensation: G = wv[2] (+ wv[5]); Q^m in wv[(nt-m) % 2]
    // (+ wv[3 + (nt-m) % 2]) with Q^nt = 0.  The TMA kernel keeps Z = kappa Q there (and no G_lo);
    // the plain kernel Q itself, so every step of one application runs on the same kernel: with
    // the TMA kernel an output that is not 16-byte aligned is written to a free field buffer
    // (Q^2's, no longer read by the final step) and copied.
    float* G = p->d_wv[2];
    auto Qbuf = [&](int m) { return p->d_wv[(nt - m) % 2]; };
    auto Qlo = [&](int m) { return p->d_wv[3 + (nt - m) % 2]; };
    PAT_TRY_CUDA(fill_launch(G, p->N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(p->d_wv[5], p->N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(Qbuf(nt), p->N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(Qlo(nt), p->N, 0.f, st));
    a.dbuf = G;
    a.dbuf_lo = p->d_wv[5];
    a.inj_r = y;  // G^{m+1} + S^T r_m, injected by (or just before) each step
    for (int m = nt - 1; m >= 1; --m) {
      a.inj_t = m;
      a.cur = Qbuf(m + 1);
      a.cur_lo = Qlo(m + 1);
      a.next = Qbuf(m);
      a.next_lo = Qlo(m);
      a.d_zero = 0;
      a.final_step = 0;
      a.c_lap = 1.f;
      PAT_TRY_CUDA(step_launch(p, true, a, st));
    }
    a.inj_t = 0;
    a.cur = Qbuf(1);
    a.cur_lo = Qlo(1);
    const bool staged = p->tma2d && ((uintptr_t)x & 15) != 0;
    a.next = staged ? Qbuf(2) : x;
    a.next_lo = nullptr;
    a.final_step = 1;
    a.c_lap = 0.5f;
    PAT_TRY_CUDA(step_launch(p, true, a, st));
    if (staged) PAT_TRY_CUDA(cudaMemcpyAsync(x, Qbuf(2), sizeof(float) * p->N, cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
  }
  // three-level form: Q^m lives in wv[(nt-1-m) % 3]
  auto Qbuf = [&](int m) { return p->d_wv[(nt - 1 - m) % 3]; };
  PAT_TRY_CUDA(fill_launch(Qbuf(nt - 1), p->N, 0.f, st));
  PAT_TRY_CUDA(inject(Qbuf(nt - 1), nt - 1));
  a.inj_r = y;  // S^T r_m added to Q^m by (or just after) the step that makes it
  for (int m = nt - 2; m >= 1; --m) {
    a.cur = Qbuf(m + 1);
    a.prev = (m + 2 <= nt - 1) ? Qbuf(m + 2) : nullptr;
    a.next = Qbuf(m);
    a.c_cur = 2.f;
    a.c_prev = 1.f;
    a.c_lap = 1.f;
    a.inj_t = m;
    PAT_TRY_CUDA(step_launch(p, true, a, st));
  }
  a.cur = Qbuf(1);
  a.prev = (nt >= 3) ? Qbuf(2) : nullptr;
  a.next = x;
  a.c_cur = 1.f;
  a.c_prev = 1.f;
  a.c_lap = 0.5f;
  a.inj_t = 0;
  PAT_TRY_CUDA(step_launch(p, true, a, st));
  return PAT_OK;
}

// ------------------------------------------------------- measurement hooks
static pat_status prof_mark(pat_plan* p, cudaStream_t st) {
  if ((int)p->prof_ev.size() <= p->prof_used) {
    cudaEvent_t e;
    PAT_TRY_CUDA(cudaEventCreate(&e));
    p->prof_ev.push_back(e);
  }
  PAT_TRY_CUDA(cudaEventRecord(p->prof_ev[p->prof_used++], st));
  return PAT_OK;
}

static long long wave_kernels(const pat_plan* p, bool adj) {
  if (p->path == PAT_PATH_PERSISTENT) return (!adj && p->nsplit > 0) ? 2 : 1;
  const long long nt = p->nt;
  if (nt == 1) return adj ? 2 : 1;
  if (!adj) return nt;  // nt-1 steps + final sample
  const long long inj = p->n_inj > 0 ? 1 : 0;
  if (p->dim == 2) return 4 + (nt - 1) * (1 + inj) + (1 + inj);  // 4 fills, (inject+step) x (nt-1), final
  if (p->tma3d) return (1 + inj) + (nt - 2) + 1;                   // fill+inject, steps with fused injection
  return (1 + inj) + (nt - 2) * (1 + inj) + (1 + inj);             // fill+inject, (step+inject), final
}

pat_status wave_forward(pat_plan* p, const float* x, float* y, cudaStream_t st) {
  if (p->prof_on) PAT_TRY(prof_mark(p, st));
  PAT_TRY(wave_forward_impl(p, x, y, st));
  if (p->prof_on) {
    PAT_TRY(prof_mark(p, st));
    p->prof_kernels += wave_kernels(p, false);
    p->prof_points += p->N * (long long)(p->nt - 1);
  }
  return PAT_OK;
}

pat_status wave_adjoint(pat_plan* p, const float* y, float* x, cudaStream_t st) {
  if (p->prof_on) PAT_TRY(prof_mark(p, st));
  PAT_TRY(wave_adjoint_impl(p, y, x, st));
  if (p->prof_on) {
    PAT_TRY(prof_mark(p, st));
    p->prof_kernels += wave_kernels(p, true);
    p->prof_points += p->N * (long long)(p->nt - 1);
  }
  return PAT_OK;
}

static void count_kernels(pat_plan* p, long long k) {
  if (p->prof_on) p->prof_kernels += k;
}

// ------------------------------------------------------------- E_s, E_s*
static float level_weight(const pat_plan* p, int i, double s) {
  return (float)std::pow(2.0, -s * (double)(p->levels - i + p->level_offset));
}

// offset of band b (0-based) of level i in the coefficient vector
static long long band_offset(const pat_plan* p, int i, int b) {
  const int d = p->dim;
  const int nb = (1 << d) - 1;
  long long off = p->N >> (d * p->levels);
  for (int j = p->levels; j > i; --j) off += (long long)nb * (p->N >> (d * j));
  return off + (long long)b * (p->N >> (d * i));
}

pat_status apply_EsT(pat_plan* p, double s, const float* x, float* u, cudaStream_t st) {
  if (p->prior == 1) {  // Fourier form: E_s* = E_s
    count_kernels(p, 5);
    return fourier_apply(p, s, x, u, st);
  }
  const int m = p->levels;
  if (m == 0) {  // no levels: W = I, the coefficients are the image
    if (u != x) PAT_TRY_CUDA(cudaMemcpyAsync(u, x, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
  }
  float* tmp[2] = {p->d_dwt_a, p->d_dwt_b};
  const float* in = x;
  long long launched = 0;
  for (int i = 1; i <= m; ++i) {
    const int ex = p->n[0] >> (i - 1), ey = p->n[1] >> (i - 1), ez = p->n[2] >> (i - 1);
    float* approx = (i == m) ? u : tmp[i & 1];
    const float wd = level_weight(p, i, s);
    cudaError_t fused = cudaErrorNotSupported;
    if (p->dim == 3) {
      float* bands[8] = {approx};
      for (int c = 1; c < 8; ++c) bands[c] = u + band_offset(p, i, c - 1);
      fused = dwt3d_analysis_level(in, ex, ey, ez, bands, wd, p->hf, p->gf, p->L, st);
      if (fused != cudaErrorNotSupported) PAT_TRY_CUDA(fused);
    }
    if (p->dim == 2) {
      PAT_TRY_CUDA(dwt2d_analysis_level(in, ex, ey, approx, u + band_offset(p, i, 0), u + band_offset(p, i, 1),
                                        u + band_offset(p, i, 2), wd, p->hf, p->gf, p->L, st));
      launched += 1;
    } else if (fused == cudaSuccess) {
      launched += 1;
    } else {
      launched += 7;
      const long long ni = (long long)ex * ey * ez;
      float* T1 = p->d_dwt_t1;  // x-pass: lo | hi (ni/2 each)
      float* T2 = p->d_dwt_t2;  // y-pass: 4 quarters, index xb | yb<<1
      PAT_TRY_CUDA(dwt1d_analysis_axis(in, ex, ey, ez, 0, T1, T1 + ni / 2, 1.f, 1.f, p->hf, p->gf, p->L, st));
      for (int xb = 0; xb < 2; ++xb)
        PAT_TRY_CUDA(dwt1d_analysis_axis(T1 + xb * (ni / 2), ex / 2, ey, ez, 1, T2 + (xb | 0) * (ni / 4),
                                         T2 + (xb | 2) * (ni / 4), 1.f, 1.f, p->hf, p->gf, p->L, st));
      for (int q = 0; q < 4; ++q) {
        float* lo = (q == 0) ? approx : u + band_offset(p, i, q - 1);
        float* hi = u + band_offset(p, i, (q | 4) - 1);
        PAT_TRY_CUDA(dwt1d_analysis_axis(T2 + q * (ni / 4), ex / 2, ey / 2, ez, 2, lo, hi, q == 0 ? 1.f : wd, wd,
                                         p->hf, p->gf, p->L, st));
      }
    }
    in = approx;
  }
  count_kernels(p, launched);
  return PAT_OK;
}

pat_status apply_Es(pat_plan* p, double s, const float* u, float* x, cudaStream_t st) {
  if (p->prior == 1) {
    count_kernels(p, 5);
    return fourier_apply(p, s, u, x, st);
  }
  const int m = p->levels;
  if (m == 0) {
    if (u != x) PAT_TRY_CUDA(cudaMemcpyAsync(x, u, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
  }
  float* tmp[2] = {p->d_dwt_a, p->d_dwt_b};
  const float* approx = u;
  long long launched = 0;
  for (int i = m; i >= 1; --i) {
    const int ex = p->n[0] >> (i - 1), ey = p->n[1] >> (i - 1), ez = p->n[2] >> (i - 1);
    float* out = (i == 1) ? x : tmp[i & 1];
    const float wd = level_weight(p, i, s);
    cudaError_t fused = cudaErrorNotSupported;
    if (p->dim == 3) {
      const float* bands[8] = {approx};
      for (int c = 1; c < 8; ++c) bands[c] = u + band_offset(p, i, c - 1);
      fused = dwt3d_synthesis_level(bands, wd, ex, ey, ez, out, p->hf, p->gf, p->L, st);
      if (fused != cudaErrorNotSupported) PAT_TRY_CUDA(fused);
    }
    if (p->dim == 2) {
      PAT_TRY_CUDA(dwt2d_synthesis_level(approx, u + band_offset(p, i, 0), u + band_offset(p, i, 1),
                                         u + band_offset(p, i, 2), wd, ex, ey, out, p->hf, p->gf, p->L, st));
      launched += 1;
    } else if (fused == cudaSuccess) {
      launched += 1;
    } else {
      launched += 7;
      const long long ni = (long long)ex * ey * ez;
      float* T1 = p->d_dwt_t1;
      float* T2 = p->d_dwt_t2;
      for (int q = 0; q < 4; ++q) {  // z: (code q, code q|4) -> T2 quarter q
        const float* lo = (q == 0) ? approx : u + band_offset(p, i, q - 1);
        const float* hi = u + band_offset(p, i, (q | 4) - 1);
        PAT_TRY_CUDA(dwt1d_synthesis_axis(lo, hi, q == 0 ? 1.f : wd, wd, ex / 2, ey / 2, ez / 2, 2,
                                          T2 + q * (ni / 4), p->hf, p->gf, p->L, st));
      }
      for (int xb = 0; xb < 2; ++xb)  // y: (xb, xb|2) -> T1 half xb
        PAT_TRY_CUDA(dwt1d_synthesis_axis(T2 + xb * (ni / 4), T2 + (xb | 2) * (ni / 4), 1.f, 1.f, ex / 2, ey / 2, ez,
                                          1, T1 + xb * (ni / 2), p->hf, p->gf, p->L, st));
      PAT_TRY_CUDA(dwt1d_synthesis_axis(T1, T1 + ni / 2, 1.f, 1.f, ex / 2, ey, ez, 0, out, p->hf, p->gf, p->L, st));
    }
    approx = out;
  }
  count_kernels(p, launched);
  return PAT_OK;
}

// ------------------------------------------------------- medium gradient
// g = d<r, K x>/d kappa with sqrt(nt)-style checkpointing: the forward run
// keeps the restart state every C steps, the adjoint runs backwards and, for
// each segment it reaches, the segment's fields are recomputed from its
// checkpoint so that L P^n is available in reverse order.
static void kg_free(pat_plan* p) {
  cudaFree(p->kg_ckpt);
  cudaFree(p->kg_seg);
  cudaFree(p->kg_work);
  cudaFree(p->kg_acc);
  p->kg_ckpt = p->kg_seg = p->kg_work = nullptr;
  p->kg_acc = nullptr;
  p->kg_segment = 0;
}

static pat_status kg_alloc(pat_plan* p, int C, int nseg) {
  if (p->kg_segment == C) return PAT_OK;
  kg_free(p);
  const size_t N = (size_t)p->N;
  cudaError_t e = cudaMalloc(&p->kg_ckpt, sizeof(float) * N * 2 * nseg);
  if (e == cudaSuccess) e = cudaMalloc(&p->kg_seg, sizeof(float) * N * C);
  if (e == cudaSuccess) e = cudaMalloc(&p->kg_work, sizeof(float) * N * 3);
  if (e == cudaSuccess) e = cudaMalloc(&p->kg_acc, sizeof(double) * N);
  if (e != cudaSuccess) {
    cudaGetLastError();
    kg_free(p);
    return cuda_fail(e, "cudaMalloc(gradient checkpoints)");
  }
  p->kg_segment = C;
  return PAT_OK;
}

pat_status kappa_grad_device(pat_plan* p, const float* x, const float* r, float* g, int C, cudaStream_t st) {
  const long long N = p->N;
  const int nt = p->nt;
  if (nt < 2) {
    PAT_TRY_CUDA(fill_launch(g, N, 0.f, st));
    return PAT_OK;
  }
  if (C <= 0) C = (int)std::ceil(std::sqrt((double)nt));
  if (C > nt - 1) C = nt - 1;
  const int nseg = (nt - 2) / C + 1;  // segments of n = 0 .. nt-2
  PAT_TRY(kg_alloc(p, C, nseg));
  const bool two_d = p->dim == 2;
  float* W0 = p->kg_work;
  float* W1 = p->kg_work + N;
  float* W2 = p->kg_work + 2 * N;
  auto ck = [&](int k, int f) { return p->kg_ckpt + ((size_t)k * 2 + f) * N; };
  auto seg = [&](int j) { return p->kg_seg + (size_t)j * N; };
  auto copy = [&](float* d, const float* s) {
    return cudaMemcpyAsync(d, s, sizeof(float) * N, cudaMemcpyDeviceToDevice, st);
  };
  StepArgs a = step_args(p);
  a.y = nullptr;

  // ---- forward run keeping the restart state at n = 0, C, 2C, ...
  if (two_d) {  // increment form: state (P^n, D^n)
    a.dbuf = W2;
    const float* cur = x;
    for (int n = 0; n < nt - 1; ++n) {
      if (n % C == 0) {
        PAT_TRY_CUDA(copy(ck(n / C, 0), cur));
        if (n > 0) PAT_TRY_CUDA(copy(ck(n / C, 1), W2));
      }
      a.cur = cur;
      a.next = (n % 2) ? W1 : W0;
      a.d_zero = (n == 0);
      a.c_lap = (n == 0) ? 0.5f : 1.f;
      PAT_TRY_CUDA(step_launch(p, false, a, st));
      cur = a.next;
    }
  } else {  // three-level form: state (P^n, P^{n-1})
    const float* prev = nullptr;
    const float* cur = x;
    float* bufs[3] = {W0, W1, W2};
    for (int n = 0; n < nt - 1; ++n) {
      if (n % C == 0) {
        PAT_TRY_CUDA(copy(ck(n / C, 0), cur));
        if (n > 0) PAT_TRY_CUDA(copy(ck(n / C, 1), prev));
      }
      a.cur = cur;
      a.prev = prev;
      a.next = bufs[n % 3];
      a.c_cur = (n == 0) ? 1.f : 2.f;
      a.c_prev = (n == 0) ? 0.f : 1.f;
      a.c_lap = (n == 0) ? 0.5f : 1.f;
      PAT_TRY_CUDA(step_launch(p, false, a, st));
      prev = cur;
      cur = a.next;
    }
  }

  // ---- segment k holds P^n for n in [kC, min(kC + C, nt - 1))
  int loaded = -1;
  auto load_segment = [&](int k) -> pat_status {
    const int n0 = k * C, n1 = std::min(n0 + C, nt - 1);
    StepArgs b = step_args(p);
    b.y = nullptr;
    PAT_TRY_CUDA(copy(seg(0), ck(k, 0)));
    if (two_d) {
      if (n0 > 0) PAT_TRY_CUDA(copy(W2, ck(k, 1)));
      b.dbuf = W2;
      for (int n = n0; n < n1 - 1; ++n) {
        b.cur = seg(n - n0);
        b.next = seg(n + 1 - n0);
        b.d_zero = (n == 0);
        b.c_lap = (n == 0) ? 0.5f : 1.f;
        PAT_TRY_CUDA(step_launch(p, false, b, st));
      }
    } else {
      if (n0 > 0) PAT_TRY_CUDA(copy(W0, ck(k, 1)));
      for (int n = n0; n < n1 - 1; ++n) {
        b.cur = seg(n - n0);
        b.prev = (n == 0) ? nullptr : (n == n0 ? W0 : seg(n - 1 - n0));
        b.next = seg(n + 1 - n0);
        b.c_cur = (n == 0) ? 1.f : 2.f;
        b.c_prev = (n == 0) ? 0.f : 1.f;
        b.c_lap = (n == 0) ? 0.5f : 1.f;
        PAT_TRY_CUDA(step_launch(p, false, b, st));
      }
    }
    loaded = k;
    return PAT_OK;
  };
  // gradient term of the adjoint state Q^m: Q^m .* L P^{m-1}, halved for m = 1
  auto accumulate = [&](int m, const float* Q, const float* Qlo) -> pat_status {
    const int n = m - 1;
    if (n / C != loaded) PAT_TRY(load_segment(n / C));
    PAT_TRY_CUDA(grad_acc_launch(p->R, p->kg_acc, Q, Qlo, seg(n - loaded * C), n == 0 ? 0.5f : 1.f, a, p->dim,
                                 two_d && p->tma2d, st));
    return PAT_OK;
  };
  PAT_TRY_CUDA(dfill_launch(p->kg_acc, N, st));

  // ---- adjoint run with the residual r, accumulating the gradient
  auto inject = [&](float* Q, int t) {
    return inject_launch(Q, p->n_inj, p->d_inj_cell, p->d_inj_ptr, p->d_ent_sensor, p->d_ent_w, r, nt, t, 1.f, st);
  };
  StepArgs c = step_args(p);
  c.y = nullptr;
  if (two_d) {
    float* G = p->d_wv[2];
    auto Qbuf = [&](int m) { return p->d_wv[(nt - m) % 2]; };
    auto Qlo = [&](int m) { return p->d_wv[3 + (nt - m) % 2]; };
    PAT_TRY_CUDA(fill_launch(G, N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(p->d_wv[5], N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(Qbuf(nt), N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(Qlo(nt), N, 0.f, st));
    c.dbuf = G;
    c.dbuf_lo = p->d_wv[5];
    c.inj_r = r;
    for (int m = nt - 1; m >= 1; --m) {
      c.inj_t = m;
      c.cur = Qbuf(m + 1);
      c.cur_lo = Qlo(m + 1);
      c.next = Qbuf(m);
      c.next_lo = Qlo(m);
      c.d_zero = 0;
      c.final_step = 0;
      c.c_lap = 1.f;
      PAT_TRY_CUDA(step_launch(p, true, c, st));
      PAT_TRY(accumulate(m, Qbuf(m), Qlo(m)));
    }
  } else {
    auto Qbuf = [&](int m) { return p->d_wv[(nt - 1 - m) % 3]; };
    PAT_TRY_CUDA(fill_launch(Qbuf(nt - 1), N, 0.f, st));
    PAT_TRY_CUDA(inject(Qbuf(nt - 1), nt - 1));
    PAT_TRY(accumulate(nt - 1, Qbuf(nt - 1), nullptr));
    for (int m = nt - 2; m >= 1; --m) {
      c.cur = Qbuf(m + 1);
      c.prev = (m + 2 <= nt - 1) ? Qbuf(m + 2) : nullptr;
      c.next = Qbuf(m);
      c.c_cur = 2.f;
      c.c_prev = 1.f;
      c.c_lap = 1.f;
      PAT_TRY_CUDA(step_launch(p, true, c, st));
      PAT_TRY_CUDA(inject(Qbuf(m), m));
      PAT_TRY(accumulate(m, Qbuf(m), nullptr));
    }
  }
  PAT_TRY_CUDA(d2f_launch(g, p->kg_acc, N, st));
  return PAT_OK;
}

// --------------------------------------------------------------------- CG
static pat_status apply_normal(pat_plan* p, double s, const float* v, float* out, cudaStream_t st) {
  // out = E_s* K* K E_s v   (alpha v is added by the fused dot kernel)
  PAT_TRY(apply_Es(p, s, v, p->d_img, st));
  PAT_TRY(wave_forward(p, p->d_img, p->d_ybuf, st));
  PAT_TRY(wave_adjoint(p, p->d_ybuf, p->d_img, st));
  PAT_TRY(apply_EsT(p, s, p->d_img, out, st));
  return PAT_OK;
}

pat_status solve_device(pat_plan* p, const float* y, double alpha, double s, int iters, const float* u0, float* u,
                        float* x, double* log, cudaStream_t st) {
  const long long N = p->N;
  float* uu = u ? u : p->d_u;
  // r = b = E_s* K* y
  PAT_TRY(wave_adjoint(p, y, p->d_img, st));
  PAT_TRY(apply_EsT(p, s, p->d_img, p->d_r, st));
  if (u0) {
    if (u0 != uu) PAT_TRY_CUDA(cudaMemcpyAsync(uu, u0, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    PAT_TRY(apply_normal(p, s, uu, p->d_q, st));
    PAT_TRY_CUDA(cg_pq_launch(p->d_q, uu, alpha, N, p->d_partials, p->d_counter, p->d_sc, st));
    PAT_TRY_CUDA(cg_sub_launch(p->d_r, p->d_q, N, st));
    PAT_TRY_CUDA(cg_rr_launch(p->d_r, p->d_p, N, p->d_partials, p->d_counter, p->d_sc, st));
    count_kernels(p, 3);
  } else {
    PAT_TRY_CUDA(cg_init_launch(p->d_r, p->d_r, p->d_p, uu, N, true, p->d_partials, p->d_counter, p->d_sc, st));
    count_kernels(p, 1);
  }
  for (int k = 0; k < iters; ++k) {
    PAT_TRY(apply_normal(p, s, p->d_p, p->d_q, st));
    PAT_TRY_CUDA(cg_pq_launch(p->d_q, p->d_p, alpha, N, p->d_partials, p->d_counter, p->d_sc, st));
    PAT_TRY_CUDA(cg_update_launch(uu, p->d_r, p->d_p, p->d_q, N, p->d_partials, p->d_counter, p->d_sc, log,
                                  p->d_status, st));
    PAT_TRY_CUDA(cg_direction_launch(p->d_p, p->d_r, N, p->d_sc, st));
    count_kernels(p, 3);
  }
  if (x) PAT_TRY(apply_Es(p, s, uu, x, st));
  return PAT_OK;
}

// ------------------------------------------------ several right-hand sides
// Buffers of the second right-hand side and the two-field exchange strips.
static pat_status multi_setup(pat_plan* p, cudaStream_t st) {
  if (p->m2.ready) return PAT_OK;
  auto fl = [&](float** q, size_t n, const char* what) {
    return plan_alloc(p, reinterpret_cast<void**>(q), std::max<size_t>(n, 1) * sizeof(float), what);
  };
  const size_t N = (size_t)p->N, M = (size_t)p->ns * p->nt;
  PAT_TRY(fl(&p->m2.r, N, "cg r (second right-hand side)"));
  PAT_TRY(fl(&p->m2.p, N, "cg p (second right-hand side)"));
  PAT_TRY(fl(&p->m2.q, N, "cg q (second right-hand side)"));
  PAT_TRY(fl(&p->m2.img, N, "image buffer (second right-hand side)"));
  PAT_TRY(fl(&p->m2.u, N, "cg u (second right-hand side)"));
  PAT_TRY(fl(&p->m2.ybuf, M, "sensor data buffer (second right-hand side)"));
  PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->m2.sc), sizeof(CgScalars), "cg scalars (second)"));
  PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->m2.partials), sizeof(double) * cg_grid_blocks(),
                     "cg partials (second)"));
  PAT_TRY(plan_alloc(p, reinterpret_cast<void**>(&p->m2.counter), sizeof(unsigned), "cg counter (second)"));
  PAT_TRY_CUDA(cudaMemsetAsync(p->m2.counter, 0, sizeof(unsigned), st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->m2.sc, 0, sizeof(CgScalars), st));
  p->m2.two_field = false;
  if (p->path == PAT_PATH_PERSISTENT && p->sponge_w == 0 &&
      persist2d_max_ctas2(p->R, false, p->varc) >= p->ntiles && persist2d_max_ctas2(p->R, true, p->varc) >= p->ntiles) {
    PAT_TRY(fl(&p->m2.part, (size_t)4 * p->nsplit * p->nt, "split sensor parts (second)"));
    p->m2.xbuf_bytes = persist2d_xbuf_words(p->R, true, p->ntiles, 2) * 8;
    PAT_TRY(plan_alloc(p, &p->m2.xbuf, p->m2.xbuf_bytes, "two-field exchange strips"));
    p->m2.two_field = true;
  }
  p->m2.ready = true;
  return PAT_OK;
}

static bool two_field(const pat_plan* p) {
  return p->m2.ready && p->m2.two_field && p->path == PAT_PATH_PERSISTENT && p->sponge_w == 0;
}

// K on two right-hand sides: one two-field persistent launch, else two applications.
static pat_status wave_forward2(pat_plan* p, const float* x0, const float* x1, float* y0, float* y1,
                                cudaStream_t st) {
  if (!two_field(p)) {
    PAT_TRY(wave_forward(p, x0, y0, st));
    return wave_forward(p, x1, y1, st);
  }
  if (p->prof_on) PAT_TRY(prof_mark(p, st));
  Persist2DArgs a = persist_args(p);
  a.in = x0;
  a.out = y0;
  a.in1 = x1;
  a.out1 = y1;
  a.part1 = p->m2.part;
  a.xbuf = p->m2.xbuf;
  PAT_TRY_CUDA(cudaMemsetAsync(p->m2.xbuf, 0xff, p->m2.xbuf_bytes, st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_abort, 0, sizeof(int), st));
  PAT_TRY_CUDA(persist2d_launch2(p->R, false, p->varc, a, p->ntiles, st));
  PAT_TRY_CUDA(persist2d_split_combine(p->d_part, p->d_split_sensor, p->nsplit, p->nt, y0, st));
  PAT_TRY_CUDA(persist2d_split_combine(p->m2.part, p->d_split_sensor, p->nsplit, p->nt, y1, st));
  if (p->prof_on) {
    PAT_TRY(prof_mark(p, st));
    p->prof_kernels += 1 + (p->nsplit > 0 ? 2 : 0);
    p->prof_points += 2 * p->N * (long long)(p->nt - 1);
  }
  return PAT_OK;
}

// K* on two right-hand sides.
static pat_status wave_adjoint2(pat_plan* p, const float* y0, const float* y1, float* x0, float* x1,
                                cudaStream_t st) {
  if (!two_field(p)) {
    PAT_TRY(wave_adjoint(p, y0, x0, st));
    return wave_adjoint(p, y1, x1, st);
  }
  if (p->prof_on) PAT_TRY(prof_mark(p, st));
  Persist2DArgs a = persist_args(p);
  a.in = y0;
  a.out = x0;
  a.in1 = y1;
  a.out1 = x1;
  a.xbuf = p->m2.xbuf;
  PAT_TRY_CUDA(cudaMemsetAsync(p->m2.xbuf, 0xff, p->m2.xbuf_bytes, st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_abort, 0, sizeof(int), st));
  PAT_TRY_CUDA(persist2d_launch2(p->R, true, p->varc, a, p->ntiles, st));
  if (p->prof_on) {
    PAT_TRY(prof_mark(p, st));
    p->prof_kernels += 1;
    p->prof_points += 2 * p->N * (long long)(p->nt - 1);
  }
  return PAT_OK;
}

// Two CG solves of the same plan in lockstep (paper Eq. linear_minimization, the coefficient form of
// solve_device, u0 = 0): each iteration's K and K* of both run as one two-field launch each.
static pat_status solve_pair(pat_plan* p, const float* y0, const float* y1, double a0, double a1, double s0,
                             double s1, int iters, float* x0, float* x1, cudaStream_t st) {
  struct Cg {
    float *r, *pp, *q, *img, *u, *ybuf;
    CgScalars* sc;
    double* partials;
    unsigned* counter;
    double alpha, s;
  };
  Cg c[2] = {{p->d_r, p->d_p, p->d_q, p->d_img, p->d_u, p->d_ybuf, p->d_sc, p->d_partials, p->d_counter, a0, s0},
             {p->m2.r, p->m2.p, p->m2.q, p->m2.img, p->m2.u, p->m2.ybuf, p->m2.sc, p->m2.partials, p->m2.counter, a1,
              s1}};
  const long long N = p->N;
  PAT_TRY(wave_adjoint2(p, y0, y1, c[0].img, c[1].img, st));  // r = b = E_s* K* y
  for (auto& v : c) {
    PAT_TRY(apply_EsT(p, v.s, v.img, v.r, st));
    PAT_TRY_CUDA(cg_init_launch(v.r, v.r, v.pp, v.u, N, true, v.partials, v.counter, v.sc, st));
    count_kernels(p, 1);
  }
  for (int k = 0; k < iters; ++k) {
    for (auto& v : c) PAT_TRY(apply_Es(p, v.s, v.pp, v.img, st));
    PAT_TRY(wave_forward2(p, c[0].img, c[1].img, c[0].ybuf, c[1].ybuf, st));
    PAT_TRY(wave_adjoint2(p, c[0].ybuf, c[1].ybuf, c[0].img, c[1].img, st));
    for (auto& v : c) {
      PAT_TRY(apply_EsT(p, v.s, v.img, v.q, st));
      PAT_TRY_CUDA(cg_pq_launch(v.q, v.pp, v.alpha, N, v.partials, v.counter, v.sc, st));
      PAT_TRY_CUDA(cg_update_launch(v.u, v.r, v.pp, v.q, N, v.partials, v.counter, v.sc, nullptr, p->d_status, st));
      PAT_TRY_CUDA(cg_direction_launch(v.pp, v.r, N, v.sc, st));
      count_kernels(p, 3);
    }
  }
  PAT_TRY(apply_Es(p, s0, c[0].u, x0, st));
  PAT_TRY(apply_Es(p, s1, c[1].u, x1, st));
  return PAT_OK;
}

pat_status solve_multi_device(pat_plan* p, int nrhs, const float* const* ys, const double* alphas, const double* ss,
                              int iters, float* const* xs, cudaStream_t st) {
  if (nrhs >= 2) PAT_TRY(multi_setup(p, st));
  int r = 0;
  for (; r + 1 < nrhs; r += 2)
    PAT_TRY(solve_pair(p, ys[r], ys[r + 1], alphas[r], alphas[r + 1], ss[r], ss[r + 1], iters, xs[r], xs[r + 1], st));
  if (r < nrhs) PAT_TRY(solve_device(p, ys[r], alphas[r], ss[r], iters, nullptr, nullptr, xs[r], nullptr, st));
  return PAT_OK;
}

// ------------------------------------------------------- host staging
static bool is_device_ptr(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static pat_status stage(pat_plan* p, int slot, size_t bytes, float** out) {
  if (p->stage_bytes[slot] < bytes) {
    if (p->d_stage[slot]) cudaFree(p->d_stage[slot]);
    p->d_stage[slot] = nullptr;
    p->stage_bytes[slot] = 0;
    cudaError_t e = cudaMalloc(&p->d_stage[slot], bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p->d_stage[slot] = nullptr;
      return cuda_fail(e, "cudaMalloc(staging)");
    }
    p->stage_bytes[slot] = bytes;
  }
  *out = p->d_stage[slot];
  return PAT_OK;
}

// Resolve an input array: device pointers pass through, host arrays are copied in.
static pat_status in_arr(pat_plan* p, int slot, const float* a, size_t count, const float** dev, bool* host,
                         cudaStream_t st) {
  *host = false;
  *dev = a;
  if (!a || is_device_ptr(a)) return PAT_OK;
  float* d;
  PAT_TRY(stage(p, slot, count * sizeof(float), &d));
  PAT_TRY_CUDA(cudaMemcpyAsync(d, a, count * sizeof(float), cudaMemcpyHostToDevice, st));
  *dev = d;
  *host = true;
  return PAT_OK;
}

static pat_status out_arr(pat_plan* p, int slot, float* a, size_t count, float** dev, bool* host) {
  *host = false;
  *dev = a;
  if (!a || is_device_ptr(a)) return PAT_OK;
  PAT_TRY(stage(p, slot, count * sizeof(float), dev));
  *host = true;
  return PAT_OK;
}

static pat_status out_back(float* host_dst, const float* dev, size_t count, bool host, cudaStream_t st) {
  if (!host) return PAT_OK;
  PAT_TRY_CUDA(cudaMemcpyAsync(host_dst, dev, count * sizeof(float), cudaMemcpyDeviceToHost, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

static pat_status check_plan(const pat_plan* p) {
  if (!p) {
    set_error("plan is NULL");
    return PAT_ERR_INVALID;
  }
  return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_forward(pat_plan* plan, const float* x, float* y, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!x || (!y && plan->ns > 0)) {
    set_error("x and y must not be NULL");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float* dx;
  float* dy;
  bool hx, hy;
  PAT_TRY(in_arr(plan, 0, x, plan->N, &dx, &hx, st));
  PAT_TRY(out_arr(plan, 1, y, ny, &dy, &hy));
  if (plan->ns > 0) PAT_TRY(wave_forward(plan, dx, dy, st));
  return out_back(y, dy, ny, hy, st);
}

pat_status pat_adjoint(pat_plan* plan, const float* y, float* x, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!x || (!y && plan->ns > 0)) {
    set_error("x and y must not be NULL");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float* dy;
  float* dx;
  bool hx, hy;
  PAT_TRY(in_arr(plan, 0, y, ny, &dy, &hy, st));
  PAT_TRY(out_arr(plan, 1, x, plan->N, &dx, &hx));
  if (plan->ns > 0) {
    PAT_TRY(wave_adjoint(plan, dy, dx, st));
  } else {
    PAT_TRY_CUDA(fill_launch(dx, plan->N, 0.f, st));
  }
  return out_back(x, dx, plan->N, hx, st);
}

pat_status pat_Es(pat_plan* plan, double s, const float* u, float* x, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!u || !x || !std::isfinite(s)) {
    set_error("u and x must not be NULL and s must be finite");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float* du;
  float* dx;
  bool hu, hx;
  PAT_TRY(in_arr(plan, 0, u, plan->N, &du, &hu, st));
  PAT_TRY(out_arr(plan, 1, x, plan->N, &dx, &hx));
  PAT_TRY(apply_Es(plan, s, du, dx, st));
  return out_back(x, dx, plan->N, hx, st);
}

pat_status pat_EsT(pat_plan* plan, double s, const float* x, float* u, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!u || !x || !std::isfinite(s)) {
    set_error("u and x must not be NULL and s must be finite");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float* dx;
  float* du;
  bool hu, hx;
  PAT_TRY(in_arr(plan, 0, x, plan->N, &dx, &hx, st));
  PAT_TRY(out_arr(plan, 1, u, plan->N, &du, &hu));
  PAT_TRY(apply_EsT(plan, s, dx, du, st));
  return out_back(u, du, plan->N, hu, st);
}

pat_status pat_solve(pat_plan* plan, const float* y, double alpha, double s, int iters, const float* u0, float* u,
                     float* x, double* log, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!y || !(alpha > 0.0) || !std::isfinite(alpha) || !std::isfinite(s) || iters < 0) {
    set_error("y must not be NULL, alpha finite and > 0, s finite, iters >= 0");
    return PAT_ERR_INVALID;
  }
  if (log && !is_device_ptr(log)) {
    set_error("log must be a device array");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float *dy, *du0;
  float *du, *dx;
  bool hy, hu0, hu, hx;
  PAT_TRY(in_arr(plan, 0, y, ny, &dy, &hy, st));
  PAT_TRY(in_arr(plan, 1, u0, plan->N, &du0, &hu0, st));
  PAT_TRY(out_arr(plan, 2, u, plan->N, &du, &hu));
  PAT_TRY(out_arr(plan, 3, x, plan->N, &dx, &hx));
  PAT_TRY(solve_device(plan, dy, alpha, s, iters, du0, du, dx, log, st));
  if (u) PAT_TRY(out_back(u, du, plan->N, hu, st));
  if (x) PAT_TRY(out_back(x, dx, plan->N, hx, st));
  return PAT_OK;
}

pat_status pat_solve_landweber(pat_plan* plan, const float* y, double alpha, double s, int iters, double omega,
                               float* u, float* x, double* J, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!y || !(alpha > 0.0) || !std::isfinite(alpha) || !std::isfinite(s) || iters < 0 || !(omega > 0.0) ||
      !std::isfinite(omega)) {
    set_error("y must not be NULL, alpha and omega finite and > 0, s finite, iters >= 0");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float* dy;
  float *du, *dx;
  bool hy, hu, hx;
  PAT_TRY(in_arr(plan, 0, y, ny, &dy, &hy, st));
  PAT_TRY(out_arr(plan, 2, u, plan->N, &du, &hu));
  PAT_TRY(out_arr(plan, 3, x, plan->N, &dx, &hx));
  PAT_TRY(landweber_device(plan, dy, alpha, s, iters, omega, du, dx, J, st));
  if (u) PAT_TRY(out_back(u, du, plan->N, hu, st));
  if (x) PAT_TRY(out_back(x, dx, plan->N, hx, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

pat_status pat_solve_multi(pat_plan* plan, int nrhs, const float* const* ys, const double* alphas,
                           const double* ss, int iters, float* const* xs, void* stream) {
  PAT_TRY(check_plan(plan));
  if (nrhs < 1 || !ys || !alphas || !ss || !xs || iters < 0) {
    set_error("nrhs >= 1, non-NULL ys / alphas / ss / xs and iters >= 0 required");
    return PAT_ERR_INVALID;
  }
  for (int r = 0; r < nrhs; ++r) {
    if (!ys[r] || !xs[r] || !is_device_ptr(ys[r]) || !is_device_ptr(xs[r]) || !(alphas[r] > 0.0) ||
        !std::isfinite(alphas[r]) || !std::isfinite(ss[r])) {
      set_error("right-hand side %d: ys / xs must be device arrays, alpha finite and > 0, s finite", r);
      return PAT_ERR_INVALID;
    }
  }
  return solve_multi_device(plan, nrhs, ys, alphas, ss, iters, xs, (cudaStream_t)stream);
}

pat_status pat_objective(pat_plan* plan, const float* y, double alpha, double s, const float* u, double* J,
                         float* grad, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!y || !u || !J || !(alpha >= 0.0) || !std::isfinite(alpha) || !std::isfinite(s)) {
    set_error("y, u and J must not be NULL, alpha finite and >= 0, s finite");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float *dy, *du;
  float* dg;
  bool hy, hu, hg;
  PAT_TRY(in_arr(plan, 0, y, ny, &dy, &hy, st));
  PAT_TRY(in_arr(plan, 1, u, plan->N, &du, &hu, st));
  PAT_TRY(out_arr(plan, 2, grad, plan->N, &dg, &hg));
  PAT_TRY(objective_device(plan, dy, alpha, s, du, J, dg, st));
  if (grad) PAT_TRY(out_back(grad, dg, plan->N, hg, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

pat_status pat_solve_gmres(pat_plan* plan, const float* y, double alpha, double s, int iters, float* x, double* res,
                           double* J, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!y || !x || !(alpha > 0.0) || !std::isfinite(alpha) || !std::isfinite(s) || iters < 0) {
    set_error("y and x must not be NULL, alpha finite and > 0, s finite, iters >= 0");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float* dy;
  float* dx;
  bool hy, hx;
  PAT_TRY(in_arr(plan, 0, y, ny, &dy, &hy, st));
  PAT_TRY(out_arr(plan, 3, x, plan->N, &dx, &hx));
  PAT_TRY(gmres_device(plan, dy, alpha, s, iters, dx, res, J, st));
  PAT_TRY(out_back(x, dx, plan->N, hx, st));
  return PAT_OK;
}

pat_status pat_solve_batched(pat_plan* const* plans, int B, const float* const* ys, const double* alphas,
                             const double* ss, int iters, float* const* xs, pat_status* per_inst, void* stream) {
  if (B < 0 || (B > 0 && (!plans || !ys || !alphas || !ss || !xs))) {
    set_error("batched solve: B >= 0 and all arrays are required");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // one batched engine over all instances when they qualify and the arrays live on the device
  bool dev = batch_eligible(plans, B);
  for (int i = 0; dev && i < B; ++i) dev = ys[i] && xs[i] && is_device_ptr(ys[i]) && is_device_ptr(xs[i]);
  if (dev) {
    pat_batch* b = nullptr;
    pat_status s = pat_batch_create(plans, B, stream, &b);
    if (s == PAT_OK) {
      s = pat_batch_solve(b, ys, alphas, ss, iters, xs, per_inst, stream);
      pat_batch_destroy(b);
    }
    return s;
  }
  pat_status first = PAT_OK;
  for (int i = 0; i < B; ++i) {
    pat_status s = pat_solve(plans[i], ys[i], alphas[i], ss[i], iters, nullptr, nullptr, xs[i], nullptr, stream);
    if (s == PAT_OK) s = pat_plan_check(plans[i], st);
    if (per_inst) per_inst[i] = s;
    if (s != PAT_OK && first == PAT_OK) first = s;
  }
  return first;
}

pat_status pat_grad_kappa(pat_plan* plan, const float* x, const float* r, float* g, int segment, void* stream) {
  PAT_TRY(check_plan(plan));
  if (!x || !g || (!r && plan->ns > 0) || segment < 0) {
    set_error("x, r and g must not be NULL and segment >= 0");
    return PAT_ERR_INVALID;
  }
  if (plan->sponge_w > 0) {
    set_error("the medium gradient is defined for plans without an absorbing layer");
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ny = (size_t)plan->ns * plan->nt;
  const float *dx, *dr;
  float* dg;
  bool hx, hr, hg;
  PAT_TRY(in_arr(plan, 0, x, plan->N, &dx, &hx, st));
  PAT_TRY(in_arr(plan, 1, r, ny, &dr, &hr, st));
  PAT_TRY(out_arr(plan, 2, g, plan->N, &dg, &hg));
  PAT_TRY(kappa_grad_device(plan, dx, dr, dg, segment, st));
  return out_back(g, dg, plan->N, hg, st);
}

pat_status pat_plan_profile(pat_plan* plan, int enable) {
  PAT_TRY(check_plan(plan));
  plan->prof_on = enable != 0;
  plan->prof_used = 0;
  plan->prof_kernels = 0;
  plan->prof_points = 0;
  return PAT_OK;
}

pat_status pat_plan_profile_read(pat_plan* plan, long long* kernels, int* wave_calls, double* wave_ms,
                                 long long* point_updates) {
  PAT_TRY(check_plan(plan));
  double total = 0.0;
  for (int i = 0; i + 1 < plan->prof_used; i += 2) {
    PAT_TRY_CUDA(cudaEventSynchronize(plan->prof_ev[i + 1]));
    float ms = 0.f;
    PAT_TRY_CUDA(cudaEventElapsedTime(&ms, plan->prof_ev[i], plan->prof_ev[i + 1]));
    total += ms;
  }
  if (kernels) *kernels = plan->prof_kernels;
  if (wave_calls) *wave_calls = plan->prof_used / 2;
  if (wave_ms) *wave_ms = total;
  if (point_updates) *point_updates = plan->prof_points;
  return PAT_OK;
}

pat_status pat_plan_check(pat_plan* plan, void* stream) {
  PAT_TRY(check_plan(plan));
  cudaStream_t st = (cudaStream_t)stream;
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  int status = 0;
  PAT_TRY_CUDA(cudaMemcpy(&status, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  const int zero = 0;
  PAT_TRY_CUDA(cudaMemcpy(plan->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (status == PAT_ERR_TIMEOUT) set_error("a bounded wait in a wave kernel ran out");
  if (status == PAT_ERR_BREAKDOWN) set_error("CG breakdown: p.q <= 0 or a non-finite step length");
  return (pat_status)status;
}

}  // extern "C"
