// Plan creation: validation, device constants and workspace.
//
// Everything the time loops need is precomputed here in FP64 and rounded
// once: the composed stencil weights of the staggered scheme (paper Sec. 2),
// kappa = (c dt / h)^2 per cell, the bilinear/trilinear sensor weights and
// their transposed (injection) lists, and the Daubechies filters of the
// wavelet transform (paper Sec. 4).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>

#include "plan.h"

namespace pat {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

pat_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA;
}

const char* last_error() { return g_last_error.c_str(); }

pat_status plan_alloc(pat_plan* p, void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    set_error("cudaMalloc(%zu bytes) for %s: %s", bytes, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA;
  }
  p->allocations.push_back(*ptr);
  return PAT_OK;
}

template <typename T>
static pat_status alloc_n(pat_plan* p, T** ptr, size_t count, const char* what) {
  return plan_alloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T), what);
}

template <typename T>
static pat_status upload(pat_plan* p, T** ptr, const std::vector<T>& host, const char* what, cudaStream_t st) {
  PAT_TRY(alloc_n(p, ptr, host.size(), what));
  if (!host.empty()) PAT_TRY_CUDA(cudaMemcpyAsync(*ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return PAT_OK;
}

// ------------------------------------------------------ staggered weights
// Staggered first-derivative weights of order 2M at half-integer offsets.
static const double kStag[4][4] = {{1.0, 0, 0, 0},
                                   {9.0 / 8.0, -1.0 / 24.0, 0, 0},
                                   {75.0 / 64.0, -25.0 / 384.0, 3.0 / 640.0, 0},
                                   {1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0}};

// Weights w_m (m = 1..2M-1) of L = -G^T G along one axis: minus the
// autocorrelation of the staggered difference filter.
static void composed_weights(int M, double* w) {
  double g[2 * 4];
  for (int k = 1; k <= M; ++k) {
    g[M - k] = -kStag[M - 1][k - 1];  // offset -(k - 1/2)
    g[M + k - 1] = kStag[M - 1][k - 1];  // offset +(k - 1/2)
  }
  const int R = 2 * M - 1;
  for (int m = 0; m <= R; ++m) {
    double s = 0.0;
    for (int i = 0; i + m < 2 * M; ++i) s += g[i] * g[i + m];
    w[m] = -s;
  }
}

// ------------------------------------------------------ Daubechies filters
// Minimum-length orthonormal Daubechies scaling filter with nv vanishing
// moments by spectral factorisation: the roots y of
//   P(y) = sum_{k<nv} C(nv-1+k, k) y^k
// give the extra zeros z of H(z) = sum h_k z^k through y = (2 - z - 1/z)/4,
// taking the root outside the unit circle; H(z) = (1+z)^nv prod (z - z_r),
// normalised to sum h = sqrt 2.  Roots by Durand-Kerner iteration.
bool daubechies_filter(int nv, double* h) {
  using cd = std::complex<double>;
  if (nv == 1) {
    h[0] = h[1] = std::sqrt(0.5);
    return true;
  }
  std::vector<double> a(nv);
  for (int k = 0; k < nv; ++k) {
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (nv - 1 + i) / i;  // C(nv-1+k, k)
    a[k] = c;
  }
  const int deg = nv - 1;
  std::vector<cd> y(deg);
  if (deg == 1) {
    y[0] = cd(-a[0] / a[1], 0.0);
  } else {
    for (int i = 0; i < deg; ++i) y[i] = std::pow(cd(0.4, 0.9), i);
    for (int it = 0; it < 2000; ++it) {
      double delta = 0.0;
      for (int i = 0; i < deg; ++i) {
        cd pv = a[deg];
        for (int k = deg - 1; k >= 0; --k) pv = pv * y[i] + a[k];
        pv /= a[deg];
        cd den = 1.0;
        for (int j = 0; j < deg; ++j)
          if (j != i) den *= (y[i] - y[j]);
        const cd step = pv / den;
        y[i] -= step;
        delta = std::max(delta, std::abs(step));
      }
      if (delta < 1e-16) break;
    }
  }
  std::vector<cd> poly(1, cd(1.0, 0.0));  // ascending powers of z
  for (int i = 0; i < deg; ++i) {
    const cd b = 2.0 - 4.0 * y[i];
    const cd disc = std::sqrt(b * b - 4.0);
    const cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
    const cd zr = std::abs(z1) > 1.0 ? z1 : z2;
    std::vector<cd> nxt(poly.size() + 1, cd(0.0, 0.0));
    for (size_t k = 0; k < poly.size(); ++k) {
      nxt[k] -= zr * poly[k];
      nxt[k + 1] += poly[k];
    }
    poly.swap(nxt);
  }
  for (int i = 0; i < nv; ++i) {
    std::vector<cd> nxt(poly.size() + 1, cd(0.0, 0.0));
    for (size_t k = 0; k < poly.size(); ++k) {
      nxt[k] += poly[k];
      nxt[k + 1] += poly[k];
    }
    poly.swap(nxt);
  }
  double sum = 0.0;
  for (int k = 0; k < 2 * nv; ++k) sum += poly[k].real();
  for (int k = 0; k < 2 * nv; ++k) h[k] = poly[k].real() * std::sqrt(2.0) / sum;
  // self-check: double-shift orthonormality
  for (int m = 0; m < nv; ++m) {
    double s = 0.0;
    for (int k = 0; k + 2 * m < 2 * nv; ++k) s += h[k] * h[k + 2 * m];
    if (std::fabs(s - (m == 0 ? 1.0 : 0.0)) > 1e-12) return false;
  }
  return true;
}

// --------------------------------------------------- persistent 2D set-up
static pat_status setup_persistent(pat_plan* p, cudaStream_t st) {
  const int TX = persist2d_tile_x(), TY = persist2d_tile_y();
  p->tiles_x = (p->n[0] + TX - 1) / TX;
  p->tiles_y = (p->n[1] + TY - 1) / TY;
  p->ntiles = p->tiles_x * p->tiles_y;
  const int nx = p->n[0];

  // sampling entries grouped by the tile holding each sensor's base cell; a
  // sensor whose 2x2 block crosses a tile corner is split into four parts
  std::vector<std::vector<SampEntry>> per_tile(p->ntiles);
  std::vector<int> split_sensor;
  for (int s = 0; s < p->ns; ++s) {
    const int c0 = p->h_sens_cell[s * 4];
    const int bx = c0 % nx, by = c0 / nx;
    const bool split = (bx % TX == TX - 1) && (by % TY == TY - 1);
    if (!split) {
      const int tile = (by / TY) * p->tiles_x + bx / TX;
      SampEntry e;
      e.sensor = s;
      e.part = -1;
      e.lx = (short)(bx % TX);
      e.ly = (short)(by % TY);
      for (int k = 0; k < 4; ++k) e.w[k] = p->h_sens_w[s * 4 + k];
      per_tile[tile].push_back(e);
      continue;
    }
    const int q = (int)split_sensor.size();
    split_sensor.push_back(s);
    for (int k = 0; k < 4; ++k) {
      const int cell = p->h_sens_cell[s * 4 + k];
      const int cx = cell % nx, cy = cell / nx;
      SampEntry e;
      e.sensor = s;
      e.part = 4 * q + k;
      e.lx = (short)(cx % TX);
      e.ly = (short)(cy % TY);
      e.w[0] = p->h_sens_w[s * 4 + k];
      e.w[1] = e.w[2] = e.w[3] = 0.f;
      per_tile[(cy / TY) * p->tiles_x + cx / TX].push_back(e);
    }
  }
  p->nsplit = (int)split_sensor.size();
  PAT_TRY(upload(p, &p->d_split_sensor, split_sensor, "split sensors", st));
  PAT_TRY(alloc_n(p, &p->d_part, (size_t)4 * p->nsplit * p->nt, "split sensor parts"));
  std::vector<int> samp_ptr(p->ntiles + 1, 0);
  std::vector<SampEntry> samp;
  for (int t = 0; t < p->ntiles; ++t) {
    samp_ptr[t] = (int)samp.size();
    samp.insert(samp.end(), per_tile[t].begin(), per_tile[t].end());
  }
  samp_ptr[p->ntiles] = (int)samp.size();

  // injected cells grouped by tile
  std::vector<std::vector<InjCell>> inj_tile(p->ntiles);
  for (int i = 0; i < p->n_inj; ++i) {
    const int c = p->h_inj_cell[i];
    const int cx = c % nx, cy = c / nx;
    const int tile = (cy / TY) * p->tiles_x + cx / TX;
    InjCell ic;
    ic.local = (cy % TY) * TX + (cx % TX);
    ic.beg = p->h_inj_ptr[i];
    ic.end = p->h_inj_ptr[i + 1];
    inj_tile[tile].push_back(ic);
  }
  std::vector<int> inj_ptr(p->ntiles + 1, 0);
  std::vector<InjCell> inj;
  for (int t = 0; t < p->ntiles; ++t) {
    inj_ptr[t] = (int)inj.size();
    inj.insert(inj.end(), inj_tile[t].begin(), inj_tile[t].end());
  }
  inj_ptr[p->ntiles] = (int)inj.size();

  PAT_TRY(upload(p, &p->d_tile_samp_ptr, samp_ptr, "tile sampling offsets", st));
  PAT_TRY(upload(p, &p->d_samp, samp, "tile sampling entries", st));
  PAT_TRY(upload(p, &p->d_tile_inj_ptr, inj_ptr, "tile injection offsets", st));
  PAT_TRY(upload(p, &p->d_tinj, inj, "tile injection cells", st));
  // tagged exchange words, invalidated (0xff bytes) before every launch
  p->xbuf_bytes = persist2d_xbuf_words(p->R, true, p->ntiles) * 8;
  PAT_TRY(plan_alloc(p, &p->d_xbuf, p->xbuf_bytes, "exchange strips"));
  if (const char* e = getenv("PAT_POLL_NS")) p->poll_ns = std::max(0, atoi(e));
  PAT_TRY(alloc_n(p, &p->d_abort, 1, "abort flag"));
  return PAT_OK;
}

static pat_status create(const pat_grid* grid, const double* c, double c0, const double* sensors, int ns, double dt,
                         int nt, int order, const pat_wavelet* wav, cudaStream_t st, pat_plan* p) {
  if (!grid || !wav) {
    set_error("grid and wavelet descriptions are required");
    return PAT_ERR_INVALID;
  }
  if (grid->dim != 2 && grid->dim != 3) {
    set_error("dim must be 2 or 3 (got %d)", grid->dim);
    return PAT_ERR_INVALID;
  }
  p->dim = grid->dim;
  for (int a = 0; a < 3; ++a) p->n[a] = (a < p->dim) ? grid->n[a] : 1;
  for (int a = 0; a < p->dim; ++a)
    if (p->n[a] < 2 || p->n[a] > (1 << 20)) {
      set_error("grid extent n[%d] = %d out of range [2, 2^20]", a, p->n[a]);
      return PAT_ERR_INVALID;
    }
  p->N = (long long)p->n[0] * p->n[1] * p->n[2];
  if (p->N >= (1LL << 31)) {
    set_error("grid has %lld cells; the limit is 2^31 - 1", p->N);
    return PAT_ERR_INVALID;
  }
  if (!(grid->h > 0.0) || !std::isfinite(grid->h) || !(dt > 0.0) || !std::isfinite(dt)) {
    set_error("h and dt must be finite and positive");
    return PAT_ERR_INVALID;
  }
  if (nt < 1 || nt >= (1 << 20)) {
    set_error("nt = %d out of range [1, 2^20)", nt);
    return PAT_ERR_INVALID;
  }
  if (order != 2 && order != 4 && order != 6 && order != 8) {
    set_error("order must be 2, 4, 6 or 8 (got %d)", order);
    return PAT_ERR_INVALID;
  }
  if (ns < 0 || (ns > 0 && !sensors)) {
    set_error("ns must be >= 0 with a sensor array when > 0");
    return PAT_ERR_INVALID;
  }
  if (wav->family != 1 && wav->family != 2 && wav->family != 4) {
    set_error("wavelet family must be 1 (haar), 2 (db2) or 4 (db4)");
    return PAT_ERR_INVALID;
  }
  if (wav->levels < 0 || wav->levels > kMaxLevels || wav->level_offset < 0) {
    set_error("wavelet levels must be in [0, %d] and level_offset >= 0", kMaxLevels);
    return PAT_ERR_INVALID;
  }
  for (int a = 0; a < p->dim; ++a)
    if (p->n[a] % (1 << wav->levels) != 0) {
      set_error("n[%d] = %d is not divisible by 2^levels = %d", a, p->n[a], 1 << wav->levels);
      return PAT_ERR_INVALID;
    }
  p->h = grid->h;
  p->dt = dt;
  p->nt = nt;
  p->order = order;
  p->M = order / 2;
  p->R = 2 * p->M - 1;
  p->ns = ns;
  p->corners = 1 << p->dim;

  // ---- medium and CFL (c_max dt / h <= 1 / (sqrt(d) sum |c_k|))
  double cmax = 0.0, cmin = 0.0;
  bool constant = true;
  if (c) {
    cmax = c[0];
    cmin = c[0];
    for (long long i = 0; i < p->N; ++i) {
      const double v = c[i];
      if (!(v > 0.0) || !std::isfinite(v)) {
        set_error("speed of sound at cell %lld is not finite and positive", i);
        return PAT_ERR_INVALID;
      }
      cmax = std::max(cmax, v);
      cmin = std::min(cmin, v);
    }
    constant = (cmax == cmin);
    c0 = cmax;
  } else {
    if (!(c0 > 0.0) || !std::isfinite(c0)) {
      set_error("constant speed of sound c0 must be finite and positive");
      return PAT_ERR_INVALID;
    }
    cmax = c0;
  }
  p->c_max = cmax;
  double ssum = 0.0;
  for (int k = 0; k < p->M; ++k) ssum += std::fabs(kStag[p->M - 1][k]);
  const double limit = 1.0 / (std::sqrt((double)p->dim) * ssum);
  const double cfl = cmax * dt / p->h;
  if (cfl > limit * (1.0 + 1e-12)) {
    set_error("CFL number c_max dt / h = %.6g exceeds the limit %.6g of order %d in %dD", cfl, limit, order, p->dim);
    return PAT_ERR_CFL;
  }
  double wd[kMaxR + 1];
  composed_weights(p->M, wd);
  for (int m = 0; m <= p->R; ++m) p->w[m] = (float)wd[m];
  p->varc = !constant;
  {
    const double k0 = (c0 * dt / p->h) * (c0 * dt / p->h);
    p->kappa0 = (float)k0;
    p->kappa0_lo = (float)(k0 - (double)p->kappa0);
  }
  if (p->varc) {
    std::vector<float> kap(p->N), kap_lo(p->N);
    for (long long i = 0; i < p->N; ++i) {
      const double r = c[i] * dt / p->h;
      kap[i] = (float)(r * r);
      kap_lo[i] = (float)(r * r - (double)kap[i]);
    }
    PAT_TRY(upload(p, &p->d_kappa, kap, "kappa", st));
    PAT_TRY(upload(p, &p->d_kappa_lo, kap_lo, "kappa residual", st));
  }

  // ---- sensors: interpolation weights in FP64, cell index floor(u) clamped to n-2
  p->h_sens_cell.assign((size_t)ns * p->corners, 0);
  p->h_sens_w.assign((size_t)ns * p->corners, 0.f);
  std::vector<std::tuple<int, int, float>> ent;  // (cell, sensor, weight)
  for (int s = 0; s < ns; ++s) {
    int i0[3] = {0, 0, 0};
    double f[3] = {0, 0, 0};
    for (int a = 0; a < p->dim; ++a) {
      const double u = sensors[(size_t)s * p->dim + a] / p->h;
      if (!std::isfinite(u) || u < 0.0 || u > (double)(p->n[a] - 1)) {
        set_error("sensor %d coordinate %d lies outside [0, (n-1) h]", s, a);
        return PAT_ERR_INVALID;
      }
      int i = (int)std::floor(u);
      if (i > p->n[a] - 2) i = p->n[a] - 2;
      i0[a] = i;
      f[a] = u - (double)i;
    }
    for (int k = 0; k < p->corners; ++k) {
      int cc[3] = {0, 0, 0};
      double wv = 1.0;
      for (int a = 0; a < p->dim; ++a) {
        const int bit = (k >> a) & 1;
        cc[a] = i0[a] + bit;
        wv *= bit ? f[a] : 1.0 - f[a];
      }
      const int cell = (int)(((long long)cc[2] * p->n[1] + cc[1]) * p->n[0] + cc[0]);
      p->h_sens_cell[(size_t)s * p->corners + k] = cell;
      p->h_sens_w[(size_t)s * p->corners + k] = (float)wv;
      if (wv != 0.0) ent.emplace_back(cell, s, (float)wv);
    }
  }
  std::stable_sort(ent.begin(), ent.end(), [](const auto& x, const auto& y) {
    return std::get<0>(x) < std::get<0>(y) || (std::get<0>(x) == std::get<0>(y) && std::get<1>(x) < std::get<1>(y));
  });
  std::vector<int> ent_sensor(ent.size());
  std::vector<float> ent_w(ent.size());
  p->h_inj_cell.clear();
  p->h_inj_ptr.clear();
  for (size_t e = 0; e < ent.size(); ++e) {
    ent_sensor[e] = std::get<1>(ent[e]);
    ent_w[e] = std::get<2>(ent[e]);
    if (e == 0 || std::get<0>(ent[e]) != std::get<0>(ent[e - 1])) {
      p->h_inj_cell.push_back(std::get<0>(ent[e]));
      p->h_inj_ptr.push_back((int)e);
    }
  }
  p->h_inj_ptr.push_back((int)ent.size());
  p->n_inj = (int)p->h_inj_cell.size();
  PAT_TRY(upload(p, &p->d_sens_cell, p->h_sens_cell, "sensor cells", st));
  PAT_TRY(upload(p, &p->d_sens_w, p->h_sens_w, "sensor weights", st));
  PAT_TRY(upload(p, &p->d_inj_cell, p->h_inj_cell, "injection cells", st));
  PAT_TRY(upload(p, &p->d_inj_ptr, p->h_inj_ptr, "injection offsets", st));
  PAT_TRY(upload(p, &p->d_ent_sensor, ent_sensor, "injection sensors", st));
  PAT_TRY(upload(p, &p->d_ent_w, ent_w, "injection weights", st));

  // ---- wavelet filters
  p->family = wav->family;
  p->L = 2 * wav->family;
  p->levels = wav->levels;
  p->level_offset = wav->level_offset;
  double hd[kMaxTaps];
  if (!daubechies_filter(wav->family, hd)) {
    set_error("Daubechies filter construction failed its orthonormality check");
    return PAT_ERR_INVALID;
  }
  for (int j = 0; j < p->L; ++j) {
    p->hf[j] = (float)hd[j];
    p->gf[j] = (float)(((j & 1) ? -1.0 : 1.0) * hd[p->L - 1 - j]);
  }

  // ---- workspace
  const size_t N = (size_t)p->N;
  for (int i = 0; i < (p->dim == 2 ? 6 : 3); ++i) PAT_TRY(alloc_n(p, &p->d_wv[i], N, "wave fields"));
  PAT_TRY(alloc_n(p, &p->d_dwt_a, N >> p->dim, "dwt approximation"));
  PAT_TRY(alloc_n(p, &p->d_dwt_b, N >> p->dim, "dwt approximation"));
  if (p->dim == 3) {
    PAT_TRY(alloc_n(p, &p->d_dwt_t1, N, "dwt pass buffer"));
    PAT_TRY(alloc_n(p, &p->d_dwt_t2, N, "dwt pass buffer"));
  }
  PAT_TRY(alloc_n(p, &p->d_r, N, "cg r"));
  PAT_TRY(alloc_n(p, &p->d_p, N, "cg p"));
  PAT_TRY(alloc_n(p, &p->d_q, N, "cg q"));
  PAT_TRY(alloc_n(p, &p->d_img, N, "image buffer"));
  PAT_TRY(alloc_n(p, &p->d_u, N, "cg u"));
  PAT_TRY(alloc_n(p, &p->d_ybuf, (size_t)ns * nt, "sensor data buffer"));
  PAT_TRY(alloc_n(p, &p->d_sc, 1, "cg scalars"));
  PAT_TRY(alloc_n(p, &p->d_partials, (size_t)cg_grid_blocks(), "cg partials"));
  PAT_TRY(alloc_n(p, &p->d_counter, 1, "cg counter"));
  PAT_TRY(alloc_n(p, &p->d_status, 1, "status"));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned), st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
  PAT_TRY_CUDA(cudaMemsetAsync(p->d_sc, 0, sizeof(CgScalars), st));

  // ---- engine choice: the persistent kernel when all tiles can be co-resident
  p->persist_ok = false;
  if (p->dim == 2 && persist2d_supported(p->R, p->varc)) {
    const int TX = persist2d_tile_x(), TY = persist2d_tile_y();
    const int ntiles = ((p->n[0] + TX - 1) / TX) * ((p->n[1] + TY - 1) / TY);
    const int cap = std::min(persist2d_max_ctas(p->R, false, p->varc), persist2d_max_ctas(p->R, true, p->varc));
    if (ntiles <= cap) {
      PAT_TRY(setup_persistent(p, st));
      p->persist_ok = true;
    }
  }
  p->path = p->persist_ok ? PAT_PATH_PERSISTENT : PAT_PATH_STEP;
  const char* env = getenv("PAT_WAVE_PATH");
  if (env && strcmp(env, "step") == 0) p->path = PAT_PATH_STEP;

  // 2D per-step engine: TMA tile pipelines when the driver can encode the descriptors
  p->tma2d = false;
  const char* env2 = getenv("PAT_STEP2D");
  if (p->dim == 2 && tma2d_supported(p->n[0], p->R) && !(env2 && strcmp(env2, "plain") == 0)) {
    CUtensorMap mh, mo;
    if (tma2d_encode(p->d_wv[0], p->n[0], p->n[1], p->R, &mh, &mo) == cudaSuccess) p->tma2d = true;
  }
  // 3D constant media: TMA plane pipelines when the driver can encode the descriptors
  p->tma3d = false;
  const char* env3 = getenv("PAT_STEP3D");
  if (p->dim == 3 && tma3d_supported(p->n[0], p->R, p->varc) && !(env3 && strcmp(env3, "plain") == 0)) {
    CUtensorMap mc, mp;
    if (tma3d_encode(p->d_wv[0], p->n[0], p->n[1], p->n[2], p->R, &mc, &mp) == cudaSuccess) {
      p->tma3d_split = tma3d_split(p->R, p->n[0], p->n[1], p->n[2]);
      p->tma3d = p->tma3d_split.nctas > 0;
    }
  }
  if (p->tma3d) {  // injection lists per CTA of the 3D TMA grid (the adjoint injects after each step)
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2], G = p->tma3d_split.nctas;
    std::vector<std::vector<InjCell>> bins((size_t)G);
    for (int i = 0; i < p->n_inj; ++i) {
      const long long c = p->h_inj_cell[i];
      const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
      bins[tma3d_cta_of(nx, ny, nz, p->tma3d_split, x, y, z)].push_back(InjCell{(int)c, p->h_inj_ptr[i], p->h_inj_ptr[i + 1]});
    }
    std::vector<int> ptr(1, 0);
    std::vector<InjCell> cells;
    for (auto& b : bins) {
      cells.insert(cells.end(), b.begin(), b.end());
      ptr.push_back((int)cells.size());
    }
    PAT_TRY(alloc_n(p, &p->d_tinj3_ptr, ptr.size(), "CTA injection lists"));
    PAT_TRY(alloc_n(p, &p->d_tinj3, std::max<size_t>(cells.size(), 1), "CTA injection lists"));
    PAT_TRY_CUDA(cudaMemcpyAsync(p->d_tinj3_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, st));
    if (!cells.empty())
      PAT_TRY_CUDA(cudaMemcpyAsync(p->d_tinj3, cells.data(), sizeof(InjCell) * cells.size(), cudaMemcpyHostToDevice,
                                   st));
  }
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_plan_create(const pat_grid* grid, const double* c, double c0, const double* sensors, int ns, double dt,
                           int nt, int order, const pat_wavelet* wavelet, void* stream, pat_plan** out) {
  if (!out) {
    set_error("out must not be NULL");
    return PAT_ERR_INVALID;
  }
  *out = nullptr;
  pat_plan* p = new (std::nothrow) pat_plan();
  if (!p) {
    set_error("host allocation failed");
    return PAT_ERR_OOM;
  }
  const pat_status s = create(grid, c, c0, sensors, ns, dt, nt, order, wavelet, (cudaStream_t)stream, p);
  if (s != PAT_OK) {
    std::string keep = last_error();
    pat_plan_destroy(p);
    set_error("%s", keep.c_str());
    return s;
  }
  *out = p;
  return PAT_OK;
}

void pat_plan_destroy(pat_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  for (void* ptr : plan->allocations) cudaFree(ptr);
  for (int i = 0; i < 4; ++i)
    if (plan->d_stage[i]) cudaFree(plan->d_stage[i]);
  for (cudaEvent_t e : plan->prof_ev) cudaEventDestroy(e);
  cudaFree(plan->kg_ckpt);
  cudaFree(plan->kg_seg);
  cudaFree(plan->kg_work);
  cudaFree(plan->kg_acc);
  delete plan;
}

pat_status pat_plan_info(const pat_plan* plan, long long* n_cells, int* ns, int* nt) {
  if (!plan) {
    set_error("plan is NULL");
    return PAT_ERR_INVALID;
  }
  if (n_cells) *n_cells = plan->N;
  if (ns) *ns = plan->ns;
  if (nt) *nt = plan->nt;
  return PAT_OK;
}

pat_status pat_plan_set_path(pat_plan* plan, int path) {
  if (!plan) {
    set_error("plan is NULL");
    return PAT_ERR_INVALID;
  }
  const bool persist = plan->persist_ok;
  if (path == PAT_PATH_AUTO) {
    plan->path = persist ? PAT_PATH_PERSISTENT : PAT_PATH_STEP;
  } else if (path == PAT_PATH_PERSISTENT) {
    if (!persist) {
      set_error("the persistent engine is not available for this plan (3D, or too many tiles to co-reside)");
      return PAT_ERR_INVALID;
    }
    plan->path = path;
  } else if (path == PAT_PATH_STEP) {
    plan->path = path;
  } else {
    set_error("unknown path %d", path);
    return PAT_ERR_INVALID;
  }
  return PAT_OK;
}

pat_status pat_plan_set_prior(pat_plan* plan, int kind, double length_cells, void* stream) {
  if (!plan) {
    set_error("plan is NULL");
    return PAT_ERR_INVALID;
  }
  if (kind == 0) {
    plan->prior = 0;
    return PAT_OK;
  }
  if (kind != 1 || !std::isfinite(length_cells) || !(length_cells > 0.0)) {
    set_error("prior kind must be 0 (wavelet) or 1 (Fourier) with length_cells finite and > 0");
    return PAT_ERR_INVALID;
  }
  if (!fourier_supported(plan->dim, plan->n[0], plan->n[1])) {
    set_error("the Fourier prior needs a 2D grid with power-of-two extents up to 4096");
    return PAT_ERR_INVALID;
  }
  PAT_TRY(fourier_setup(plan, length_cells, (cudaStream_t)stream));
  plan->prior = 1;
  return PAT_OK;
}

pat_status pat_plan_set_sponge(pat_plan* plan, int width, double sigma_max, void* stream) {
  if (!plan) {
    set_error("plan is NULL");
    return PAT_ERR_INVALID;
  }
  if (width < 0 || !std::isfinite(sigma_max) || sigma_max < 0.0) {
    set_error("absorbing layer: width >= 0 and a finite sigma_max >= 0 are required");
    return PAT_ERR_INVALID;
  }
  if (width > 0 && plan->dim != 2) {
    set_error("the absorbing layer is implemented for 2D grids");
    return PAT_ERR_INVALID;
  }
  const int nx = plan->n[0], ny = plan->n[1];
  if (width > 0 && (2 * width > nx || 2 * width > ny)) {
    set_error("absorbing layer of %d cells does not fit a %d x %d grid", width, nx, ny);
    return PAT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (width == 0) {
    plan->sponge_w = 0;
    plan->sponge_sigma_max = 0.0;
    return PAT_OK;
  }
  // quadratic profile: within `width` cells of a face sigma = sigma_max ((width - d) / width)^2,
  // d = cells to that face; the axes' contributions add (corners twice).  Default sigma_max for a
  // nominal reflection of 1e-3: 3 c_max ln(1e3) / (2 width h).
  const double smax = sigma_max > 0.0 ? sigma_max : 3.0 * plan->c_max * std::log(1e3) / (2.0 * width * plan->h);
  if (!plan->d_sp_a) {
    PAT_TRY(plan_alloc(plan, reinterpret_cast<void**>(&plan->d_sp_a), sizeof(float) * plan->N, "layer factors"));
    PAT_TRY(plan_alloc(plan, reinterpret_cast<void**>(&plan->d_sp_b), sizeof(float) * plan->N, "layer factors"));
  }
  std::vector<float> fa((size_t)plan->N), fb((size_t)plan->N);
  auto prof = [&](int i, int n) {
    const int d = std::min(i, n - 1 - i);
    if (d >= width) return 0.0;
    const double r = double(width - d) / width;
    return smax * r * r;
  };
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const double q = 0.5 * (prof(x, nx) + prof(y, ny)) * plan->dt;
      fa[(size_t)y * nx + x] = (float)((1.0 - q) / (1.0 + q));
      fb[(size_t)y * nx + x] = (float)(1.0 / (1.0 + q));
    }
  PAT_TRY_CUDA(cudaMemcpyAsync(plan->d_sp_a, fa.data(), sizeof(float) * plan->N, cudaMemcpyHostToDevice, st));
  PAT_TRY_CUDA(cudaMemcpyAsync(plan->d_sp_b, fb.data(), sizeof(float) * plan->N, cudaMemcpyHostToDevice, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  plan->sponge_w = width;
  plan->sponge_sigma_max = smax;
  return PAT_OK;
}

pat_status pat_plan_get_path(const pat_plan* plan, int* path) {
  if (!plan || !path) {
    set_error("plan and path must not be NULL");
    return PAT_ERR_INVALID;
  }
  *path = plan->path;
  return PAT_OK;
}

pat_status pat_plan_set_timeout(pat_plan* plan, long long timeout_ns) {
  if (!plan || timeout_ns < 0) {
    set_error("plan must not be NULL and the timeout must be >= 0");
    return PAT_ERR_INVALID;
  }
  plan->timeout_ns = timeout_ns;
  return PAT_OK;
}

const char* pat_last_error(void) { return pat::last_error(); }

}  // extern "C"
