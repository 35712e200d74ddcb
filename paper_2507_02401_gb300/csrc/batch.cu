// Batched reconstructions behind the C ABI: tile tables, the per-step launch
// sequence of a batched K / K*, the tile-shape autotuner and the CG iteration
// of all instances captured as one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "batch.h"
#include "tma.cuh"

namespace pat {
namespace {

template <typename T>
pat_status balloc(pat_batch* b, T** ptr, size_t count, const char* what) {
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc for %s: %s", what, cudaGetErrorString(e));
    return PAT_ERR_OOM;
  }
  b->allocations.push_back(p);
  *ptr = static_cast<T*>(p);
  return PAT_OK;
}

void bfree_all(pat_batch* b) {
  for (void* p : b->allocations) cudaFree(p);
  b->allocations.clear();
  b->d_inst = nullptr;
  b->d_tiles = nullptr;
  b->d_maps = nullptr;
  b->d_status = nullptr;
  b->d_active = nullptr;
  b->d_bar = nullptr;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Why a plan cannot join a batch, or nullptr.
const char* ineligible(const pat_plan* p, int R) {
  if (p->dim != 2) return "batched instances are 2D";
  if (p->R != R) return "batched instances share one stencil order";
  if (p->n[0] % 4 != 0) return "batched instances have nx divisible by 4";
  if (p->sponge_w > 0) return "batched instances have no absorbing layer";
  return nullptr;
}

// Tile table, per-tile sampling / injection lists, instance descriptors and
// tensor maps for tile height `variant`; replaces earlier tables.
pat_status build_tables(pat_batch* b, int variant, cudaStream_t st) {
  bfree_all(b);
  b->variant = variant;
  const int TX = 64, TY = batch_tile_y(variant);
  const int B = b->B;
  std::vector<BInst> inst(B);
  std::vector<BTile> tiles;
  std::vector<std::vector<int>> samp(B);
  std::vector<std::vector<InjCell>> inj(B);
  for (int k = 0; k < B; ++k) {
    const pat_plan* p = b->plans[b->order[k]];
    const int nx = p->n[0], ny = p->n[1];
    const int tx = (nx + TX - 1) / TX, ty = (ny + TY - 1) / TY, nt_tiles = tx * ty;
    BInst& I = inst[k];
    std::memset(&I, 0, sizeof(I));
    I.nx = nx;
    I.ny = ny;
    I.nt = p->nt;
    I.tiles_x = tx;
    I.tile0 = (int)tiles.size();
    I.ns = p->ns;
    I.corners = p->corners;
    I.kappa0 = p->kappa0;
    I.kappa0_lo = p->kappa0_lo;
    I.kappa = p->varc ? p->d_kappa : nullptr;
    I.kappa_lo = p->varc ? p->d_kappa_lo : nullptr;
    I.img = p->d_img;
    I.P[0] = p->d_wv[0];
    I.P[1] = p->d_wv[1];
    I.P_lo[0] = p->d_wv[3];
    I.P_lo[1] = p->d_wv[4];
    I.D = p->d_wv[2];
    I.y = p->d_ybuf;
    I.sens_cell = p->d_sens_cell;
    I.sens_w = p->d_sens_w;
    I.ent_sensor = p->d_ent_sensor;
    I.ent_w = p->d_ent_w;
    auto tile_of = [&](int cell) { return ((cell / nx) / TY) * tx + (cell % nx) / TX; };
    std::vector<std::vector<int>> sb(nt_tiles);
    for (int s = 0; s < p->ns; ++s) sb[tile_of(p->h_sens_cell[(size_t)s * p->corners])].push_back(s);
    std::vector<std::vector<InjCell>> ib(nt_tiles);
    for (int i = 0; i < p->n_inj; ++i)
      ib[tile_of(p->h_inj_cell[i])].push_back(InjCell{p->h_inj_cell[i], p->h_inj_ptr[i], p->h_inj_ptr[i + 1]});
    for (int tl = 0; tl < nt_tiles; ++tl) {
      BTile d{};
      d.inst = k;
      d.gx0 = (tl % tx) * TX;
      d.gy0 = (tl / tx) * TY;
      d.lt = tl;
      d.s0 = (int)samp[k].size();
      samp[k].insert(samp[k].end(), sb[tl].begin(), sb[tl].end());
      d.s1 = (int)samp[k].size();
      d.j0 = (int)inj[k].size();
      inj[k].insert(inj[k].end(), ib[tl].begin(), ib[tl].end());
      d.j1 = (int)inj[k].size();
      tiles.push_back(d);
    }
  }
  b->ntiles = (int)tiles.size();
  // tiles running at global step t: instances with nt > t (a prefix, longest first)
  b->active.assign(b->max_nt, 0);
  for (int k = 0; k < B; ++k) {
    const int tiles = (k + 1 < B ? inst[k + 1].tile0 : b->ntiles) - inst[k].tile0;
    for (int t = 0; t < inst[k].nt; ++t) b->active[t] += tiles;
  }
  // per-instance lists in device memory
  for (int k = 0; k < B; ++k) {
    int* ds;
    InjCell* di;
    PAT_TRY(balloc(b, &ds, samp[k].size(), "batch sampling lists"));
    PAT_TRY(balloc(b, &di, inj[k].size(), "batch injection lists"));
    if (!samp[k].empty())
      PAT_TRY_CUDA(cudaMemcpyAsync(ds, samp[k].data(), sizeof(int) * samp[k].size(), cudaMemcpyHostToDevice, st));
    if (!inj[k].empty())
      PAT_TRY_CUDA(cudaMemcpyAsync(di, inj[k].data(), sizeof(InjCell) * inj[k].size(), cudaMemcpyHostToDevice, st));
    inst[k].samp = ds;
    inst[k].inj = di;
  }
  std::vector<CUtensorMap> maps(BATCH_MAPS * (size_t)B);
  for (int k = 0; k < B; ++k) {
    const BInst& I = inst[k];
    const float* fields[BATCH_MAPS] = {I.P[0], I.P[1], I.img, I.P_lo[0], I.P_lo[1]};
    for (int f = 0; f < BATCH_MAPS; ++f)
      PAT_TRY_CUDA(batch_encode(fields[f], I.nx, I.ny, b->R, variant, &maps[BATCH_MAPS * k + f]));
  }
  PAT_TRY(balloc(b, &b->d_inst, (size_t)B, "batch instances"));
  PAT_TRY(balloc(b, &b->d_tiles, tiles.size(), "batch tile table"));  // cudaMalloc: 16-byte aligned entries
  PAT_TRY(balloc(b, &b->d_maps, maps.size(), "batch tensor maps"));  // cudaMalloc: 256-byte aligned
  PAT_TRY(balloc(b, &b->d_status, 1, "batch status"));
  PAT_TRY_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int), st));
  PAT_TRY(balloc(b, &b->d_active, (size_t)b->max_nt, "batch active tiles per step"));
  PAT_TRY_CUDA(cudaMemcpyAsync(b->d_active, b->active.data(), sizeof(int) * b->max_nt, cudaMemcpyHostToDevice, st));
  PAT_TRY(balloc(b, &b->d_bar, 1, "batch grid barrier"));
  PAT_TRY_CUDA(cudaMemcpyAsync(b->d_inst, inst.data(), sizeof(BInst) * B, cudaMemcpyHostToDevice, st));
  PAT_TRY_CUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BTile) * tiles.size(), cudaMemcpyHostToDevice, st));
  PAT_TRY_CUDA(cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));  // host vectors go out of scope
  b->nctas = batch_max_ctas(b->R, variant, false);
  b->nctas_adj = batch_max_ctas(b->R, variant, true);
  if (b->nctas <= 0 || b->nctas_adj <= 0) {
    set_error("batched step kernel does not fit on this device");
    return PAT_ERR_CUDA;
  }
  return PAT_OK;
}

BatchStepArgs step_args(const pat_batch* b, int t, bool adjoint) {
  BatchStepArgs a{};
  a.inst = b->d_inst;
  a.tiles = b->d_tiles;
  a.maps = b->d_maps;
  a.t = t;
  a.adjoint = adjoint ? 1 : 0;
  a.active = b->active[t];
  const pat_plan* p0 = b->plans[0];
  for (int m = 0; m <= kMaxR; ++m) a.w[m] = p0->w[m];
  a.status = b->d_status;
  a.timeout_ns = b->timeout_ns;
  return a;
}

// Steps 0 .. T-1 of K or K*: one launch per step, or all of them in one
// cooperative launch with a grid barrier between steps (b->runall).
pat_status batch_steps(pat_batch* b, int T, bool adjoint, cudaStream_t st) {
  const int nctas = adjoint ? b->nctas_adj : b->nctas;
  if (b->runall) {
    if (T <= 0) return PAT_OK;
    PAT_TRY_CUDA(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), st));
    BatchStepArgs a = step_args(b, 0, adjoint);
    a.t_end = T;
    a.active_dev = b->d_active;
    a.bar = b->d_bar;
    PAT_TRY_CUDA(batch_run_launch(b->R, b->variant, a, nctas, st));
    return PAT_OK;
  }
  for (int t = 0; t < T; ++t) PAT_TRY_CUDA(batch_step_launch(b->R, b->variant, step_args(b, t, adjoint), nctas, st));
  return PAT_OK;
}

// K of every instance: the plans' image buffers -> the plans' sensor-data buffers.
pat_status batch_forward(pat_batch* b, cudaStream_t st, int steps = -1) {
  const int T = steps < 0 ? b->max_nt : std::min(steps, b->max_nt);
  return batch_steps(b, T, false, st);
}

// K* of every instance: the plans' sensor-data buffers -> the plans' image buffers.
pat_status batch_adjoint(pat_batch* b, cudaStream_t st, int steps = -1) {
  for (pat_plan* p : b->plans) {
    PAT_TRY_CUDA(fill_launch(p->d_wv[0], p->N, 0.f, st));  // Z^{nt} = 0
    PAT_TRY_CUDA(fill_launch(p->d_wv[3], p->N, 0.f, st));  // Z_lo^{nt} = 0
    PAT_TRY_CUDA(fill_launch(p->d_wv[2], p->N, 0.f, st));  // G = 0
  }
  const int T = steps < 0 ? b->max_nt : std::min(steps, b->max_nt);
  return batch_steps(b, T, true, st);
}

// Autotuner: times the first steps of a batched K and of a batched K* with
// each tile shape and keeps the faster pair (64 x 64 tiles, or 64 x 32 tiles
// with twice as many CTAs in flight; the adjoint stages two boxes per tile, so
// it fits fewer CTAs per SM than the forward).  PAT_BATCH_TILE_Y=64|32 fixes
// the shape instead.
pat_status tune_launch(pat_batch* b, cudaStream_t st);

pat_status tune(pat_batch* b, cudaStream_t st) {
  const char* env = getenv("PAT_BATCH_TILE_Y");
  if (env && (strcmp(env, "64") == 0 || strcmp(env, "32") == 0)) {
    PAT_TRY(build_tables(b, strcmp(env, "64") == 0 ? 0 : 1, st));
    return tune_launch(b, st);
  }
  b->runall = 0;
  for (pat_plan* p : b->plans) {
    PAT_TRY_CUDA(fill_launch(p->d_img, p->N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(p->d_ybuf, (long long)p->ns * p->nt, 0.f, st));
  }
  const int steps = std::min(b->max_nt, 48);
  cudaEvent_t e0, e1;
  PAT_TRY_CUDA(cudaEventCreate(&e0));
  PAT_TRY_CUDA(cudaEventCreate(&e1));
  pat_status rc = PAT_OK;
  for (int v = 0; v < 2 && rc == PAT_OK; ++v) {
    rc = build_tables(b, v, st);
    if (rc == PAT_OK) rc = batch_forward(b, st, 4);  // warm-up
    if (rc != PAT_OK) break;
    cudaEventRecord(e0, st);
    rc = batch_forward(b, st, steps);
    if (rc == PAT_OK) rc = batch_adjoint(b, st, steps);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("batched tuning run failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = PAT_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tune_ms[v] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PAT_TRY(rc);
  const int best = b->tune_ms[1] < b->tune_ms[0] ? 1 : 0;
  if (best != b->variant) PAT_TRY(build_tables(b, best, st));
  return tune_launch(b, st);
}

// Launch form for the chosen tile shape: the first steps of a batched K plus
// K* timed as one launch per step and as one cooperative launch each (grid
// barrier between steps); the faster is kept unless the caller fixed the form.
pat_status tune_launch(pat_batch* b, cudaStream_t st) {
  for (pat_plan* p : b->plans) {
    PAT_TRY_CUDA(fill_launch(p->d_img, p->N, 0.f, st));
    PAT_TRY_CUDA(fill_launch(p->d_ybuf, (long long)p->ns * p->nt, 0.f, st));
  }
  const int steps = std::min(b->max_nt, 48);
  cudaEvent_t e0, e1;
  PAT_TRY_CUDA(cudaEventCreate(&e0));
  PAT_TRY_CUDA(cudaEventCreate(&e1));
  pat_status rc = PAT_OK;
  for (int ra = 0; ra < 2 && rc == PAT_OK; ++ra) {
    b->runall = ra;
    rc = batch_forward(b, st, 4);  // warm-up
    if (rc != PAT_OK) break;
    cudaEventRecord(e0, st);
    rc = batch_forward(b, st, steps);
    if (rc == PAT_OK) rc = batch_adjoint(b, st, steps);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("batched launch tuning failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = PAT_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->launch_ms[ra] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PAT_TRY(rc);
  int status = 0;
  PAT_TRY_CUDA(cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != PAT_OK) {
    set_error("batched kernel wait timed out while tuning");
    return (pat_status)status;
  }
  b->runall = b->launch_req == 1 ? 0 : b->launch_req == 2 ? 1 : (b->launch_ms[1] < b->launch_ms[0] ? 1 : 0);
  return PAT_OK;
}

// One CG iteration of every instance (the sequence a captured graph replays).
pat_status cg_iteration(pat_batch* b, const double* alphas, const double* ss, cudaStream_t st) {
  for (size_t i = 0; i < b->plans.size(); ++i) {
    pat_plan* p = b->plans[i];
    PAT_TRY(apply_Es(p, ss[i], p->d_p, p->d_img, st));
  }
  PAT_TRY(batch_forward(b, st));
  PAT_TRY(batch_adjoint(b, st));
  for (size_t i = 0; i < b->plans.size(); ++i) {
    pat_plan* p = b->plans[i];
    PAT_TRY(apply_EsT(p, ss[i], p->d_img, p->d_q, st));
    PAT_TRY_CUDA(cg_pq_launch(p->d_q, p->d_p, alphas[i], p->N, p->d_partials, p->d_counter, p->d_sc, st));
    PAT_TRY_CUDA(cg_update_launch(p->d_u, p->d_r, p->d_p, p->d_q, p->N, p->d_partials, p->d_counter, p->d_sc,
                                  nullptr, p->d_status, st));
    PAT_TRY_CUDA(cg_direction_launch(p->d_p, p->d_r, p->N, p->d_sc, st));
  }
  return PAT_OK;
}

// (Re)capture the CG iteration as a graph for these alphas and s values.
pat_status capture(pat_batch* b, const double* alphas, const double* ss) {
  const std::vector<double> A(alphas, alphas + b->B), S(ss, ss + b->B);
  if (b->graph && A == b->graph_alpha && S == b->graph_s) return PAT_OK;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!b->cap) PAT_TRY_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  PAT_TRY_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  const pat_status rc = cg_iteration(b, alphas, ss, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (rc != PAT_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  PAT_TRY_CUDA(e);
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  PAT_TRY_CUDA(ei);
  b->graph_nodes = nodes;
  b->graph_alpha = A;
  b->graph_s = S;
  return PAT_OK;
}

}  // namespace

bool batch_eligible(pat_plan* const* plans, int B) {
  if (B < 1 || !plans || !tma_encoder()) return false;
  for (int i = 0; i < B; ++i) {
    if (!plans[i] || ineligible(plans[i], plans[0]->R)) return false;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return false;
  }
  return true;
}

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_batch_create(pat_plan* const* plans, int B, void* stream, pat_batch** out) {
  if (!out) {
    set_error("out must not be NULL");
    return PAT_ERR_INVALID;
  }
  *out = nullptr;
  if (B < 1 || !plans) {
    set_error("a batch needs B >= 1 plans");
    return PAT_ERR_INVALID;
  }
  for (int i = 0; i < B; ++i) {
    if (!plans[i]) {
      set_error("plan %d is NULL", i);
      return PAT_ERR_INVALID;
    }
    if (const char* why = ineligible(plans[i], plans[0]->R)) {
      set_error("plan %d: %s", i, why);
      return PAT_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) {
        set_error("plan %d appears twice in the batch (each instance needs its own plan)", i);
        return PAT_ERR_INVALID;
      }
  }
  if (!tma_encoder()) {
    set_error("the driver does not provide tensor-map encoding");
    return PAT_ERR_CUDA;
  }
  pat_batch* b = new (std::nothrow) pat_batch();
  if (!b) {
    set_error("host allocation failed");
    return PAT_ERR_OOM;
  }
  b->plans.assign(plans, plans + B);
  b->B = B;
  b->R = plans[0]->R;
  b->order.resize(B);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return plans[x]->nt > plans[y]->nt; });
  b->max_nt = plans[b->order[0]]->nt;
  b->timeout_ns = plans[0]->timeout_ns;
  const pat_status rc = tune(b, (cudaStream_t)stream);
  if (rc != PAT_OK) {
    pat_batch_destroy(b);
    return rc;
  }
  *out = b;
  return PAT_OK;
}

void pat_batch_destroy(pat_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  bfree_all(b);
  delete b;
}

pat_status pat_batch_launch(pat_batch* b, int mode, int* runall, double* ms) {
  if (!b || mode < -1 || mode > 2) {
    set_error("batch must not be NULL and mode in -1 .. 2");
    return PAT_ERR_INVALID;
  }
  if (mode >= 0) {
    b->launch_req = mode;
    const int want = mode == 1 ? 0 : mode == 2 ? 1 : (b->launch_ms[1] < b->launch_ms[0] ? 1 : 0);
    if (want != b->runall) {
      b->runall = want;
      if (b->graph) {  // the captured iteration holds the other launch form
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_nodes = 0;
      }
    }
  }
  if (runall) *runall = b->runall;
  if (ms) {
    ms[0] = b->launch_ms[0];
    ms[1] = b->launch_ms[1];
  }
  return PAT_OK;
}

pat_status pat_batch_info(pat_batch* b, int* tile_rows, int* ctas, long long* graph_nodes, double* tune_ms) {
  if (!b) {
    set_error("batch is NULL");
    return PAT_ERR_INVALID;
  }
  if (tile_rows) *tile_rows = batch_tile_y(b->variant);
  if (ctas) *ctas = b->nctas;
  if (graph_nodes) *graph_nodes = (long long)b->graph_nodes;
  if (tune_ms) {
    tune_ms[0] = b->tune_ms[0];
    tune_ms[1] = b->tune_ms[1];
  }
  return PAT_OK;
}

static pat_status check_arrays(pat_batch* b, const void* const* a, const char* what) {
  if (!b) {
    set_error("batch is NULL");
    return PAT_ERR_INVALID;
  }
  if (!a) {
    set_error("%s: array of B device pointers required", what);
    return PAT_ERR_INVALID;
  }
  for (int i = 0; i < b->B; ++i)
    if (!a[i] || !device_ptr(a[i])) {
      set_error("%s[%d] must be a device pointer", what, i);
      return PAT_ERR_INVALID;
    }
  return PAT_OK;
}

pat_status pat_batch_forward(pat_batch* b, const float* const* xs, float* const* ys, void* stream) {
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(xs), "xs"));
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(ys), "ys"));
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < b->B; ++i)
    PAT_TRY_CUDA(cudaMemcpyAsync(b->plans[i]->d_img, xs[i], sizeof(float) * b->plans[i]->N,
                                 cudaMemcpyDeviceToDevice, st));
  PAT_TRY(batch_forward(b, st));
  for (int i = 0; i < b->B; ++i) {
    const pat_plan* p = b->plans[i];
    PAT_TRY_CUDA(cudaMemcpyAsync(ys[i], p->d_ybuf, sizeof(float) * p->ns * p->nt, cudaMemcpyDeviceToDevice, st));
  }
  return PAT_OK;
}

pat_status pat_batch_adjoint(pat_batch* b, const float* const* ys, float* const* xs, void* stream) {
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(ys), "ys"));
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(xs), "xs"));
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < b->B; ++i) {
    const pat_plan* p = b->plans[i];
    PAT_TRY_CUDA(cudaMemcpyAsync(p->d_ybuf, ys[i], sizeof(float) * p->ns * p->nt, cudaMemcpyDeviceToDevice, st));
  }
  PAT_TRY(batch_adjoint(b, st));
  for (int i = 0; i < b->B; ++i)
    PAT_TRY_CUDA(cudaMemcpyAsync(xs[i], b->plans[i]->d_img, sizeof(float) * b->plans[i]->N,
                                 cudaMemcpyDeviceToDevice, st));
  return PAT_OK;
}

pat_status pat_batch_solve(pat_batch* b, const float* const* ys, const double* alphas, const double* ss, int iters,
                           float* const* xs, pat_status* per_inst, void* stream) {
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(ys), "ys"));
  PAT_TRY(check_arrays(b, reinterpret_cast<const void* const*>(xs), "xs"));
  if (!alphas || !ss || iters < 0) {
    set_error("alphas and ss (B doubles each) are required and iters >= 0");
    return PAT_ERR_INVALID;
  }
  for (int i = 0; i < b->B; ++i)
    if (!(alphas[i] > 0.0) || !std::isfinite(alphas[i]) || !std::isfinite(ss[i])) {
      set_error("alpha[%d] must be finite and > 0, s[%d] finite", i, i);
      return PAT_ERR_INVALID;
    }
  cudaStream_t st = (cudaStream_t)stream;
  // right-hand sides b_i = E_s* K* y_i, CG start u = 0, p = r = b
  for (int i = 0; i < b->B; ++i) {
    const pat_plan* p = b->plans[i];
    PAT_TRY_CUDA(cudaMemcpyAsync(p->d_ybuf, ys[i], sizeof(float) * p->ns * p->nt, cudaMemcpyDeviceToDevice, st));
  }
  PAT_TRY(batch_adjoint(b, st));
  for (int i = 0; i < b->B; ++i) {
    pat_plan* p = b->plans[i];
    PAT_TRY(apply_EsT(p, ss[i], p->d_img, p->d_r, st));
    PAT_TRY_CUDA(cg_init_launch(p->d_r, p->d_r, p->d_p, p->d_u, p->N, true, p->d_partials, p->d_counter, p->d_sc, st));
  }
  if (iters > 0) {
    PAT_TRY(capture(b, alphas, ss));
    for (int k = 0; k < iters; ++k) PAT_TRY_CUDA(cudaGraphLaunch(b->graph, st));
  }
  for (int i = 0; i < b->B; ++i) PAT_TRY(apply_Es(b->plans[i], ss[i], b->plans[i]->d_u, xs[i], st));
  PAT_TRY_CUDA(cudaStreamSynchronize(st));
  int bstat = 0;
  PAT_TRY_CUDA(cudaMemcpy(&bstat, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (bstat != 0) {
    const int zero = 0;
    cudaMemcpy(b->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  }
  pat_status first = (pat_status)bstat;
  for (int i = 0; i < b->B; ++i) {
    pat_status s = pat_plan_check(b->plans[i], stream);
    if (s == PAT_OK) s = (pat_status)bstat;
    if (per_inst) per_inst[i] = s;
    if (s != PAT_OK && first == PAT_OK) first = s;
  }
  if (bstat == PAT_ERR_TIMEOUT) set_error("a bounded wait in the batched wave kernel ran out");
  return first;
}

}  // extern "C"
