// Batched 2D engine: many independent problems (constant or varying medium)
// advanced one time step per launch over a common table of 64-column tiles.
#pragma once

#include <vector>

#include "plan.h"

namespace pat {

// One instance as seen by the batched step kernel (device memory).
struct BInst {
  int nx, ny, nt, tiles_x;
  int tile0;  // first entry of this instance in the tile table
  int ns, corners;
  float kappa0, kappa0_lo;
  const float* kappa;     // per-cell kappa of a varying medium, or nullptr (constant kappa0 + kappa0_lo)
  const float* kappa_lo;  // its rounding residual (forward), or nullptr
  const float* img;  // forward input P^0 / adjoint output x (the plan's image buffer)
  float* P[2];       // ping-pong fields: P^n (forward) or Z^m = kappa Q^m (adjoint)
  float* P_lo[2];    // adjoint: ping-pong compensation Z_lo^m
  float* D;          // increment D (forward) or G (adjoint), updated in place
  float* y;          // sensor data: forward output, adjoint input (ns x nt)
  const int* sens_cell;
  const float* sens_w;
  const int* samp;       // sensors grouped by the tile holding their base cell
  const InjCell* inj;    // injected cells grouped by tile; .local holds the cell's linear index
  const int* ent_sensor;
  const float* ent_w;
};

// One entry of the tile table (32 bytes, read as two 16-byte words).
struct alignas(16) BTile {
  int inst;        // instance slot
  int gx0, gy0;    // tile origin in the instance's grid
  int lt;          // tile index within the instance
  int s0, s1;      // range into the instance's samp list (forward sampling)
  int j0, j1;      // range into the instance's inj list (adjoint injection)
};

struct BatchStepArgs {
  const BInst* inst;
  const BTile* tiles;         // tile table
  const CUtensorMap* maps;    // BATCH_MAPS per instance: P[0], P[1], img, P_lo[0], P_lo[1] (halo boxes)
  int t;                      // global step: forward n = t, adjoint m = nt - 1 - t
  int adjoint;
  int active;                 // tiles of the instances still running at step t (a prefix of the table)
  float w[kMaxR + 1];
  int* status;
  long long timeout_ns;
  // whole-application launch (one cooperative launch for every step):
  int t_end;                  // steps t .. t_end - 1; 0 for a one-step launch
  const int* active_dev;      // active tiles per global step (device)
  unsigned* bar;              // grid-barrier arrival counter, zero at launch
};

constexpr int BATCH_MAPS = 5;

// batch.cu: every plan 2D, constant medium, one stencil order, nx % 4 == 0, no plan twice
bool batch_eligible(pat_plan* const* plans, int B);

// batch_kernels.cu
int batch_tile_y(int variant);  // tile height of a kernel variant (0: 64 rows, 1: 32 rows)
size_t batch_smem(int R, int variant, bool adj);
int batch_max_ctas(int R, int variant, bool adj);  // co-resident CTAs on this device
cudaError_t batch_step_launch(int R, int variant, const BatchStepArgs& a, int nctas, cudaStream_t st);
// All steps a.t .. a.t_end - 1 in one cooperative launch of nctas co-resident CTAs,
// a bounded grid-wide barrier between steps (a.bar zeroed beforehand).
cudaError_t batch_run_launch(int R, int variant, const BatchStepArgs& a, int nctas, cudaStream_t st);
cudaError_t batch_encode(const float* base, int nx, int ny, int R, int variant, CUtensorMap* map);

}  // namespace pat

struct pat_batch {
  std::vector<pat_plan*> plans;  // borrowed, in the caller's order
  std::vector<int> order;        // instance slots sorted by nt, longest first (slot -> caller index)
  int B = 0, R = 1, variant = 0, nctas = 0, nctas_adj = 0, max_nt = 0, ntiles = 0;
  std::vector<int> active;       // active[t]: tiles still running at global step t
  pat::BInst* d_inst = nullptr;
  pat::BTile* d_tiles = nullptr;
  CUtensorMap* d_maps = nullptr;
  int* d_status = nullptr;       // timeout of a bounded wait in the batched kernel
  int* d_active = nullptr;       // active[] in device memory (run-all launches)
  unsigned* d_bar = nullptr;     // grid-barrier counter of a run-all launch
  int runall = 0;                // 1: K / K* as one cooperative launch each; 0: one launch per time step
  int launch_req = 0;            // 0: the autotuner chooses; 1: per step; 2: one launch per application
  double launch_ms[2] = {0, 0};  // autotuner: per-step launches, one launch (first steps of K plus K*)
  long long timeout_ns = 2000000000LL;
  std::vector<void*> allocations;
  cudaStream_t cap = nullptr;    // capture stream
  cudaGraphExec_t graph = nullptr;  // one CG iteration of every instance
  std::vector<double> graph_alpha, graph_s;
  size_t graph_nodes = 0;
  double tune_ms[2] = {0, 0};
};
