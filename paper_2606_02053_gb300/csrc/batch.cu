// Batched evolution of many independent grids (threshold scan): plan, run
// (optionally as one captured CUDA graph), the stage timing and the
// autotuner that picks the work-list mapping and launch shape.  Declared in
// include/cosmos.h.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <fstream>
#include <string>
#include <vector>

#include "common.cuh"

namespace cosmos {

static size_t al256(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

static bool tuning_ok(const cosmos_batch_tuning* t) {
  if (!t) return false;
  if (t->mapping != BATCH_MAP_TILE2D && t->mapping != BATCH_MAP_LINEAR) return false;
  if (t->block_x < 1 || t->block_y < 1 || t->block_x * t->block_y != BX * BY) return false;
  return t->blocks_per_sm >= 1 && t->blocks_per_sm <= 3;
}

// Work items for a tuning; the 2D mapping needs block_x * block_y = 128 threads.
static long count_tiles(const cosmos_grid& g, const cosmos_batch_tuning& t) {
  if (t.mapping == BATCH_MAP_LINEAR) {
    const long npts = (long)g.nx * g.ny * g.nz;
    return (npts + BX * BY - 1) / (BX * BY);
  }
  return (long)((g.nx + t.block_x - 1) / t.block_x) * ((g.ny + t.block_y - 1) / t.block_y) * g.nz;
}

// Largest work list over every tuning cosmos_batch_set_tuning accepts.
static long max_tiles(const cosmos_grid& g) {
  long m = 0;
  for (int bx = 1; bx <= BX * BY; bx *= 2) {
    cosmos_batch_tuning t = {BATCH_MAP_TILE2D, bx, BX * BY / bx, 1};
    m = std::max(m, count_tiles(g, t));
  }
  cosmos_batch_tuning lin = {BATCH_MAP_LINEAR, BX, BY, 1};
  return std::max(m, count_tiles(g, lin));
}

struct BatchLayout {
  std::vector<size_t> A, B, acc, prim, flux, D, limbs;  // per instance, in doubles from ws
  size_t args, tiles, dtiles, kref, expo, erec;         // byte offsets (expo: n x nslot exponents; erec:
                                                        // the algebra passes' record, 32 unsigned per slot)
  size_t total;
};

// limb slots of the integer derivative pass (stage_int.cuh)
static int nslot_of(const cosmos_params* p) { return 24 + 2 * p->scalar; }

// BX x DBY (32 x 8) tiles of every plane: the derivative pass's work list
static long deriv_tiles(const cosmos_grid& g) {
  return (long)((g.nx + BX - 1) / BX) * ((g.ny + DBY - 1) / DBY) * g.nz;
}

static BatchLayout batch_layout(int n, const cosmos_grid* grids, const cosmos_params* p, int max_steps) {
  BatchLayout L;
  const int nf = 24 + 4 * p->fluid + 2 * p->scalar;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al256(bytes);
    return o;
  };
  long tiles = 0, dtiles = 0;
  for (int i = 0; i < n; ++i) {
    const size_t fs = (size_t)grids[i].pitch * grids[i].ny * grids[i].nz;
    L.A.push_back(take(nf * fs * 8) / 8);
    L.B.push_back(take(nf * fs * 8) / 8);
    L.acc.push_back(take(nf * fs * 8) / 8);
    L.prim.push_back(p->fluid ? take(4 * fs * 8) / 8 : 0);
    L.flux.push_back(p->fluid ? take(12 * fs * 8) / 8 : 0);
    L.D.push_back(take((size_t)nder(p->scalar) * fs * 8) / 8);
    L.limbs.push_back(take((size_t)nslot_of(p) * fs * 8) / 8);
    tiles += max_tiles(grids[i]);
    dtiles += deriv_tiles(grids[i]);
  }
  L.args = take(sizeof(StageArgs) * 4 * (size_t)n);
  L.tiles = take(sizeof(BatchTile) * (size_t)tiles);
  L.dtiles = take(sizeof(BatchTile) * (size_t)dtiles);
  L.kref = take(sizeof(double) * (size_t)max_steps * 4 * n);
  L.expo = take(sizeof(int) * (size_t)n * nslot_of(p));
  L.erec = take(sizeof(unsigned) * 32 * (size_t)n * nslot_of(p));  // per instance and slot, one line each
  L.total = off;
  return L;
}

}  // namespace cosmos

using namespace cosmos;

struct cosmos_batch_s {
  int n = 0;
  cosmos_params p;
  std::vector<cosmos_grid> grids;
  int max_steps = 0;
  cosmos_batch_tuning tune;
  int sms = 0;
  char* ws = nullptr;
  BatchLayout L;
  long ntiles = 0, ndtiles = 0;
  StageArgs* d_args = nullptr;  // [4][n]
  BatchTile* d_tiles = nullptr;
  BatchTile* d_dtiles = nullptr;  // derivative-pass tiles (BX x DBY of one z-plane; c = the plane)
  double* d_kref = nullptr;     // [max_steps][4][n]
  cudaGraphExec_t gexec = nullptr;
  int g_first = -1, g_steps = -1;
  cudaStream_t g_stream = nullptr;
};

static void drop_graph(cosmos_batch b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_first = b->g_steps = -1;
}

static int upload_tiles(cosmos_batch b) {
  std::vector<BatchTile> tiles;
  const int tpb = BX * BY;
  for (int i = 0; i < b->n; ++i) {
    const cosmos_grid& g = b->grids[i];
    if (b->tune.mapping == BATCH_MAP_LINEAR) {
      const long npts = (long)g.nx * g.ny * g.nz;
      for (long s = 0; s < npts; s += tpb) tiles.push_back(BatchTile{i, (int)s, 0, 0});
    } else {
      const int tx = (g.nx + b->tune.block_x - 1) / b->tune.block_x;
      const int ty = (g.ny + b->tune.block_y - 1) / b->tune.block_y;
      for (int k = 0; k < g.nz; ++k)
        for (int by = 0; by < ty; ++by)
          for (int bx = 0; bx < tx; ++bx) tiles.push_back(BatchTile{i, bx, by, k});
    }
  }
  // interleave instances so that consecutive work items (taken by different
  // persistent blocks in the same round) come from different grids
  std::vector<BatchTile> mixed;
  mixed.reserve(tiles.size());
  {
    std::vector<size_t> start(b->n + 1, 0);
    for (auto& t : tiles) start[t.inst + 1]++;
    for (int i = 0; i < b->n; ++i) start[i + 1] += start[i];
    std::vector<size_t> pos(start.begin(), start.end() - 1);
    bool any = true;
    while (any) {
      any = false;
      for (int i = 0; i < b->n; ++i)
        if (pos[i] < start[i + 1]) {
          mixed.push_back(tiles[pos[i]++]);
          any = true;
        }
    }
  }
  b->ntiles = (long)mixed.size();
  if (cudaMemcpy(b->d_tiles, mixed.data(), sizeof(BatchTile) * mixed.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return COSMOS_ECUDA;
  return COSMOS_OK;
}

extern "C" {

size_t cosmos_batch_workspace_bytes(int n, const cosmos_grid* grids, const cosmos_params* p, int max_steps) {
  if (n < 1 || !grids || !p || max_steps < 1) return 0;
  for (int i = 0; i < n; ++i)
    if (validate(&grids[i], p) != COSMOS_OK) return 0;
  return batch_layout(n, grids, p, max_steps).total;
}

int cosmos_batch_plan(int n, const cosmos_grid* grids, const cosmos_params* p, const double* dt, const double* t0,
                      double* const* states, int max_steps, const cosmos_batch_tuning* tuning, void* ws,
                      size_t ws_bytes, cosmos_batch* plan_out) {
  if (n < 1 || !grids || !p || !dt || !t0 || !states || max_steps < 1 || !plan_out) return COSMOS_EINVAL;
  *plan_out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (validate(&grids[i], p) != COSMOS_OK) return COSMOS_EINVAL;
    if (!states[i] || !(dt[i] > 0.0)) return COSMOS_EINVAL;
    if ((uintptr_t)states[i] & 15u) return COSMOS_EALIGN;
  }
  cosmos_batch_tuning def = {BATCH_MAP_TILE2D, BX, BY, 3};
  if (tuning && !tuning_ok(tuning)) return COSMOS_EINVAL;
  const BatchLayout L = batch_layout(n, grids, p, max_steps);
  if (!ws) return COSMOS_EINVAL;
  if (ws_bytes < L.total) return COSMOS_EWORKSPACE;
  if ((uintptr_t)ws & 255u) return COSMOS_EALIGN;

  cosmos_batch b = new cosmos_batch_s();
  b->n = n;
  b->p = *p;
  b->grids.assign(grids, grids + n);
  b->max_steps = max_steps;
  b->tune = tuning ? *tuning : def;
  b->ws = (char*)ws;
  b->L = L;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  double* wsd = (double*)ws;
  b->d_args = (StageArgs*)(b->ws + L.args);
  b->d_tiles = (BatchTile*)(b->ws + L.tiles);
  b->d_dtiles = (BatchTile*)(b->ws + L.dtiles);
  b->d_kref = (double*)(b->ws + L.kref);

  // per-stage, per-instance arguments (same fields as the single-grid stages)
  std::vector<StageArgs> args(4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double* A = wsd + L.A[i];
    double* B = wsd + L.B[i];
    double* acc = wsd + L.acc[i];
    double* U = states[i];
    const double* Us[4] = {U, A, B, A};
    double* outs[4] = {A, B, A, nullptr};
    const double cdt[4] = {0.5 * dt[i], 0.5 * dt[i], dt[i], dt[i] / 6.0};
    for (int s = 0; s < 4; ++s) {
      StageArgs& a = args[(size_t)s * n + i];
      memset(&a, 0, sizeof(a));
      a.g = make_devgrid(&grids[i]);
      a.c = make_coef(&grids[i], p->ko_sigma);
      a.ap = algebra_params(p, t0[i]);
      a.U = Us[s];
      a.U0 = U;
      a.U0w = U;
      a.out = outs[s];
      a.acc = acc;
      a.cdt = cdt[s];
      a.bk = 2.0;
      a.D = wsd + L.D[i];
      a.L = (const long long*)(wsd + L.limbs[i]);
      a.E = (const int*)(b->ws + L.expo) + (size_t)i * nslot_of(p);
      // stages 1-3 record the exponents of the state they write for the next stage
      if (s < 3) a.E_rec = (unsigned*)(b->ws + L.erec) + 32 * (size_t)i * nslot_of(p);
      if (p->fluid) {
        a.prim = wsd + L.prim[i];
        a.flux = wsd + L.flux[i];
      }
    }
  }
  // K_ref at every stage time: t = (t0 + step dt) + c_s dt, c = 0, 1/2, 1/2, 1
  // (the same sums as cosmos_rk4_step at t0 + step dt)
  static const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};
  std::vector<double> kref((size_t)max_steps * 4 * n);
  for (int st = 0; st < max_steps; ++st)
    for (int s = 0; s < 4; ++s)
      for (int i = 0; i < n; ++i) {
        const double tn = t0[i] + st * dt[i];
        const double ts = s == 0 ? tn : (s == 3 ? tn + dt[i] : tn + c_stage[s] * dt[i]);
        kref[((size_t)st * 4 + s) * n + i] = K_ref(p, ts);
      }
  if (cudaMemcpy(b->d_args, args.data(), sizeof(StageArgs) * args.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_kref, kref.data(), sizeof(double) * kref.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->ws + L.erec, 0, sizeof(unsigned) * 32 * (size_t)n * nslot_of(p)) != cudaSuccess) {
    delete b;
    return COSMOS_ECUDA;
  }
  {
    // Derivative-pass tiles instance by instance, plane by plane: the resident
    // blocks of the persistent pass then work on neighbouring planes of one grid,
    // whose z-stencils share their planes in L2 (interleaving the instances, as
    // for the pointwise passes, spread them over every grid at once and sent the
    // shared planes back to DRAM).
    std::vector<BatchTile> dt;
    for (int i = 0; i < n; ++i) {
      const cosmos_grid& g = grids[i];
      const int tx = (g.nx + BX - 1) / BX, ty = (g.ny + DBY - 1) / DBY;
      for (long w = 0; w < deriv_tiles(g); ++w)
        dt.push_back(BatchTile{i, (int)(w % tx), (int)((w / tx) % ty), (int)(w / ((long)tx * ty))});
    }
    b->ndtiles = (long)dt.size();
    if (cudaMemcpy(b->d_dtiles, dt.data(), sizeof(BatchTile) * dt.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      delete b;
      return COSMOS_ECUDA;
    }
  }
  const int e = upload_tiles(b);
  if (e != COSMOS_OK) {
    delete b;
    return e;
  }
  *plan_out = b;
  return COSMOS_OK;
}

int cosmos_batch_set_tuning(cosmos_batch b, const cosmos_batch_tuning* tuning) {
  if (!b || !tuning_ok(tuning)) return COSMOS_EINVAL;
  drop_graph(b);
  b->tune = *tuning;
  return upload_tiles(b);
}

// persistent grid of the integer derivative pass: its resident blocks on every SM
static int ideriv_blocks(cosmos_batch b) { return b->sms * COSMOS_IDERIV_MIN_BLOCKS; }

// every grid of the batch admits the integer pass's division-free periodic wrap
static bool ideriv_near(cosmos_batch b) {
  for (int i = 0; i < b->n; ++i)
    if (!near_indices(make_devgrid(&b->grids[i]))) return false;
  return true;
}

static int batch_launch_steps(cosmos_batch b, int first_step, int steps, cudaStream_t s) {
  BatchStageLauncher launch = launch_batch_stage_vac;
  if (b->p.fluid && b->p.scalar)
    launch = launch_batch_stage_fluid_scalar;
  else if (b->p.fluid)
    launch = launch_batch_stage_fluid;
  else if (b->p.scalar)
    launch = launch_batch_stage_scalar;
  const dim3 grid(b->sms * b->tune.blocks_per_sm), block(b->tune.block_x, b->tune.block_y);
  static const int modes[4] = {MODE_S1, MODE_S23, MODE_S23, MODE_S4};
  for (int st = first_step; st < first_step + steps; ++st)
    for (int stage = 0; stage < 4; ++stage) {
      const StageArgs* args = b->d_args + (size_t)stage * b->n;
      if (b->p.fluid &&
          launch_batch_fluid(args, b->d_tiles, b->ntiles, b->tune.mapping, b->p.w, grid, block, s) != cudaSuccess)
        return COSMOS_ECUDA;
      const double* kref = b->d_kref + ((size_t)st * 4 + stage) * b->n;
      const int ns = nslot_of(&b->p);
      // stage 1 scans every instance's state; stages 2-4 take the exponents the previous
      // stage's algebra pass recorded
      const cudaError_t le = stage == 0
                                 ? launch_batch_limbs(args, b->n, ns, b->p.fluid, (int*)(b->ws + b->L.expo), s)
                                 : launch_batch_to_limbs(args, b->n, ns, b->p.fluid, s);
      if (le != cudaSuccess ||
          launch(args, b->d_tiles, b->ntiles, b->tune.mapping, kref, modes[stage], grid, block, s, b->d_dtiles,
                 b->ndtiles, ideriv_blocks(b), ideriv_near(b)) != cudaSuccess)
        return COSMOS_ECUDA;
      if (stage < 3 && launch_exponents_from_record((unsigned*)(b->ws + b->L.erec), (int*)(b->ws + b->L.expo),
                                                    b->n * ns, s) != cudaSuccess)
        return COSMOS_ECUDA;
    }
  return COSMOS_OK;
}

int cosmos_batch_run(cosmos_batch b, int first_step, int steps, int use_graph, void* stream) {
  if (!b || first_step < 0 || steps < 0 || first_step + steps > b->max_steps) return COSMOS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return batch_launch_steps(b, first_step, steps, s);
  if (!s) return COSMOS_EINVAL;  // the legacy default stream cannot be captured
  if (!(b->gexec && b->g_first == first_step && b->g_steps == steps && b->g_stream == s)) {
    drop_graph(b);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return COSMOS_ECUDA;
    const int e = batch_launch_steps(b, first_step, steps, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (e != COSMOS_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e != COSMOS_OK ? e : COSMOS_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      b->gexec = nullptr;
      return COSMOS_ECUDA;
    }
    b->g_first = first_step;
    b->g_steps = steps;
    b->g_stream = s;
  }
  return cudaGraphLaunch(b->gexec, s) == cudaSuccess ? COSMOS_OK : COSMOS_ECUDA;
}

int cosmos_batch_time_stage(cosmos_batch b, int reps, double* ms_out, void* stream) {
  if (!b || reps < 1 || !ms_out) return COSMOS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  BatchStageLauncher launch = b->p.fluid ? (b->p.scalar ? launch_batch_stage_fluid_scalar : launch_batch_stage_fluid)
                                         : (b->p.scalar ? launch_batch_stage_scalar : launch_batch_stage_vac);
  const dim3 grid(b->sms * b->tune.blocks_per_sm), block(b->tune.block_x, b->tune.block_y);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return COSMOS_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return COSMOS_ECUDA;
  }
  int rc = COSMOS_OK;
  for (int r = -1; r < reps && rc == COSMOS_OK; ++r) {  // r = -1: warm-up
    if (r == 0) cudaEventRecord(e0, s);
    if (b->p.fluid &&
        launch_batch_fluid(b->d_args, b->d_tiles, b->ntiles, b->tune.mapping, b->p.w, grid, block, s) != cudaSuccess)
      rc = COSMOS_ECUDA;
    if (rc == COSMOS_OK &&
        (launch_batch_limbs(b->d_args, b->n, nslot_of(&b->p), b->p.fluid, (int*)(b->ws + b->L.expo), s) != cudaSuccess ||
         launch(b->d_args, b->d_tiles, b->ntiles, b->tune.mapping, b->d_kref, MODE_S1, grid, block, s, b->d_dtiles,
                b->ndtiles, ideriv_blocks(b), ideriv_near(b)) != cudaSuccess ||
         launch_exponents_from_record((unsigned*)(b->ws + b->L.erec), (int*)(b->ws + b->L.expo),
                                      b->n * nslot_of(&b->p), s) != cudaSuccess))  // leaves the record cleared
      rc = COSMOS_ECUDA;
  }
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) rc = COSMOS_ECUDA;
  float ms = 0.f;
  if (rc == COSMOS_OK) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return rc;
}

static const cosmos_batch_tuning kDefaultCandidates[] = {
    {BATCH_MAP_TILE2D, 32, 4, 3}, {BATCH_MAP_TILE2D, 16, 8, 3}, {BATCH_MAP_TILE2D, 64, 2, 3},
    {BATCH_MAP_TILE2D, 8, 16, 3}, {BATCH_MAP_LINEAR, 32, 4, 3}, {BATCH_MAP_LINEAR, 32, 4, 2},
    {BATCH_MAP_TILE2D, 32, 4, 2}, {BATCH_MAP_LINEAR, 32, 4, 1}};
static const int kNumDefault = (int)(sizeof(kDefaultCandidates) / sizeof(kDefaultCandidates[0]));

int cosmos_batch_default_candidates(cosmos_batch_tuning* out, int max) {
  if (out)
    for (int i = 0; i < std::min(max, kNumDefault); ++i) out[i] = kDefaultCandidates[i];
  return kNumDefault;
}

}  // extern "C"

// Cache key of a plan: device name, matter model and every grid size, in order.
static int cache_key(cosmos_batch b, std::string* key) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return COSMOS_ECUDA;
  std::string k = prop.name;
  for (char& c : k)
    if (c == '\t' || c == '\n') c = ' ';
  char buf[64];
  snprintf(buf, sizeof(buf), "|fluid=%d|scalar=%d|", b->p.fluid, b->p.scalar);
  k += buf;
  for (int i = 0; i < b->n; ++i) {
    snprintf(buf, sizeof(buf), "%s%dx%dx%d", i ? "," : "", b->grids[i].nx, b->grids[i].ny, b->grids[i].nz);
    k += buf;
  }
  *key = k;
  return COSMOS_OK;
}

// Cache file: one line per key, "<key>\t<mapping> <block_x> <block_y> <blocks_per_sm>\t<ms>".
static bool cache_lookup(const char* path, const std::string& key, cosmos_batch_tuning* t) {
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t tab = line.find('\t');
    if (tab == std::string::npos || line.compare(0, tab, key) != 0 || tab != key.size()) continue;
    cosmos_batch_tuning c;
    if (sscanf(line.c_str() + tab + 1, "%d %d %d %d", &c.mapping, &c.block_x, &c.block_y, &c.blocks_per_sm) == 4 &&
        tuning_ok(&c)) {
      *t = c;
      return true;
    }
  }
  return false;
}

// Rewrites the file with this key's line replaced or appended (through a
// temporary file renamed over the old one).
static int cache_store(const char* path, const std::string& key, const cosmos_batch_tuning& t, double ms) {
  std::vector<std::string> lines;
  {
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line))
      if (!(line.size() > key.size() && line.compare(0, key.size(), key) == 0 && line[key.size()] == '\t'))
        lines.push_back(line);
  }
  char buf[96];
  snprintf(buf, sizeof(buf), "\t%d %d %d %d\t%.6g", t.mapping, t.block_x, t.block_y, t.blocks_per_sm, ms);
  lines.push_back(key + buf);
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
  {
    std::ofstream f(tmp, std::ios::trunc);
    for (const std::string& l : lines) f << l << '\n';
    f.flush();
    if (!f) {
      remove(tmp.c_str());
      return COSMOS_EIO;
    }
  }
  if (rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return COSMOS_EIO;
  }
  return COSMOS_OK;
}

extern "C" {

int cosmos_batch_autotune(cosmos_batch b, const cosmos_batch_tuning* candidates, int n_candidates, int reps,
                          const char* cache_path, cosmos_batch_tuning* best_out, double* ms_out, int* cache_hit,
                          void* stream) {
  if (!b || reps < 1 || n_candidates < 0 || (n_candidates > 0 && !candidates)) return COSMOS_EINVAL;
  if (n_candidates == 0) {
    candidates = kDefaultCandidates;
    n_candidates = kNumDefault;
  }
  for (int i = 0; i < n_candidates; ++i)
    if (!tuning_ok(&candidates[i])) return COSMOS_EINVAL;
  if (cache_hit) *cache_hit = 0;
  std::string key;
  if (cache_path) {
    const int e = cache_key(b, &key);
    if (e != COSMOS_OK) return e;
    cosmos_batch_tuning t;
    if (cache_lookup(cache_path, key, &t)) {
      const int r = cosmos_batch_set_tuning(b, &t);
      if (r != COSMOS_OK) return r;
      if (best_out) *best_out = t;
      if (ms_out)
        for (int i = 0; i < n_candidates; ++i) ms_out[i] = NAN;
      if (cache_hit) *cache_hit = 1;
      return COSMOS_OK;
    }
  }
  int best = -1;
  double best_ms = 0.0;
  for (int i = 0; i < n_candidates; ++i) {
    double ms = 0.0;
    int r = cosmos_batch_set_tuning(b, &candidates[i]);
    if (r == COSMOS_OK) r = cosmos_batch_time_stage(b, reps, &ms, stream);
    if (r != COSMOS_OK) return r;
    if (ms_out) ms_out[i] = ms;
    if (best < 0 || ms < best_ms) {
      best = i;
      best_ms = ms;
    }
  }
  const int r = cosmos_batch_set_tuning(b, &candidates[best]);
  if (r != COSMOS_OK) return r;
  if (best_out) *best_out = candidates[best];
  return cache_path ? cache_store(cache_path, key, candidates[best], best_ms) : COSMOS_OK;
}

void cosmos_batch_free(cosmos_batch b) {
  if (!b) return;
  drop_graph(b);
  delete b;
}

}  // extern "C"
