// hse_batch.cu -- many small independent instances in few launches.
//
// Instances are grouped by (kernel mask, xi level), xi = 0.7 (N/V)^(1/3) on a
// factor-sqrt(2) ladder (or the level the autotuner picked for the group), so
// that a group shares one plan (r_c, M, P, truncated-kernel tables).  A group
// is processed in chunks: the chunk's particles are concatenated, binned with
// key = instance * cells + cell and sorted once, and every stage then runs as
// one launch over all instances of the chunk -- the real-space half list over
// the concatenated cell lists, the spread with one z-tile range per instance,
// batched pruned cuFFT transforms over slab-major grids (buffer b = component
// * C + instance; the data planes of all buffers form one contiguous half), the
// k-space scaling and the gather.
// Small instances alone cannot fill 152 SMs; a chunk of hundreds can.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "hse_internal.cuh"

namespace {

struct InstDesc {
  const double* src;
  const double* str;
  double* vel;
  int64_t n, off;
};

// Concatenate the chunk's instances (positions and strength rows, each
// component contiguous over the chunk), check them, and bin them into
// key = instance * cells + cell.
__global__ void k_batch_gather(const InstDesc* __restrict__ d, int n_inst, int rows, int64_t n_tot,
                               double* __restrict__ pos, double* __restrict__ str, double ix, double iy, double iz,
                               int nx, int ny, int nz, int ncells, int32_t* __restrict__ key, int32_t* __restrict__ val,
                               double L1, double L2, double L3, int* flag) {
  for (int i = blockIdx.y; i < n_inst; i += gridDim.y) {
    const InstDesc D = d[i];
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < D.n; l += (int64_t)gridDim.x * blockDim.x) {
      const int64_t g = D.off + l;
      double x = D.src[l], y = D.src[D.n + l], z = D.src[2 * D.n + l];
      pos[g] = x;
      pos[n_tot + g] = y;
      pos[2 * n_tot + g] = z;
      for (int r = 0; r < rows; ++r) {
        double v = D.str[r * D.n + l];
        str[r * n_tot + g] = v;
        if (!isfinite(v)) atomicOr(flag, 2);
      }
      bool ok = isfinite(x) && isfinite(y) && isfinite(z) && x >= 0.0 && x < L1 && y >= 0.0 && y < L2 && z > 0.0 &&
                z <= L3;
      if (!ok) atomicOr(flag, 1);
      int cx = hse::cell_coord(x, ix, nx), cy = hse::cell_coord(y, iy, ny), cz = hse::cell_coord(z, iz, nz);
      key[g] = i * ncells + (cz * ny + cy) * nx + cx;
      val[g] = (int32_t)g;
    }
  }
}

__global__ void k_inst_of(const int32_t* __restrict__ key, int64_t n, int ncells, int32_t* __restrict__ inst_of) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inst_of[i] = key[i] / ncells;
}

__global__ void k_batch_scatter(const InstDesc* __restrict__ d, int n_inst, int64_t n_tot,
                                const double* __restrict__ res) {
  for (int i = blockIdx.y; i < n_inst; i += gridDim.y) {
    const InstDesc D = d[i];
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < D.n; l += (int64_t)gridDim.x * blockDim.x)
      for (int c = 0; c < 3; ++c) D.vel[c * D.n + l] = res[c * n_tot + D.off + l];
  }
}

// spread tiles the autotuner tries (warp sub-tile along x, y, z; the first is
// the plans' default)
constexpr int kTiles[][3] = {{2, 4, 4}, {4, 4, 2}, {2, 2, 8}, {4, 2, 4}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

struct Bucket {
  int mask = 0;
  double xi = 0.0;
  int P = 0, M = 0;    // explicit support width and grid size (0: chosen from tol)
  int tile = 0;        // spread tile (index into kTiles)
  double tol = 0.0;    // tolerance the plan was made for
  hse_plan plan = nullptr;
  hse::BatchFFT fft;  // batched transforms, per chunk size met so far
};

constexpr double kMaxXStride = 256.0 * (1 << 20);

// A captured stage sequence of one chunk (sort ... scatter).  It bakes in
// sizes, the group's plan and the addresses of the batch's work arrays, so it
// is replayed only when all of them match; the caller's arrays are read
// through the device descriptor table and may change between calls.
constexpr int kGraphPtrs = 22;
struct GraphEntry {
  const void* bucket;
  int m;
  int64_t n_tot, nmax;
  const void* ptrs[kGraphPtrs];
  cudaGraphExec_t exec;
  int64_t launches, ffts;
  uint64_t last_use;
};
constexpr size_t kMaxGraphs = 64;
constexpr size_t kTrialInstances = 256;  // instances timed per autotuner trial
constexpr int kTuneSteps = 4;            // ladder steps tried in each direction
// support / grid refinement: a candidate (P, M) is kept when it is faster
// and its result on the trial instances is within kAcceptFrac tol of a plan
// made for tol / kRefFactor (the library's own tighter evaluation)
constexpr double kAcceptFrac = 0.4;
constexpr double kRefFactor = 10.0;
constexpr double kTileMargin = 0.97;
constexpr double kLadderMargin = 0.97;  // a ladder step is taken only when this much faster
constexpr int kTrialReps = 2;           // timed passes per trial (the fastest counts)

// the autotuner's choice for a (mask, default level) group
struct Choice {
  int level = 0;
  int P = 0, M = 0;  // 0: from tol
  int tile = 0;      // index into kTiles
};

double ladder_xi(int k) { return std::exp2(k / 2.0); }
int ladder_level(int64_t n, const double box[3]) {
  double v = box[0] * box[1] * box[2];
  double xi = 0.7 * std::cbrt((double)(n > 1 ? n : 1) / v);
  return (int)std::lround(2.0 * std::log2(xi));
}

}  // namespace

struct hse_batch_s {
  double tol = 0.0;
  int precision = HSE_FP64;
  double box[3] = {1, 1, 1};
  size_t budget = 0;
  int autotune = 0;
  std::map<std::pair<int, int>, Choice> tuned;  // (mask, default level) -> chosen level, P, M
  std::vector<Bucket*> buckets;
  InstDesc* d_desc = nullptr;
  InstDesc* h_desc = nullptr;
  int desc_cap = 0;
  double *d_pos = nullptr, *d_str = nullptr, *d_res = nullptr;
  int64_t pos_cap = 0, str_cap = 0, res_cap = 0;
  int32_t* inst_of = nullptr;  // instance of each sorted particle
  int64_t inst_cap = 0;
  char* spec = nullptr;        // component-major grids of one chunk (shared by all groups)
  int64_t spec_cap = 0;
  char* fft_work = nullptr;    // work area of every batched cuFFT plan
  int64_t fft_work_cap = 0;
  hse::Workspace ws;           // cell-list and particle work arrays, lent to the plan in use
  bool timing = false;
  bool graphs = true;          // replay captured stage sequences
  cudaStream_t cap = nullptr;  // capture stream (never executes work)
  std::vector<GraphEntry> graph_cache;
  uint64_t tick = 0;
  int* d_flag = nullptr;
  int* h_flag = nullptr;
  double* d_ref = nullptr;     // autotuner: reference result of the trial chunk
  int64_t ref_cap = 0;
  double* d_sums = nullptr;    // autotuner: two FP64 sums per instance of the error reduction
  int64_t sums_cap = 0;
  std::string err;
  hse_batch_stats st{};
  std::vector<const Bucket*> inst_bucket;  // group whose plan evaluated each instance of the last call
};

namespace {

// Lends the batch's work arrays to a group's plan for the duration of a scope,
// so that the plans of all groups share one (grow-only) set.
struct WorkspaceLease {
  hse_plan p;
  hse::Workspace* shared;
  WorkspaceLease(hse_plan plan, hse::Workspace* w) : p(plan), shared(w) { std::swap(p->ws, *shared); }
  ~WorkspaceLease() { std::swap(p->ws, *shared); }
};

hse_status berr(hse_batch b, hse_status s, const std::string& msg) {
  b->err = msg;
  return s;
}

hse_status bcuda(hse_batch b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HSE_OK;
  cudaGetLastError();
  return berr(b, e == cudaErrorMemoryAllocation ? HSE_ERR_OOM : HSE_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define BTRY(expr)               \
  do {                           \
    hse_status _s = (expr);      \
    if (_s != HSE_OK) return _s; \
  } while (0)

// grow-only device array of `need` elements of `esz` bytes
template <typename T>
hse_status grow(hse_batch b, T** p, int64_t* cap, int64_t need, size_t esz) {
  if (need <= *cap) return HSE_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t bytes = esz * (size_t)need;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    return berr(b, HSE_ERR_OOM,
                "cudaMalloc of " + std::to_string(bytes >> 20) + " MiB failed (" + std::to_string(fr >> 20) +
                    " MiB free)");
  }
  *cap = need;
  return HSE_OK;
}

Bucket* get_bucket(hse_batch b, int mask, double xi, hse_status* st, int P = 0, int M = 0, double tol = 0.0,
                   int tile = 0) {
  if (tol <= 0.0) tol = b->tol;
  for (Bucket* k : b->buckets)
    if (k->mask == mask && k->xi == xi && k->P == P && k->M == M && k->tol == tol && k->tile == tile) return k;
  Bucket* k = new (std::nothrow) Bucket();
  if (!k) {
    *st = berr(b, HSE_ERR_OOM, "host allocation");
    return nullptr;
  }
  k->mask = mask;
  k->xi = xi;
  k->P = P;
  k->M = M;
  k->tol = tol;
  k->tile = tile;
  *st = hse_plan_create(mask, b->box, xi, 0.0, P, tol, b->precision, &k->plan);
  if (*st == HSE_OK && M > 0) *st = hse_plan_set_grid(k->plan, M);
  if (*st == HSE_OK && tile > 0)
    *st = hse_plan_set_spread_tile(k->plan, kTiles[tile][0], kTiles[tile][1], kTiles[tile][2]);
  if (*st != HSE_OK) {
    b->err = std::string("plan: ") + hse_last_error(k->plan);
    if (k->plan) hse_plan_destroy(k->plan);
    delete k;
    return nullptr;
  }
  if (b->timing && hse_plan_set_timing(k->plan, 1) != HSE_OK) {
    *st = berr(b, HSE_ERR_CUDA, "timing events");
    hse_plan_destroy(k->plan);
    delete k;
    return nullptr;
  }
  b->buckets.push_back(k);
  ++b->st.plans;
  return k;
}

struct Chunk {
  const int* idx;  // caller's instance indices
  int m;           // instances
  int64_t n_tot;   // particles
};

// Instances per chunk: device bytes of the chunk (grids of each instance, work
// arrays of each particle; the FFT work area is bounded by the exec sizes of
// the batched transforms) against the budget, the int32 key range (instance * cells + cell), the int32 particle
// index and the 65535 limit on the spread launch's z blocks.
Chunk next_chunk(hse_batch b, Bucket* k, const hse_instance* inst, const int* idx, int remaining) {
  const hse_plan p = k->plan;
  const hse_params& q = p->prm;
  const size_t esz = b->precision == HSE_MIXED ? 4 : 8;
  const double per_inst = (double)p->g.buf_doubles * esz * p->comps.n;
  const double per_part = 320.0 + 8.0 * hse::prep_stride_max(q.kernel_mask, q.P, q.spread_tile) + 8.0 * p->n_rows;
  const int64_t ncells = (int64_t)q.ncell[0] * q.ncell[1] * q.ncell[2];
  int64_t cap = 4096;
  // the x lines of the slab-major grids have a stride of nc * C planes; past a
  // few hundred MB the transforms along x slow down (address translation), so
  // C is held to a stride of kMaxXStride bytes
  const double plane_bytes = (double)p->g.buf_doubles / p->g.Nx * esz;
  cap = std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)(kMaxXStride / (plane_bytes * p->comps.n))));
  cap = std::min<int64_t>(cap, (int64_t(1) << 30) / ncells);
  // spread grid: z blocks = instances x z tiles of 8 (up to 7 points of the
  // first tile below z = 0 with double-float grids)
  const int tz = 2 * q.spread_tile[2];  // z extent of a spread block
  cap = std::min<int64_t>(cap, 65535 / ((2 * q.Mt + 2 * tz - 2) / tz));
  const int64_t max_particles = int64_t(1) << 28;
  Chunk c{idx, 0, 0};
  while (c.m < remaining && c.m < cap) {
    int64_t n = inst[idx[c.m]].n;
    double bytes = (c.m + 1) * per_inst + (double)(c.n_tot + n) * per_part;
    if (c.m > 0 && (c.n_tot + n > max_particles || bytes > (double)b->budget)) break;
    c.n_tot += n;
    ++c.m;
  }
  return c;
}

// Allocations and cuFFT plans a chunk needs (untimed by the autotuner).
hse_status prepare_chunk(hse_batch b, Bucket* k, const Chunk& c) {
  hse_plan p = k->plan;
  const hse_params& q = p->prm;
  if (c.m > b->desc_cap) {
    cudaFree(b->d_desc);
    cudaFreeHost(b->h_desc);
    b->d_desc = nullptr;
    b->h_desc = nullptr;
    b->desc_cap = 0;
    BTRY(bcuda(b, cudaMalloc(&b->d_desc, sizeof(InstDesc) * c.m), "cudaMalloc"));
    BTRY(bcuda(b, cudaMallocHost(&b->h_desc, sizeof(InstDesc) * c.m), "cudaMallocHost"));
    b->desc_cap = c.m;
  }
  BTRY(grow(b, &b->d_pos, &b->pos_cap, 3 * c.n_tot, sizeof(double)));
  BTRY(grow(b, &b->d_str, &b->str_cap, (int64_t)p->n_rows * c.n_tot, sizeof(double)));
  BTRY(grow(b, &b->d_res, &b->res_cap, 3 * c.n_tot, sizeof(double)));
  BTRY(grow(b, &b->inst_of, &b->inst_cap, c.n_tot, sizeof(int32_t)));
  if (hse::ensure_workspace(p, c.n_tot) != HSE_OK)
    return berr(b, HSE_ERR_OOM, std::string("workspace: ") + hse_last_error(p));
  const int64_t need_cells = (int64_t)q.ncell[0] * q.ncell[1] * q.ncell[2] * c.m + 1;
  if (p->ws.cell_cap < need_cells) {
    cudaFree(p->ws.cell_start);
    p->ws.cell_start = nullptr;
    p->ws.cell_cap = 0;
    BTRY(bcuda(b, cudaMalloc(&p->ws.cell_start, sizeof(int32_t) * need_cells), "cudaMalloc"));
    p->ws.cell_cap = need_cells;
  }
  const size_t esz = b->precision == HSE_MIXED ? 4 : 8;
  BTRY(grow(b, &b->spec, &b->spec_cap, (int64_t)((size_t)p->g.buf_doubles * esz * p->comps.n * c.m), 1));
  hse_status st = hse::batch_fft_prepare(p, k->fft, c.m, &b->fft_work, &b->fft_work_cap);
  if (st != HSE_OK) return berr(b, st, hse_last_error(p));
  return HSE_OK;
}

// Stages after the input check: sort, sorted copy, instance index, real
// space, Fourier space, scatter to the instances.  *launches / *ffts count
// this library's kernels and the cuFFT executions.
hse_status enqueue_stages(hse_batch b, Bucket* k, const Chunk& c, int64_t nmax, cudaStream_t s, int64_t* launches,
                          int64_t* ffts) {
  hse_plan p = k->plan;
  const hse_params& q = p->prm;
  const int ncells = q.ncell[0] * q.ncell[1] * q.ncell[2];
  const int64_t nkeys = (int64_t)ncells * c.m;
  hse::stage_mark(p, HSE_STAGE_CELLS, s);
  BTRY(bcuda(b,
             hse::sort_keys_and_starts(c.n_tot, nkeys, p->ws.key_a, p->ws.val_a, p->ws.key_b, p->ws.val_b,
                                       p->ws.radix_hist, p->ws.cell_start, s),
             "sort"));
  int bits = 0;
  while ((int64_t(1) << bits) < nkeys) ++bits;
  const int sort_launches = 3 * ((bits + 7) / 8) + 1;
  p->n_launch = 0;
  p->n_fft = 0;
  if (hse::gather_sorted(p, c.n_tot, b->d_pos, b->d_str, s) != HSE_OK)
    return berr(b, HSE_ERR_CUDA, hse_last_error(p));
  k_inst_of<<<(unsigned)std::min<int64_t>((c.n_tot + 255) / 256, 152 * 32), 256, 0, s>>>(p->ws.key_a, c.n_tot,
                                                                                        ncells, b->inst_of);
  BTRY(bcuda(b, cudaGetLastError(), "k_inst_of"));
  hse::stage_mark(p, HSE_STAGE_REAL, s);
  hse_status st = hse::real_space_batch(p, c.n_tot, b->inst_of, b->d_res, s);
  hse::stage_mark(p, HSE_STAGE_SPREAD, s);
  if (st == HSE_OK) st = hse::fourier_space_batch(p, c.n_tot, c.m, b->inst_of, b->spec, k->fft, b->d_res, s);
  if (st != HSE_OK) return berr(b, st, hse_last_error(p));
  dim3 grid((unsigned)std::min<int64_t>((nmax + 255) / 256, 64), (unsigned)std::min(c.m, 65535));
  k_batch_scatter<<<grid, 256, 0, s>>>(b->d_desc, c.m, c.n_tot, b->d_res);
  BTRY(bcuda(b, cudaGetLastError(), "k_batch_scatter"));
  *launches = p->n_launch + sort_launches + 2;  // + k_inst_of, k_batch_scatter
  *ffts = p->n_fft;
  return HSE_OK;
}

void graph_ptrs(hse_batch b, const void** v) {
  const hse::Workspace& w = b->ws;
  const void* a[kGraphPtrs] = {b->spec,    b->fft_work, b->d_pos,  b->d_str,     b->d_res, b->inst_of, b->d_desc,
                               w.key_a,    w.val_a,     w.key_b,   w.val_b,      w.radix_hist, w.cell_start, w.spos,
                               w.spos32,   w.spos32lo,  w.sstr,    w.sstr32,     w.usort,  w.prep,
                               w.supp,     w.usort4};
  for (int i = 0; i < kGraphPtrs; ++i) v[i] = a[i];
}

// The chunk's stages as a replayed CUDA graph: found in the cache, or
// captured on the batch's capture stream and instantiated.
hse_status graph_stages(hse_batch b, Bucket* k, const Chunk& c, int64_t nmax, cudaStream_t s, int64_t* launches,
                        int64_t* ffts) {
  const void* ptrs[kGraphPtrs];
  graph_ptrs(b, ptrs);
  GraphEntry* hit = nullptr;
  for (auto& g : b->graph_cache)
    if (g.bucket == k && g.m == c.m && g.n_tot == c.n_tot && g.nmax == nmax &&
        std::equal(ptrs, ptrs + kGraphPtrs, g.ptrs)) {
      hit = &g;
      break;
    }
  if (!hit) {
    if (b->graph_cache.size() >= kMaxGraphs) {
      auto lru = std::min_element(b->graph_cache.begin(), b->graph_cache.end(),
                                  [](const GraphEntry& x, const GraphEntry& y) { return x.last_use < y.last_use; });
      cudaGraphExecDestroy(lru->exec);
      b->graph_cache.erase(lru);
    }
    GraphEntry g{};
    g.bucket = k;
    g.m = c.m;
    g.n_tot = c.n_tot;
    g.nmax = nmax;
    std::copy(ptrs, ptrs + kGraphPtrs, g.ptrs);
    BTRY(bcuda(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"));
    hse_status st = enqueue_stages(b, k, c, nmax, b->cap, &g.launches, &g.ffts);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (st != HSE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    BTRY(bcuda(b, e, "cudaStreamEndCapture"));
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    BTRY(bcuda(b, e, "cudaGraphInstantiate"));
    ++b->st.graphs_captured;
    b->graph_cache.push_back(g);
    hit = &b->graph_cache.back();
  }
  hit->last_use = ++b->tick;
  BTRY(bcuda(b, cudaGraphLaunch(hit->exec, s), "cudaGraphLaunch"));
  ++b->st.graph_launches;
  *launches = hit->launches;
  *ffts = hit->ffts;
  return HSE_OK;
}

// One chunk: descriptor upload, concatenation and input check (one stream
// synchronisation), then the stages, replayed from a graph when allowed.
hse_status run_chunk(hse_batch b, Bucket* k, const hse_instance* inst, const Chunk& c, cudaStream_t s,
                     bool allow_graph) {
  hse_plan p = k->plan;
  const hse_params& q = p->prm;
  int64_t off = 0, nmax = 0;
  for (int i = 0; i < c.m; ++i) {
    const hse_instance& I = inst[c.idx[i]];
    b->h_desc[i] = InstDesc{I.src_xyz, I.strengths, I.vel, I.n, off};
    off += I.n;
    nmax = std::max<int64_t>(nmax, I.n);
  }
  const int ncells = q.ncell[0] * q.ncell[1] * q.ncell[2];
  hse::stage_mark(p, HSE_STAGE_CHECK, s);
  BTRY(bcuda(b, cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(InstDesc) * c.m, cudaMemcpyHostToDevice, s), "copy"));
  BTRY(bcuda(b, cudaMemsetAsync(b->d_flag, 0, sizeof(int), s), "memset"));
  dim3 grid((unsigned)std::min<int64_t>((nmax + 255) / 256, 64), (unsigned)std::min(c.m, 65535));
  k_batch_gather<<<grid, 256, 0, s>>>(b->d_desc, c.m, p->n_rows, c.n_tot, b->d_pos, b->d_str, p->inv_cell[0],
                                      p->inv_cell[1], p->inv_cell[2], q.ncell[0], q.ncell[1], q.ncell[2], ncells,
                                      p->ws.key_a, p->ws.val_a, q.box[0], q.box[1], q.box[2], b->d_flag);
  BTRY(bcuda(b, cudaGetLastError(), "k_batch_gather"));
  BTRY(bcuda(b, cudaMemcpyAsync(b->h_flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "copy"));
  BTRY(bcuda(b, cudaStreamSynchronize(s), "sync"));
  if (*b->h_flag & 1) return berr(b, HSE_ERR_INVALID, "an instance has a point non-finite or outside the box");
  if (*b->h_flag & 2) return berr(b, HSE_ERR_INVALID, "an instance has a non-finite strength");
  int64_t launches = 0, ffts = 0;
  if (allow_graph && b->graphs && !b->timing) BTRY(graph_stages(b, k, c, nmax, s, &launches, &ffts));
  else BTRY(enqueue_stages(b, k, c, nmax, s, &launches, &ffts));
  hse::stage_mark(p, HSE_N_STAGES, s);
  if (b->timing) {
    // per-chunk stage times (synchronises on the chunk's last event)
    BTRY(bcuda(b, cudaEventSynchronize(p->ev[HSE_N_STAGES]), "timing"));
    for (int i = 0; i < HSE_N_STAGES; ++i) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess) b->st.stage_ms[i] += ms;
    }
  }
  b->st.chunks += 1;
  b->st.kernel_launches += launches + 1;  // + k_batch_gather
  b->st.fft_execs += ffts;
  b->st.particles += c.n_tot;
  return HSE_OK;
}

// Per instance of the chunk: the sums over its particles of |res - ref|^2
// and |ref|^2 (results component-major 3 x n_tot, instance i at d[i].off).
__global__ void k_err_sums(const InstDesc* __restrict__ d, int n_inst, int64_t n_tot, const double* __restrict__ res,
                           const double* __restrict__ ref, double* __restrict__ sums) {
  for (int i = blockIdx.y; i < n_inst; i += gridDim.y) {
    const InstDesc D = d[i];
    double e = 0.0, r = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < D.n; l += (int64_t)gridDim.x * blockDim.x)
      for (int c = 0; c < 3; ++c) {
        const int64_t k = c * n_tot + D.off + l;
        const double df = res[k] - ref[k];
        e = fma(df, df, e);
        r = fma(ref[k], ref[k], r);
      }
    for (int off = 16; off > 0; off >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, off);
      r += __shfl_xor_sync(0xffffffffu, r, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(sums + 2 * i, e);
      atomicAdd(sums + 2 * i + 1, r);
    }
  }
}

// Seconds per particle of bucket k on chunk c (a warm-up pass, then a timed
// one).  The chunk's instances keep the result, which meets tol for every
// ladder level; candidates of the (P, M) refinement are re-run by the group's
// final jobs.
hse_status trial_bucket(hse_batch b, Bucket* k, const hse_instance* inst, const Chunk& c, cudaStream_t s, double* t) {
  WorkspaceLease lease(k->plan, &b->ws);
  BTRY(prepare_chunk(b, k, c));
  BTRY(run_chunk(b, k, inst, c, s, false));
  BTRY(bcuda(b, cudaStreamSynchronize(s), "sync"));
  double best = 0.0;
  for (int rep = 0; rep < kTrialReps; ++rep) {  // the fastest of a few passes (timing noise)
    auto t0 = std::chrono::steady_clock::now();
    BTRY(run_chunk(b, k, inst, c, s, false));
    BTRY(bcuda(b, cudaStreamSynchronize(s), "sync"));
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep == 0 || dt < best) best = dt;
  }
  *t = best / (double)c.n_tot;
  for (int j = 0; j < c.m; ++j) b->inst_bucket[c.idx[j]] = k;
  return HSE_OK;
}

hse_status trial(hse_batch b, int mask, int lv, const hse_instance* inst, const std::vector<int>& idx,
                 cudaStream_t s, double* t, int* covered) {
  hse_status st = HSE_OK;
  Bucket* k = get_bucket(b, mask, ladder_xi(lv), &st);
  if (!k) return st;
  Chunk c = next_chunk(b, k, inst, idx.data(), (int)std::min<size_t>(idx.size(), kTrialInstances));
  BTRY(trial_bucket(b, k, inst, c, s, t));
  *covered = c.m;
  return HSE_OK;
}

// The largest relative RMS difference, over the chunk's instances, of the
// last chunk result (d_res) from d_ref (the descriptors of the chunk are the
// last ones uploaded).
hse_status chunk_error(hse_batch b, const Chunk& c, cudaStream_t s, double* err) {
  BTRY(grow(b, &b->d_sums, &b->sums_cap, 2 * (int64_t)c.m, sizeof(double)));
  BTRY(bcuda(b, cudaMemsetAsync(b->d_sums, 0, 2 * sizeof(double) * c.m, s), "memset"));
  int64_t nmax = 1;
  for (int i = 0; i < c.m; ++i) nmax = std::max<int64_t>(nmax, b->h_desc[i].n);
  dim3 grid((unsigned)std::min<int64_t>((nmax + 255) / 256, 64), (unsigned)std::min(c.m, 65535));
  k_err_sums<<<grid, 256, 0, s>>>(b->d_desc, c.m, c.n_tot, b->d_res, b->d_ref, b->d_sums);
  BTRY(bcuda(b, cudaGetLastError(), "k_err_sums"));
  std::vector<double> h(2 * (size_t)c.m);
  BTRY(bcuda(b, cudaMemcpyAsync(h.data(), b->d_sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s),
             "copy"));
  BTRY(bcuda(b, cudaStreamSynchronize(s), "sync"));
  double worst = 0.0;
  for (int i = 0; i < c.m; ++i)
    if (h[2 * i + 1] > 0.0) worst = std::max(worst, std::sqrt(h[2 * i] / h[2 * i + 1]));
  *err = worst;
  return HSE_OK;
}

// Support and grid refinement at the chosen level: the trial instances are
// evaluated by a plan for tol / kRefFactor (reference), then by candidates
// with a smaller P and/or a smaller FFT-friendly grid; the fastest candidate
// whose result is within kAcceptFrac tol of the reference for EVERY trial
// instance (relative RMS over the instance's own particles) is kept.  Seed: the plan's own
// (P, M) for tol at that xi (Sec. 7: xi r_c and k_inf / xi held, then perturbed).
hse_status refine_support_grid(hse_batch b, int mask, Choice* ch, double t_default, const hse_instance* inst,
                               const std::vector<int>& idx, cudaStream_t s) {
  hse_status st = HSE_OK;
  const double xi = ladder_xi(ch->level);
  double tref = b->tol / kRefFactor;
  if (b->precision == HSE_MIXED && tref < 1e-6) tref = 1e-6;
  Bucket* def = get_bucket(b, mask, xi, &st);
  if (!def) return st;
  Bucket* ref = get_bucket(b, mask, xi, &st, 0, 0, tref);
  if (!ref) return st;
  // one chunk for all: the reference plan has the largest grids
  Chunk c = next_chunk(b, ref, inst, idx.data(), (int)std::min<size_t>(idx.size(), kTrialInstances));
  double tr = 0.0;
  BTRY(trial_bucket(b, ref, inst, c, s, &tr));
  BTRY(grow(b, &b->d_ref, &b->ref_cap, 3 * c.n_tot, sizeof(double)));
  BTRY(bcuda(b, cudaMemcpyAsync(b->d_ref, b->d_res, sizeof(double) * 3 * c.n_tot, cudaMemcpyDeviceToDevice, s),
             "copy"));
  const int P0 = def->plan->prm.P, M0 = def->plan->prm.M;
  double best = t_default;
  // the default is timed on the same chunk for a fair comparison
  BTRY(trial_bucket(b, def, inst, c, s, &best));
  std::vector<std::pair<int, int>> cand;
  for (int dP : {0, 2, 4})
    for (double f : {1.0, 0.9, 0.8}) {
      const int P = P0 - dP;
      int M = (int)std::floor(f * M0);
      if (P < 4 || (dP == 0 && f == 1.0)) continue;
      M = hse::fft_friendly_size(M + P) - P;
      if (M > M0) M = M0;
      cand.emplace_back(P, M);
    }
  for (auto& pm : cand) {
    Bucket* k = get_bucket(b, mask, xi, &st, pm.first, pm.second);
    if (!k) continue;  // e.g. eta outside (0, 1) for this grid
    double t = 0.0, err = 0.0;
    if (trial_bucket(b, k, inst, c, s, &t) != HSE_OK) continue;
    if (chunk_error(b, c, s, &err) != HSE_OK) continue;
    if (err <= kAcceptFrac * b->tol && t < best) {
      best = t;
      ch->P = pm.first;
      ch->M = pm.second;
    }
  }
  // spread tile at the chosen (P, M): the sub-tile shape sets how many lanes
  // of a warp fall outside a source's support and how many blocks cover a
  // small grid's edges.  A shape replaces the default only when it is faster
  // by kTileMargin (one timed pass per trial: the margin keeps timing noise
  // from picking a shape)
  best *= kTileMargin;
  for (int tile = 1; tile < kNumTiles; ++tile) {
    Bucket* k = get_bucket(b, mask, xi, &st, ch->P, ch->M, 0.0, tile);
    if (!k) continue;
    const int tz = 2 * kTiles[tile][2], mt = k->plan->prm.Mt;
    if ((int64_t)((2 * mt + 2 * tz - 2) / tz) * c.m > 65535) continue;  // the trial chunk's z blocks
    double t = 0.0, err = 0.0;
    if (trial_bucket(b, k, inst, c, s, &t) != HSE_OK) continue;
    if (chunk_error(b, c, s, &err) != HSE_OK) continue;
    if (err <= kAcceptFrac * b->tol && t < best) {
      best = t;
      ch->tile = tile;
    }
  }
  b->err.clear();
  return HSE_OK;
}

struct Job {
  Bucket* k;
  Chunk c;
};

// Pick the group's level, support and grid (autotuning them once per (mask,
// default level)) and append its chunks to the job list.
hse_status plan_group(hse_batch b, int mask, int level, const hse_instance* inst, const std::vector<int>& idx,
                      cudaStream_t s, std::vector<Job>* jobs) {
  const std::pair<int, int> key(mask, level);
  hse_status st = HSE_OK;
  int done = 0;
  if (b->autotune && !b->tuned.count(key)) {
    // Walk the xi ladder from the default level, downwards while each step is
    // faster per particle (by kLadderMargin: trial timings are noisy), else
    // upwards; keep the fastest level.
    double best = 0.0, t = 0.0;
    int cov = 0, best_level = level;
    BTRY(trial(b, mask, level, inst, idx, s, &best, &cov));
    for (int dir : {-1, +1}) {
      for (int step = 1; step <= kTuneSteps; ++step) {
        const int lv = level + dir * step;
        if (trial(b, mask, lv, inst, idx, s, &t, &cov) != HSE_OK) break;  // e.g. no valid plan there
        if (t >= kLadderMargin * best) break;
        best = t;
        best_level = lv;
      }
      if (best_level != level) break;  // improved going down: no need to go up
    }
    b->err.clear();
    Choice ch;
    ch.level = best_level;
    BTRY(refine_support_grid(b, mask, &ch, best, inst, idx, s));
    b->tuned[key] = ch;
    ++b->st.autotuned_groups;
  }
  Choice ch;
  ch.level = level;
  auto it = b->tuned.find(key);
  if (it != b->tuned.end()) ch = it->second;
  Bucket* k = get_bucket(b, mask, ladder_xi(ch.level), &st, ch.P, ch.M, 0.0, ch.tile);
  if (!k) return st;
  while (done < (int)idx.size()) {
    Chunk c = next_chunk(b, k, inst, idx.data() + done, (int)idx.size() - done);
    jobs->push_back({k, c});
    done += c.m;
  }
  return HSE_OK;
}

}  // namespace

extern "C" hse_status hse_batch_create(double tol, int precision, const double box[3], size_t mem_budget_bytes,
                                       int autotune, hse_batch* out) {
  if (out) *out = nullptr;
  if (!out || !box || !(tol > 0.0) || (precision != HSE_FP64 && precision != HSE_MIXED) || !(box[0] > 0) ||
      !(box[1] > 0) || !(box[2] > 0))
    return hse::set_err(nullptr, HSE_ERR_INVALID, "hse_batch_create: bad arguments");
  if (precision == HSE_MIXED && tol < 1e-6)
    return hse::set_err(nullptr, HSE_ERR_INVALID, "hse_batch_create: HSE_MIXED needs tol >= 1e-6");
  hse_batch b = new (std::nothrow) hse_batch_s();
  if (!b) return hse::set_err(nullptr, HSE_ERR_OOM, "host allocation");
  b->tol = tol;
  b->precision = precision;
  for (int d = 0; d < 3; ++d) b->box[d] = box[d];
  b->autotune = autotune ? 1 : 0;
  b->budget = mem_budget_bytes;
  if (!b->budget) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return hse::set_err(nullptr, HSE_ERR_CUDA, "hse_batch_create: cudaMemGetInfo failed");
    }
    b->budget = fr / 2;
  }
  if (cudaMalloc(&b->d_flag, sizeof(int)) != cudaSuccess || cudaMallocHost(&b->h_flag, sizeof(int)) != cudaSuccess ||

      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_flag);
    cudaFree(b->d_sums);
    if (b->h_flag) cudaFreeHost(b->h_flag);
    delete b;
    return hse::set_err(nullptr, HSE_ERR_OOM, "hse_batch_create: flag or stream");
  }
  *out = b;
  return HSE_OK;
}

extern "C" hse_status hse_batch_eval(hse_batch b, int n_inst, const hse_instance* inst, void* cuda_stream) {
  if (!b) return hse::set_err(nullptr, HSE_ERR_INVALID, "hse_batch_eval: NULL batch");
  if (n_inst < 0 || (n_inst > 0 && !inst)) return berr(b, HSE_ERR_INVALID, "hse_batch_eval: bad instance array");
  b->err.clear();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  b->inst_bucket.assign((size_t)n_inst, nullptr);
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int i = 0; i < n_inst; ++i) {
    const hse_instance& I = inst[i];
    if (!hse::valid_mask(I.kernel_mask) || I.n < 1 || I.n > (int64_t(1) << 28) || !I.src_xyz ||
        !I.strengths || !I.vel)
      return berr(b, HSE_ERR_INVALID, "instance " + std::to_string(i) + ": bad descriptor");
    groups[std::make_pair(I.kernel_mask, ladder_level(I.n, b->box))].push_back(i);
  }
  b->st.instances += n_inst;
  std::vector<Job> jobs;
  for (auto& kv : groups) BTRY(plan_group(b, kv.first.first, kv.first.second, inst, kv.second, s, &jobs));
  // size every work array for the largest chunk first, so that no array moves
  // while chunks run and captured graphs stay valid from call to call
  for (const Job& j : jobs) {
    WorkspaceLease lease(j.k->plan, &b->ws);
    BTRY(prepare_chunk(b, j.k, j.c));
  }
  for (const Job& j : jobs) {
    WorkspaceLease lease(j.k->plan, &b->ws);
    BTRY(run_chunk(b, j.k, inst, j.c, s, true));
    for (int i = 0; i < j.c.m; ++i) b->inst_bucket[j.c.idx[i]] = j.k;
  }
  return HSE_OK;
}

extern "C" hse_status hse_batch_instance_params(hse_batch b, int i, hse_params* out) {
  if (!b || !out) return HSE_ERR_INVALID;
  if (i < 0 || i >= (int)b->inst_bucket.size() || !b->inst_bucket[i])
    return berr(b, HSE_ERR_INVALID, "hse_batch_instance_params: instance " + std::to_string(i) +
                                        " was not evaluated by the last call");
  *out = b->inst_bucket[i]->plan->prm;
  return HSE_OK;
}

extern "C" hse_status hse_batch_get_stats(hse_batch b, hse_batch_stats* out) {
  if (!b || !out) return HSE_ERR_INVALID;
  *out = b->st;
  out->grid_bytes = (size_t)b->spec_cap;
  out->fft_work_bytes = (size_t)b->fft_work_cap;
  const hse::Workspace& w = b->ws;
  out->particle_bytes = 8 * (size_t)(b->pos_cap + b->str_cap + b->res_cap) + 4 * (size_t)b->inst_cap +
                        (size_t)w.cap * (16 + 24 + 12 + 12 + 48 + 24 + 16 + 96 + 16 + 8 * (size_t)w.prep_stride) +
                        4 * (size_t)(w.cell_cap + w.hist_cap);
  out->plan_bytes = 0;
  for (const Bucket* k : b->buckets) out->plan_bytes += k->plan->prm.grid_bytes;
  return HSE_OK;
}

extern "C" hse_status hse_batch_set_timing(hse_batch b, int enable) {
  if (!b) return HSE_ERR_INVALID;
  b->timing = enable != 0;
  for (Bucket* k : b->buckets)
    if (hse_plan_set_timing(k->plan, b->timing ? 1 : 0) != HSE_OK) return berr(b, HSE_ERR_CUDA, "timing events");
  return HSE_OK;
}

extern "C" hse_status hse_batch_set_graphs(hse_batch b, int enable) {
  if (!b) return HSE_ERR_INVALID;
  b->graphs = enable != 0;
  return HSE_OK;
}

extern "C" const char* hse_batch_last_error(hse_batch b) { return b ? b->err.c_str() : ""; }

extern "C" hse_status hse_batch_destroy(hse_batch b) {
  if (!b) return HSE_ERR_INVALID;
  cudaDeviceSynchronize();
  for (auto& g : b->graph_cache) cudaGraphExecDestroy(g.exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (Bucket* k : b->buckets) {
    hse::batch_fft_destroy(k->fft);
    hse_plan_destroy(k->plan);
    delete k;
  }
  cudaFree(b->d_desc);
  cudaFreeHost(b->h_desc);
  cudaFree(b->d_pos);
  cudaFree(b->d_str);
  cudaFree(b->d_res);
  cudaFree(b->inst_of);
  cudaFree(b->spec);
  cudaFree(b->fft_work);
  hse::free_workspace(b->ws);
  cudaFree(b->d_flag);
  cudaFree(b->d_sums);
  cudaFree(b->d_ref);
  cudaFreeHost(b->h_flag);
  delete b;
  return HSE_OK;
}
