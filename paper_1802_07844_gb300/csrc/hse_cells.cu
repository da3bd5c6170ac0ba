// hse_cells.cu -- input checks and the real-space cell list (Sec. 5.1):
// integer binning, a stable LSD radix sort by cell id, cell starts, and the
// gather of positions and strengths into cell-sorted order.
#include "hse_internal.cuh"

namespace hse {

// ------------------------------------------------------------------ workspace
void free_workspace(hse_plan p) { free_workspace(p->ws); }

void free_workspace(Workspace& w) {
  cudaFree(w.key_a); cudaFree(w.key_b); cudaFree(w.val_a); cudaFree(w.val_b);
  cudaFree(w.cell_start); cudaFree(w.radix_hist); cudaFree(w.spos); cudaFree(w.sstr);
  cudaFree(w.prep); cudaFree(w.prep32); cudaFree(w.supp); cudaFree(w.flag); cudaFree(w.spos32); cudaFree(w.spos32lo);
  cudaFree(w.sstr32); cudaFree(w.sstr32lo); cudaFree(w.usort); cudaFree(w.usort4);
  if (w.flag_host) cudaFreeHost(w.flag_host);
  w = Workspace();
}

hse_status ensure_workspace(hse_plan p, int64_t n) {
  Workspace& w = p->ws;
  if (!w.flag) {
    HSE_CUDA(p, cudaMalloc(&w.flag, sizeof(int)));
    HSE_CUDA(p, cudaMallocHost(&w.flag_host, sizeof(int)));
  }
  int64_t ncells = (int64_t)p->prm.ncell[0] * p->prm.ncell[1] * p->prm.ncell[2];
  if (w.cell_cap < ncells + 1) {
    cudaFree(w.cell_start);
    w.cell_start = nullptr;
    HSE_CUDA(p, cudaMalloc(&w.cell_start, sizeof(int32_t) * (ncells + 1)));
    w.cell_cap = ncells + 1;
  }
  // grow-only: a workspace sized for a wider spread record or more particles
  // serves narrower / fewer ones too
  int stride = prep_stride_max(p->prm.kernel_mask, p->prm.P, p->prm.spread_tile);
  if (n <= w.cap && stride <= w.prep_stride) return HSE_OK;
  int64_t cap = n < 1024 ? 1024 : n;
  if (cap < w.cap) cap = w.cap;
  if (stride < w.prep_stride) stride = w.prep_stride;
  cudaFree(w.key_a); cudaFree(w.key_b); cudaFree(w.val_a); cudaFree(w.val_b);
  cudaFree(w.radix_hist); cudaFree(w.spos); cudaFree(w.sstr); cudaFree(w.prep); cudaFree(w.prep32); cudaFree(w.supp);
  cudaFree(w.spos32); cudaFree(w.spos32lo); cudaFree(w.sstr32); cudaFree(w.sstr32lo); cudaFree(w.usort);
  cudaFree(w.usort4);
  w.usort = nullptr;
  w.usort4 = nullptr;
  w.key_a = w.key_b = w.val_a = w.val_b = w.radix_hist = w.supp = nullptr;
  w.spos = w.sstr = w.prep = nullptr;
  w.prep32 = nullptr;
  w.spos32 = w.spos32lo = w.sstr32 = w.sstr32lo = nullptr;
  w.cap = 0;
  int64_t ntiles = (cap + 2047) / 2048;
  HSE_CUDA(p, cudaMalloc(&w.key_a, sizeof(int32_t) * cap));
  HSE_CUDA(p, cudaMalloc(&w.key_b, sizeof(int32_t) * cap));
  HSE_CUDA(p, cudaMalloc(&w.val_a, sizeof(int32_t) * cap));
  HSE_CUDA(p, cudaMalloc(&w.val_b, sizeof(int32_t) * cap));
  HSE_CUDA(p, cudaMalloc(&w.radix_hist, sizeof(int32_t) * 256 * ntiles));
  HSE_CUDA(p, cudaMalloc(&w.spos, sizeof(double) * 3 * cap));
  HSE_CUDA(p, cudaMalloc(&w.spos32, sizeof(float) * 3 * cap));
  HSE_CUDA(p, cudaMalloc(&w.spos32lo, sizeof(float) * 3 * cap));
  HSE_CUDA(p, cudaMalloc(&w.sstr32, sizeof(float) * 12 * cap));
  HSE_CUDA(p, cudaMalloc(&w.sstr32lo, sizeof(float) * 12 * cap));
  HSE_CUDA(p, cudaMalloc(&w.usort, sizeof(double) * 3 * cap));
  HSE_CUDA(p, cudaMalloc(&w.usort4, sizeof(float4) * 2 * cap));  // partner sums, then their rounding errors
  HSE_CUDA(p, cudaMalloc(&w.sstr, sizeof(double) * 12 * cap));
  HSE_CUDA(p, cudaMalloc(&w.prep, sizeof(double) * (size_t)stride * cap));
  HSE_CUDA(p, cudaMalloc(&w.prep32, sizeof(float) * (size_t)stride * cap));
  HSE_CUDA(p, cudaMalloc(&w.supp, sizeof(int32_t) * 4 * cap));
  w.hist_cap = 256 * ntiles;
  w.cap = cap;
  w.prep_stride = stride;
  return HSE_OK;
}

// --------------------------------------------------------------- validation
// Sources: finite, 0 <= x < L1, 0 <= y < L2, 0 < z <= L3.
// Targets: finite, 0 <= x < L1, 0 <= y < L2, 0 <= z <= L3.
__global__ void k_validate(int64_t n, const double* __restrict__ pos, double L1, double L2, double L3, int is_src,
                           int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    bool ok = isfinite(x) && isfinite(y) && isfinite(z) && x >= 0.0 && x < L1 && y >= 0.0 && y < L2 && z <= L3 &&
              (is_src ? z > 0.0 : z >= 0.0);
    if (!ok) atomicOr(flag, 1);
  }
}

__global__ void k_validate_str(int64_t n, const double* __restrict__ s, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(s[i])) atomicOr(flag, 2);
}

static int nblocks(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  if (b > 152 * 32) b = 152 * 32;
  return b < 1 ? 1 : (int)b;
}

hse_status launch_validate(hse_plan p, int64_t n, const double* pos, int is_src, cudaStream_t s) {
  if (n <= 0) return HSE_OK;
  k_validate<<<nblocks(n, 256), 256, 0, s>>>(n, pos, p->prm.box[0], p->prm.box[1], p->prm.box[2], is_src,
                                              p->ws.flag);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_validate");
}

hse_status launch_validate_strengths(hse_plan p, int64_t n, const double* str, cudaStream_t s) {
  if (n <= 0) return HSE_OK;
  int64_t m = n * p->n_rows;
  k_validate_str<<<nblocks(m, 256), 256, 0, s>>>(m, str, p->ws.flag);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_validate_str");
}

hse_status read_flag(hse_plan p, cudaStream_t s, const char* what) {
  HSE_CUDA(p, cudaMemcpyAsync(p->ws.flag_host, p->ws.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  HSE_CUDA(p, cudaStreamSynchronize(s));
  int f = *p->ws.flag_host;
  if (f & 1) return set_err(p, HSE_ERR_INVALID, "%s: a point is non-finite or outside the box", what);
  if (f & 2) return set_err(p, HSE_ERR_INVALID, "%s: a strength is non-finite", what);
  return HSE_OK;
}

// ------------------------------------------------------------------- binning
__global__ void k_bin(int64_t n, const double* __restrict__ pos, double ix, double iy, double iz, int nx, int ny,
                      int nz, int32_t* __restrict__ key, int32_t* __restrict__ val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int cx = cell_coord(pos[i], ix, nx);
    int cy = cell_coord(pos[n + i], iy, ny);
    int cz = cell_coord(pos[2 * n + i], iz, nz);
    key[i] = (cz * ny + cy) * nx + cx;
    val[i] = (int32_t)i;
  }
}

// ------------------------------------------------------------- radix sort
// One stable pass on 8 bits: tile histograms, exclusive scan in digit-major
// order, and a scatter that ranks equal digits in input order.
constexpr int kTile = 2048;
constexpr int kSortThreads = 256;

__global__ void k_radix_hist(const int32_t* __restrict__ key, int64_t n, int shift, int64_t ntiles,
                             int32_t* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int k = threadIdx.x; k < kTile; k += kSortThreads) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m int32 values in place, one block of 1024 threads.
__global__ void k_scan_excl(int32_t* __restrict__ a, int64_t m) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x;
  int64_t chunk = (m + 1023) / 1024;
  int64_t lo = t * chunk, hi = lo + chunk < m ? lo + chunk : m;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - s;
  for (int64_t i = lo; i < hi; ++i) {
    int32_t v = a[i];
    a[i] = (int32_t)run;
    run += v;
  }
}

__global__ void k_radix_scatter(const int32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                                int shift, int64_t ntiles, const int32_t* __restrict__ offs,
                                int32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int run[256];      // items of each digit already placed from this tile
  __shared__ int wcnt[8][256];  // per-warp digit counts of the current round
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  run[t] = (int)0;
  for (int d = 0; d < 8; ++d) wcnt[d][t] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int r = 0; r < kTile / kSortThreads; ++r) {
    int64_t i = base + (int64_t)r * kSortThreads + t;
    bool valid = i < n;
    int32_t k = valid ? kin[i] : 0;
    int dig = valid ? (k >> shift) & 255 : 256 + lane;  // invalid lanes get unique non-digits
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    int rank_in_warp = __popc(peers & ((1u << lane) - 1));
    if (valid && rank_in_warp == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    if (valid) {
      int before = run[dig];
      for (int ww = 0; ww < w; ++ww) before += wcnt[ww][dig];
      int64_t dst = (int64_t)offs[(int64_t)dig * ntiles + blockIdx.x] + before + rank_in_warp;
      kout[dst] = k;
      vout[dst] = vin[i];
    }
    __syncthreads();
    int add = 0;
    for (int ww = 0; ww < 8; ++ww) { add += wcnt[ww][t]; wcnt[ww][t] = 0; }
    run[t] += add;
    __syncthreads();
  }
}

// cell_start[c] = first sorted position with key >= c; cell_start[ncells] = n.
__global__ void k_cell_start(const int32_t* __restrict__ key, int64_t n, int64_t ncells, int32_t* __restrict__ start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t prev = i == 0 ? -1 : key[i - 1];
    int64_t cur = i == n ? ncells : key[i];
    for (int64_t c = prev + 1; c <= cur; ++c) start[c] = (int32_t)i;
  }
}

__global__ void k_gather_sorted(int64_t n, int rows, const int32_t* __restrict__ perm, const double* __restrict__ pos,
                                const double* __restrict__ str, double* __restrict__ spos, float* __restrict__ spos32,
                                float* __restrict__ spos32lo, double* __restrict__ sstr, float* __restrict__ sstr32,
                                float* __restrict__ sstr32lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = perm[i];
    for (int d = 0; d < 3; ++d) {
      double v = pos[d * n + j];
      float hi = (float)v;
      spos[d * n + i] = v;
      spos32[d * n + i] = hi;
      spos32lo[d * n + i] = (float)(v - (double)hi);
    }
    for (int r = 0; r < rows; ++r) {
      double v = str[r * n + j];
      const float hi = (float)v;
      sstr[r * n + i] = v;
      sstr32[r * n + i] = hi;
      sstr32lo[r * n + i] = (float)(v - (double)hi);
    }
  }
}

hse_status build_cell_list(hse_plan p, int64_t n, const double* pos, int32_t* cell_id_out, int32_t* perm_out,
                           int32_t* start_out, cudaStream_t s) {
  Workspace& w = p->ws;
  const int* nc = p->prm.ncell;
  int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
  int32_t* start = start_out ? start_out : w.cell_start;
  if (n == 0) {
    HSE_CUDA(p, cudaMemsetAsync(start, 0, sizeof(int32_t) * (ncells + 1), s));
    return HSE_OK;
  }
  k_bin<<<nblocks(n, 256), 256, 0, s>>>(n, pos, p->inv_cell[0], p->inv_cell[1], p->inv_cell[2], nc[0], nc[1], nc[2],
                                         w.key_a, w.val_a);
  ++p->n_launch;
  HSE_CUDA(p, cudaGetLastError());
  if (cell_id_out) HSE_CUDA(p, cudaMemcpyAsync(cell_id_out, w.key_a, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  int bits = 0;
  while ((int64_t(1) << bits) < ncells) ++bits;
  int passes = (bits + 7) / 8;
  int64_t ntiles = (n + kTile - 1) / kTile;
  int32_t *ka = w.key_a, *va = w.val_a, *kb = w.key_b, *vb = w.val_b;
  for (int ps = 0; ps < passes; ++ps) {
    int shift = 8 * ps;
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, w.radix_hist);
    k_scan_excl<<<1, 1024, 0, s>>>(w.radix_hist, 256 * ntiles);
    k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, w.radix_hist, kb, vb);
    p->n_launch += 3;
    HSE_CUDA(p, cudaGetLastError());
    int32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  // sorted keys/values are in ka/va; keep them in key_a/val_a
  if (ka != w.key_a) {
    HSE_CUDA(p, cudaMemcpyAsync(w.key_a, ka, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    HSE_CUDA(p, cudaMemcpyAsync(w.val_a, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  k_cell_start<<<nblocks(n + 1, 256), 256, 0, s>>>(w.key_a, n, ncells, start);
  ++p->n_launch;
  HSE_CUDA(p, cudaGetLastError());
  if (perm_out) HSE_CUDA(p, cudaMemcpyAsync(perm_out, w.val_a, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (start != w.cell_start)
    HSE_CUDA(p, cudaMemcpyAsync(w.cell_start, start, sizeof(int32_t) * (ncells + 1), cudaMemcpyDeviceToDevice, s));
  return HSE_OK;
}

hse_status gather_sorted(hse_plan p, int64_t n, const double* pos, const double* str, cudaStream_t s) {
  if (n == 0) return HSE_OK;
  k_gather_sorted<<<nblocks(n, 256), 256, 0, s>>>(n, str ? p->n_rows : 0, p->ws.val_a, pos, str, p->ws.spos,
                                                   p->ws.spos32, p->ws.spos32lo, p->ws.sstr, p->ws.sstr32,
                                                   p->ws.sstr32lo);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_gather_sorted");
}

}  // namespace hse

namespace hse {

// Plan-free launcher of the cell-list kernels above on caller-provided work
// arrays (used by the entry point that allocates nothing).  key_a/val_a hold
// n entries each and receive the sorted cell ids / permutation; key_b/val_b
// (n each) and hist (256 * ceil(n/2048)) are scratch.
cudaError_t cell_list_on_buffers(int64_t n, const double* pos, const double inv_cell[3], const int ncell[3],
                                 int32_t* key_a, int32_t* val_a, int32_t* key_b, int32_t* val_b, int32_t* hist,
                                 int32_t* cell_id_out, int32_t* start_out, cudaStream_t s) {
  int64_t ncells = (int64_t)ncell[0] * ncell[1] * ncell[2];
  if (n == 0) return cudaMemsetAsync(start_out, 0, sizeof(int32_t) * (ncells + 1), s);
  k_bin<<<nblocks(n, 256), 256, 0, s>>>(n, pos, inv_cell[0], inv_cell[1], inv_cell[2], ncell[0], ncell[1], ncell[2],
                                         key_a, val_a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (cell_id_out) {
    e = cudaMemcpyAsync(cell_id_out, key_a, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  int bits = 0;
  while ((int64_t(1) << bits) < ncells) ++bits;
  int passes = (bits + 7) / 8;
  int64_t ntiles = (n + kTile - 1) / kTile;
  int32_t *ka = key_a, *va = val_a, *kb = key_b, *vb = val_b;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, n, 8 * ps, ntiles, hist);
    k_scan_excl<<<1, 1024, 0, s>>>(hist, 256 * ntiles);
    k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, va, n, 8 * ps, ntiles, hist, kb, vb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != key_a) {
    e = cudaMemcpyAsync(key_a, ka, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(val_a, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  k_cell_start<<<nblocks(n + 1, 256), 256, 0, s>>>(key_a, n, ncells, start_out);
  return cudaGetLastError();
}

}  // namespace hse

namespace hse {

// Stable sort of caller-computed keys (with values) in key_a/val_a, and the
// starts of ncells key ranges.  Used by the batched instances (keys =
// instance * cells per instance + cell).
cudaError_t sort_keys_and_starts(int64_t n, int64_t ncells, int32_t* key_a, int32_t* val_a, int32_t* key_b,
                                 int32_t* val_b, int32_t* hist, int32_t* start_out, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(start_out, 0, sizeof(int32_t) * (ncells + 1), s);
  int bits = 0;
  while ((int64_t(1) << bits) < ncells) ++bits;
  int passes = (bits + 7) / 8;
  int64_t ntiles = (n + kTile - 1) / kTile;
  int32_t *ka = key_a, *va = val_a, *kb = key_b, *vb = val_b;
  cudaError_t e;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, n, 8 * ps, ntiles, hist);
    k_scan_excl<<<1, 1024, 0, s>>>(hist, 256 * ntiles);
    k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, va, n, 8 * ps, ntiles, hist, kb, vb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != key_a) {
    e = cudaMemcpyAsync(key_a, ka, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(val_a, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  k_cell_start<<<nblocks(n + 1, 256), 256, 0, s>>>(key_a, n, ncells, start_out);
  return cudaGetLastError();
}

hse_status gather_sorted_batch(hse_plan p, int64_t n, const double* pos, const double* str, cudaStream_t s) {
  return gather_sorted(p, n, pos, str, s);
}

}  // namespace hse
