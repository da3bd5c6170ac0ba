// hse_noalloc.cu -- cell-list build that performs no device allocation.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: applications
// whose framework or pool allocator owns the whole device heap and forbids
// foreign allocations, and time-critical loops where an allocation (which can
// synchronise the device) is not allowed.  For them, hse_cell_list_noalloc
// runs the same binning + stable sort as hse_cell_list, with its work arrays
// in one file-scope device array of fixed size instead of plan memory.  The
// array is loaded with the library and stays resident on every GPU that loads
// it until the process exits.
#include <mutex>

#include "hse_internal.cuh"

namespace hse {
cudaError_t cell_list_on_buffers(int64_t n, const double* pos, const double inv_cell[3], const int ncell[3],
                                 int32_t* key_a, int32_t* val_a, int32_t* key_b, int32_t* val_b, int32_t* hist,
                                 int32_t* cell_id_out, int32_t* start_out, cudaStream_t s);
}

namespace {

constexpr int64_t kMaxPoints = HSE_NOALLOC_MAX_POINTS;
constexpr int64_t kMaxTiles = (kMaxPoints + 2047) / 2048;
// three int32 arrays of kMaxPoints (sort keys double-buffered, the second
// value buffer; the first value buffer is the caller's perm) and the radix
// histogram (256 digits x tiles): 3.3 MiB
constexpr int64_t kScratchInts = 3 * kMaxPoints + 256 * kMaxTiles;

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device (the host-side name of the array is only a stand-in).
hse_status scratch_address(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hse::cuda_check(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return hse::set_err(nullptr, HSE_ERR_UNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hse::cuda_check(nullptr, e, "cudaGetSymbolAddress(scratch)");
    g_scratch_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return HSE_OK;
}

}  // namespace

extern "C" hse_status hse_cell_list_noalloc(int64_t n, const double* pos, const double box[3], const int ncell[3],
                                            int32_t* cell_id, int32_t* perm, int32_t* cell_start,
                                            void* cuda_stream) {
  if (n < 0 || (n > 0 && (!pos || !cell_id || !perm)) || !cell_start || !box || !ncell)
    return hse::set_err(nullptr, HSE_ERR_INVALID, "hse_cell_list_noalloc: bad arguments");
  if (n > kMaxPoints)
    return hse::set_err(nullptr, HSE_ERR_INVALID,
                        "hse_cell_list_noalloc: n = %lld exceeds the fixed scratch capacity of %lld points",
                        (long long)n, (long long)kMaxPoints);
  double inv[3];
  int64_t ncells = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(box[d] > 0.0) || ncell[d] < 1 || ncell[d] > 1024)
      return hse::set_err(nullptr, HSE_ERR_INVALID, "hse_cell_list_noalloc: box > 0 and 1 <= ncell <= 1024 needed");
    inv[d] = (double)ncell[d] / box[d];
    ncells *= ncell[d];
  }
  (void)ncells;
  int32_t* base = nullptr;
  HSE_TRY(scratch_address(&base));
  int32_t* key_a = base;
  int32_t* key_b = base + kMaxPoints;
  int32_t* val_b = base + 2 * kMaxPoints;
  int32_t* hist = base + 3 * kMaxPoints;
  // the sorted permutation is produced directly in the caller's perm array
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = hse::cell_list_on_buffers(n, pos, inv, ncell, key_a, perm, key_b, val_b, hist, cell_id,
                                            cell_start, s);
  return hse::cuda_check(nullptr, e, "hse_cell_list_noalloc");
}
