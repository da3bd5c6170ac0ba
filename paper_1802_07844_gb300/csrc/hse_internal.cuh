// hse_internal.cuh -- plan structure and device helpers shared by the CUDA
// translation units of the half-space Spectral Ewald library (arXiv 1802.07844).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hse.h"

namespace hse {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kWindowC = 0.95;  // Alg. 1 step 4
constexpr int kMaxP = 32;          // support width limit (one warp lane per point)
constexpr int kCellReach = 2;      // real-space cells per r_c (cell side >= r_c / kCellReach)
constexpr int kMaxComp = 25;       // most spread components of any kernel combination
constexpr int kLowK = 8;           // mixed precision: k-points with |k_d| <= kLowK grid wave numbers scaled in FP64

// Layout of the FFT buffers: padded grid Nx x Ny x Nz = 2Mt x 2Mt x 4Mt, in-place
// R2C: real rows of pitch 2 (Nz/2 + 1) doubles, complex rows of Nz/2 + 1.
struct GridDims {
  int Mt = 0;
  int Nx = 0, Ny = 0, Nz = 0;
  int64_t pitch = 0;        // doubles per real z-row
  int64_t nh = 0;           // complex points per buffer
  int64_t buf_doubles = 0;  // real elements per buffer (double or float by precision)
};

// Spread-component description: which FFT input each component feeds and how
// its image half is formed from the source-located accumulation A:
//   mirror_sign = +1/-1 : C(k) = A(k) + s A(2Mt - k)   (C1 type: source + image)
//   mirror_sign =  0    : C(k) = A(2Mt - k)            (image-only corrections)
// kernel mask: at least one of HSE_STOKESLET / HSE_STRESSLET / HSE_ROTLET,
// optionally HSE_FREE_SPACE
inline bool valid_mask(int m) { return (m & 7) != 0 && (m & ~15) == 0; }
inline bool free_space(int m) { return (m & HSE_FREE_SPACE) != 0; }

// Derivative kind of the correction grid D for a kernel mask (product
// components): 1 the W term (stokeslet Cs), 2 first derivatives (Cv), 4 second
// derivatives (Ct); 0 in free space (no corrections).
inline int deriv_kind(int mask) {
  if (free_space(mask)) return 0;
  int dk = 2;  // every kernel has a Cv term
  if (mask & HSE_STOKESLET) dk |= 1;
  if (mask & HSE_STRESSLET) dk |= 4;
  return dk;
}
inline int c1_count(int mask) {
  return ((mask & HSE_STOKESLET) ? 3 : 0) + ((mask & HSE_STRESSLET) ? 6 : 0) + ((mask & HSE_ROTLET) ? 3 : 0);
}
// Per-particle record of the spread (elements of the grid type), three blocks
// of P entries and the components:
//   x block, entry t: {wx, XX_0 .. XX_{nxx-1}} (the window and the combined x
//                      arrays of the correction grid D) padded to kx elements
//   y block, entry t: {wy, wy', wy''} (the first nfac of them) padded to ky
//   z block, entry t: {wz, wz', wz''} padded to ky
//   components: nc values, padded to an even count
// so that a lane reads the factors of one grid offset with 16-byte loads.
// nfac = 1, 2, 3 goes with nxx = 0, 3, 6.
struct RecLayout {
  int kx, ky, x0, y0, z0, c0, stride;
  int px, py, pz;  // zero entries before and after the x, y, z blocks
};
__host__ __device__ constexpr int rec_kx(int nfac) { return nfac == 1 ? 2 : (nfac == 2 ? 4 : 8); }
__host__ __device__ constexpr int rec_ky(int nfac) { return nfac == 3 ? 4 : 2; }
// tile: the spread's warp sub-tile (hse_params.spread_tile).  Each block
// carries tile_d - 1 zero entries on both sides, so a lane whose grid point
// lies outside a source's support (at most tile_d - 1 points before or after
// it) reads zero weights: the spread needs no range test and no clamping.
__host__ __device__ inline RecLayout rec_layout(int nfac, int nc, int P, const int tile[3]) {
  RecLayout r;
  r.kx = rec_kx(nfac);
  r.ky = rec_ky(nfac);
  r.px = tile[0] - 1;
  r.py = tile[1] - 1;
  r.pz = tile[2] - 1;
  r.x0 = 0;
  r.y0 = (P + 2 * r.px) * r.kx;
  r.z0 = r.y0 + (P + 2 * r.py) * r.ky;
  r.c0 = r.z0 + (P + 2 * r.pz) * r.ky;
  r.stride = r.c0 + ((nc + 1) & ~1);
  return r;
}
// the larger of the product record (C1 + the derivative-window factors of D)
// and the paper record (C1, C2, C3 of every kernel, plain windows)
inline int prep_stride_max(int mask, int P, const int tile[3]) {
  const int dk = deriv_kind(mask);
  const int nfac = dk == 0 ? 1 : ((dk & 4) ? 3 : 2);
  const int product = rec_layout(nfac, c1_count(mask), P, tile).stride;
  const int paper = rec_layout(1, ((mask & HSE_STOKESLET) ? 7 : 0) + ((mask & HSE_STRESSLET) ? 13 : 0) +
                                      ((mask & HSE_ROTLET) ? 5 : 0), P, tile).stride;
  return product > paper ? product : paper;
}

struct CompSet {
  int n = 0;
  int mirror_sign[kMaxComp];
};

struct Workspace {
  int64_t cap = 0;   // particles
  int prep_stride = 0;  // elements per particle of prep
  int32_t *key_a = nullptr, *key_b = nullptr, *val_a = nullptr, *val_b = nullptr;
  int32_t* cell_start = nullptr;
  int64_t cell_cap = 0;
  int32_t* radix_hist = nullptr;
  int64_t hist_cap = 0;
  double* spos = nullptr;      // 3 x cap sorted source positions
  float* spos32 = nullptr;     // the same rounded to FP32 (head)
  float* spos32lo = nullptr;   // x - head, rounded to FP32 (tail)
  float* sstr32 = nullptr;     // sorted strengths in FP32 (mixed precision)
  float* sstr32lo = nullptr;   // their tails: strength - head, in FP32 (double-float pairs)
  double* usort = nullptr;     // 3 x cap real-space sums in sorted order (symmetric kernel)
  float4* usort4 = nullptr;    // cap partner sums in FP32 (mixed-precision symmetric kernel)
  double* sstr = nullptr;      // rows x cap sorted strengths
  double* prep = nullptr;      // per sorted particle: prep_stride window factors and strengths
  float* prep32 = nullptr;     // the same record in FP32 (the FP64 spread's small-weight part)
  int32_t* supp = nullptr;     // per sorted particle: ix0, iy0, iz0, pad
  int* flag = nullptr;         // device error flag
  int* flag_host = nullptr;    // pinned host mirror
};

}  // namespace hse

struct hse_plan_s {
  hse_params prm{};
  std::string err;
  bool grid_ready = false;
  // derived
  double inv_cell[3] = {0, 0, 0};
  hse::GridDims g;
  int zA0 = 0;      // lowest z index any source support can reach
  hse::CompSet comps;
  int n_rows = 0;   // strength rows
  int row_S = -1, row_T = -1, row_W = -1;
  // device grids
  double* spec = nullptr;  // n_fft_in buffers (float elements with HSE_MIXED)
  double* tabB = nullptr;  // s E B^R / Np on the octant (Mt+1)(Mt+1)(2Mt+1) (float with HSE_MIXED)
  double* tabH = nullptr;  // E H^R / Np on the octant (float with HSE_MIXED)
  // HSE_MIXED: FP64 copies of both tables on the corner |kx|, |ky|, kz <=
  // kLowK of the octant (H then B, (kLowK+1)^3 each), for the FP64 scaling of
  // the lowest wave numbers
  double* tabLow = nullptr;
  // double-float grids: the two tables again as float pairs {hi, lo} (8 bytes
  // each), so that the scaling splits no FP64 value per k-point
  double* tabB_df = nullptr;
  double* tabH_df = nullptr;
  // zero-padded transforms split into a 2-D (y,z) transform over the Mt planes
  // that hold data (fwd2d R2C / inv2d C2R) and a 1-D transform along x over
  // all (y, kz) lines (fftx, Z2Z both directions)
  cufftHandle fwd2d = 0, inv2d = 0, fftx = 0;
  bool have_fft = false;
  // double-float transforms (prm.fft == HSE_FFT_DF64): twiddle tables
  void* fft64 = nullptr;
  int fft_mode = HSE_FFT_AUTO;  // requested; resolved into prm.fft when the grids are built
  double tol = 0.0;  // tolerance the plan was created for (<= 0: explicit parameters)
  void* fft_work = nullptr;
  size_t fft_work_bytes = 0;
  hse::Workspace ws;
  // statistics of the last evaluation
  bool timing = false;
  cudaEvent_t ev[HSE_N_STAGES + 1] = {};
  // concurrent halves (hse_plan_set_overlap): real space on a low-priority
  // stream, the Fourier part on a high-priority one, joined on the caller's.
  bool overlap = false;
  // hse_plan_set_real_residency: at most this many real-space blocks per SM
  // (a persistent grid of real_bps x n_sm blocks), 0 = no cap
  int real_bps = 0;
  int n_sm = 0;  // multiprocessors of the plan's device
  cudaStream_t s_real = nullptr, s_four = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_real = nullptr, ev_four = nullptr;
  cudaEvent_t ev_real_end = nullptr;  // timing: end of the real stage on its stream
  bool last_overlap = false;
  bool ev_recorded = false;
  int n_launch = 0;
  int n_fft = 0;
};

namespace hse {

// ---------------------------------------------------------------- host utils
hse_status set_err(hse_plan p, hse_status s, const char* fmt, ...);
hse_status cuda_check(hse_plan p, cudaError_t e, const char* what);
hse_status build_grids(hse_plan p);           // tables, buffers, cuFFT plans
void free_grids(hse_plan p);
hse_status ensure_workspace(hse_plan p, int64_t n);
void free_workspace(hse_plan p);
void free_workspace(Workspace& w);
CompSet product_components(int mask);
hse_status plan_estimate(int mask, const double box[3], double xi, double tol, int precision, size_t* bytes,
                         int* M_out, int* P_out,
                         int df64_fourier = 0);
CompSet paper_components(int mask);
// smallest n' >= n whose padded transform lengths 2n', 4n' are fast sizes
int fft_friendly_size(int n);

// ----------------------------------------------------------- stage launchers
hse_status launch_validate(hse_plan p, int64_t n, const double* pos, int is_src, cudaStream_t s);
hse_status read_flag(hse_plan p, cudaStream_t s, const char* what);
hse_status build_cell_list(hse_plan p, int64_t n, const double* pos, int32_t* cell_id_out, int32_t* perm_out,
                           int32_t* start_out, cudaStream_t s);
hse_status gather_sorted(hse_plan p, int64_t n, const double* pos, const double* str, cudaStream_t s);
hse_status real_space(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                      cudaStream_t s);
hse_status neighbor_counts(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, int32_t* a, int32_t* b,
                           cudaStream_t s);
// gather_after: an event the gather waits for (the real part writing out), or null
hse_status fourier_space(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                         cudaStream_t s, cudaEvent_t gather_after = nullptr);
hse_status spread_paper_grids(hse_plan p, int64_t n_src, double* grids, cudaStream_t s);
// double-float zero-padded transforms of nb buffers, buffer b's real element
// (x, y, z) at base + x * xs + b * bs + y * pitch + z (doubles); data at
// x < Mt, y < Mt, z < 2 Mt (hse_fft64.cu)
bool fft64_supported(int Nx, int Ny, int Nz);
hse_status fft64_prepare(hse_plan p);
void fft64_destroy(hse_plan p);
hse_status fft64_forward(hse_plan p, double* base, int nb, long long bs, long long xs, cudaStream_t s);
hse_status fft64_inverse(hse_plan p, double* base, int nb, long long bs, long long xs, cudaStream_t s);
cudaError_t sort_keys_and_starts(int64_t n, int64_t ncells, int32_t* key_a, int32_t* val_a, int32_t* key_b,
                                 int32_t* val_b, int32_t* hist, int32_t* start_out, cudaStream_t s);
hse_status real_space_batch(hse_plan p, int64_t n_total, const int32_t* inst_of, double* out, cudaStream_t s);
// cuFFT plans for the batched grids of one plan.  The batched grids are
// slab-major: real element (buffer b, x, y, z) at (x * nbuf + b) * Ny * pitch
// + y * pitch + z, buffer b = component * C + instance, so that the data planes
// x < Mt of every buffer are one contiguous half and each x line has one
// stride.  Plans are made per (kind, batch, stride) on first use.
struct BatchFFT {
  struct Entry {
    int kind;
    int64_t batch, stride;
    cufftHandle h;
    size_t work;
  };
  std::vector<Entry> plans;
};
// Make the plans a chunk of n_inst instances needs and point them at a shared
// work area, grown (synchronously) when a plan needs more.
hse_status batch_fft_prepare(hse_plan p, BatchFFT& f, int n_inst, char** work, int64_t* work_cap);
void batch_fft_destroy(BatchFFT& f);
hse_status fourier_space_batch(hse_plan p, int64_t n_total, int n_inst, const int32_t* inst_of, void* spec,
                               BatchFFT& f, double* out, cudaStream_t s);

inline void stage_mark(hse_plan p, int i, cudaStream_t s) {
  if (p->timing) cudaEventRecord(p->ev[i], s);
}

// ------------------------------------------------------------- device utils
__device__ __forceinline__ int cell_coord(double x, double inv, int n) {
  double t = floor(__dmul_rn(x, inv));
  if (t < 0.0) return 0;
  if (t > (double)(n - 1)) return n - 1;
  return (int)t;
}

__device__ __forceinline__ double dist2_exact(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// support start along one axis: clamp(floor((c - o) / h) - P/2 + 1, 0, n - P)
__device__ __forceinline__ int support_start(double c, double o, double h, int P, int n) {
  double t = floor(__ddiv_rn(__dsub_rn(c, o), h));
  long long i0 = (long long)t - P / 2 + 1;
  if (i0 < 0) i0 = 0;
  if (i0 > n - P) i0 = n - P;
  return (int)i0;
}

// the same with a product by 1/h (the gather's supports)
__device__ __forceinline__ int support_start_mul(double c, double o, double inv_h, int P, int n) {
  long long i0 = (long long)floor((c - o) * inv_h) - P / 2 + 1;
  if (i0 < 0) i0 = 0;
  if (i0 > n - P) i0 = n - P;
  return (int)i0;
}

}  // namespace hse

#define HSE_TRY(expr)                     \
  do {                                    \
    hse_status _st = (expr);              \
    if (_st != HSE_OK) return _st;        \
  } while (0)

#define HSE_CUDA(p, expr) HSE_TRY(hse::cuda_check((p), (expr), #expr))
