// hse_plan.cu -- plan creation: parameter choice (Tables 2-3, Sec. 7 recipe),
// grid geometry (Alg. 1 steps 2-4), the truncated-kernel tables of Sec. 5.2 and
// the cuFFT plans of the zero-padded transforms (Alg. 1 steps 6 and 9).
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "hse_internal.cuh"

namespace hse {

// text of the last failure outside a plan, per calling thread
static thread_local std::string g_create_error;

hse_status set_err(hse_plan p, hse_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (p) p->err = buf; else g_create_error = buf;
  return s;
}

hse_status cuda_check(hse_plan p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HSE_OK;
  hse_status s = (e == cudaErrorMemoryAllocation) ? HSE_ERR_OOM : HSE_ERR_CUDA;
  cudaGetLastError();  // clear a non-sticky error
  return set_err(p, s, "%s: %s", what, cudaGetErrorString(e));
}

static hse_status cufft_check(hse_plan p, cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return HSE_OK;
  hse_status s = (r == CUFFT_ALLOC_FAILED) ? HSE_ERR_OOM : HSE_ERR_CUFFT;
  return set_err(p, s, "%s: cufft error %d", what, (int)r);
}

// ------------------------------------------------------------------------------
// Spread components.  Product path: C1 per kernel with the mirror sign of its
// image strength, and the wall corrections of all kernels merged into one
// harmonic potential phi^ = E H^R D^, D spread as one scalar grid at the images
// through window derivatives, D = Cs W + Cv . grad W - Ct : grad grad W
// (the transform of Cs^ + i k.Cv^ + k Ct^ k;  stokeslet: Cs = -2 f3,
// Cv = -2 y3 f^I; stresslet: Cv_z = 4 g.q, Ct = 4 y3 sym(g^I q^I); rotlet:
// Cv_xy = 4 (-tau2, tau1)).  Forward transforms: C1 + 1; inverse: T1 and phi.
// ------------------------------------------------------------------------------
CompSet product_components(int mask) {
  CompSet c;
  auto add = [&](int s) { c.mirror_sign[c.n++] = s; };
  if (free_space(mask)) {  // Sec. 2: C1 at the sources only, no mirror, no corrections
    if (mask & HSE_STOKESLET) for (int i = 0; i < 3; ++i) add(0);
    if (mask & HSE_STRESSLET) for (int i = 0; i < 6; ++i) add(0);
    if (mask & HSE_ROTLET) for (int i = 0; i < 3; ++i) add(0);
    return c;
  }
  if (mask & HSE_STOKESLET) { add(-1); add(-1); add(+1); }                   // -f^I  = (-f1,-f2,+f3)
  if (mask & HSE_STRESSLET) { add(-1); add(-1); add(+1); add(-1); add(+1); add(-1); }  // -sym(g^I q^I)
  if (mask & HSE_ROTLET) { add(+1); add(+1); add(-1); }                      // +tau^I
  add(0);                                                                    // D (image only)
  return c;
}

CompSet paper_components(int mask) {
  if (free_space(mask)) return product_components(mask);
  CompSet c;
  auto add = [&](int s) { c.mirror_sign[c.n++] = s; };
  if (mask & HSE_STOKESLET) { add(-1); add(-1); add(+1); for (int i = 0; i < 4; ++i) add(0); }
  if (mask & HSE_STRESSLET) {
    add(-1); add(-1); add(+1); add(-1); add(+1); add(-1);
    for (int i = 0; i < 7; ++i) add(0);
  }
  if (mask & HSE_ROTLET) { add(+1); add(+1); add(-1); add(0); add(0); }
  return c;
}

// ------------------------------------------------------------------------------
// Truncated kernels (Sec. 5.2): transforms of (1/r) 1{r<R} and r 1{r<R}.
// B^R uses the corrected closed form 4 pi [(2 - R^2k^2) cos Rk + 2Rk sin Rk - 2]/k^4
// and its Taylor series 4 pi R^4 sum (-1)^n (Rk)^2n / ((2n+1)! (2n+4)) for Rk < 1.
// ------------------------------------------------------------------------------
__device__ double trunc_H(double k, double R) {
  double x = 0.5 * R * k;
  double sinc = (x < 1e-8) ? 1.0 - x * x / 6.0 : sin(x) / x;
  return 8.0 * kPi * 0.25 * R * R * sinc * sinc;
}

__device__ double trunc_B(double k, double R) {
  double t = R * k;
  if (t < 1.0) {
    double t2 = t * t, term = 1.0, sum = 0.0;  // term = (-1)^n t^2n / (2n+1)!
    for (int n = 0; n < 20; ++n) {
      sum += term / (2.0 * n + 4.0);
      term *= -t2 / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
    }
    double R2 = R * R;
    return 4.0 * kPi * R2 * R2 * sum;
  }
  double k2 = k * k;
  return 4.0 * kPi * ((2.0 - t * t) * cos(t) + 2.0 * t * sin(t) - 2.0) / (k2 * k2);
}

// Pass 1 of the precomputation: for each fine-grid line (mx, my), sample K^R on
// the k-grid refined by s_f (spacing 2 pi/(nf h) in x, y and 2 pi/(2 nf h) in z)
// and synthesise the even cosine series along z at the padded box offsets
// iz in [0, nout).  One block per line.
__global__ void k_tab_pass1(int kind, int nf, int nfz, double h, double R, int nout, double* __restrict__ out) {
  extern __shared__ double sm[];
  int nin = nfz / 2 + 1;
  double* line = sm;           // nin
  double* ctab = sm + nin;     // nfz entries: cos(2 pi t / nfz)
  int mx = blockIdx.x, my = blockIdx.y;
  int nh = nf / 2 + 1;
  for (int t = threadIdx.x; t < nfz; t += blockDim.x) ctab[t] = cospi(2.0 * (double)t / (double)nfz);
  double ax = (double)mx / nf, ay = (double)my / nf;
  for (int m = threadIdx.x; m < nin; m += blockDim.x) {
    double az = (double)m / nfz;
    double k = 2.0 * kPi / h * sqrt(ax * ax + ay * ay + az * az);
    double v = kind == 0 ? trunc_H(k, R) : trunc_B(k, R);
    double w = (m == 0 || m == nin - 1) ? 1.0 : 2.0;
    line[m] = w * v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nout; j += blockDim.x) {
    double acc = 0.0;
    long long t = 0;
    for (int m = 0; m < nin; ++m) {
      acc += line[m] * ctab[t];
      t += j;
      if (t >= nfz) t -= nfz;
    }
    out[((size_t)mx * nh + my) * nout + j] = acc;
  }
}

// Generic even cosine pass along one axis of in[n0][n1][n2]:
//   out[.., j, ..] = scale sum_{i < nin} w_i in[.., i, ..] cos(2 pi i j / np),
// w_i = 1 at i = 0 and i = nin - 1, else 2.  The other axes keep their size.
__global__ void k_cos_pass(const double* __restrict__ in, double* __restrict__ out, int n0, int n1, int n2, int axis,
                           int nout, int np, double scale) {
  extern __shared__ double ctab[];
  for (int t = threadIdx.x; t < np; t += blockDim.x) ctab[t] = cospi(2.0 * (double)t / (double)np);
  __syncthreads();
  int d[3] = {n0, n1, n2};
  int nin = d[axis];
  int o[3] = {n0, n1, n2};
  o[axis] = nout;
  int64_t total = (int64_t)o[0] * o[1] * o[2];
  int64_t sin_[3] = {(int64_t)n1 * n2, n2, 1};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int c2 = (int)(e % o[2]);
    int c1 = (int)((e / o[2]) % o[1]);
    int c0 = (int)(e / ((int64_t)o[2] * o[1]));
    int c[3] = {c0, c1, c2};
    int j = c[axis];
    c[axis] = 0;
    const double* base = in + c[0] * sin_[0] + c[1] * sin_[1] + c[2];
    int64_t st = sin_[axis];
    double acc = 0.0;
    long long t = 0;
    for (int i = 0; i < nin; ++i) {
      double w = (i == 0 || i == nin - 1) ? 1.0 : 2.0;
      acc += w * base[i * st] * ctab[t];
      t += j;
      if (t >= np) t -= np;
    }
    out[e] = scale * acc;
  }
}

// Final tables on the padded k-grid octant: fold the remaining Gaussian
// exp(-(1 - eta) k^2 / 4 xi^2), the Hasimoto factor (1 + k^2/4xi^2) (B only)
// and the 1/Np of the unnormalised inverse FFT.
__global__ void k_tab_finish(double* __restrict__ tab, int Mt, double h, double xi, double eta, int with_s,
                             double inv_np) {
  int nx = Mt + 1, nz = 2 * Mt + 1;
  int64_t total = (int64_t)nx * nx * nz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int jz = (int)(e % nz);
    int jy = (int)((e / nz) % nx);
    int jx = (int)(e / ((int64_t)nz * nx));
    double kx = 2.0 * kPi * jx / (2.0 * Mt * h);
    double ky = 2.0 * kPi * jy / (2.0 * Mt * h);
    double kz = 2.0 * kPi * jz / (4.0 * Mt * h);
    double k2 = kx * kx + ky * ky + kz * kz;
    double q = k2 / (4.0 * xi * xi);
    double f = exp(-(1.0 - eta) * q) * inv_np;
    if (with_s) f *= (1.0 + q);
    tab[e] *= f;
  }
}

// double -> float pair {hi, lo} of every table value (double-float grids)
__global__ void k_tab_to_df(const double* __restrict__ t, float2* __restrict__ f, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = t[i];
    const float hi = __double2float_rn(v);
    f[i] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
}

// FP64 table -> FP32 copy (mixed precision)
__global__ void k_tab_to_float(const double* __restrict__ t, float* __restrict__ f, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    f[e] = (float)t[e];
}

// the corner |wx|, |wy|, kz <= K of an octant table (Mt+1)(Mt+1)(2Mt+1), in FP64
__global__ void k_tab_corner(const double* __restrict__ t, int Mt, int K, double* __restrict__ out) {
  const int n = (K + 1) * (K + 1) * (K + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int kz = e % (K + 1), wy = (e / (K + 1)) % (K + 1), wx = e / ((K + 1) * (K + 1));
    out[e] = t ? t[((int64_t)wx * (Mt + 1) + wy) * (2 * Mt + 1) + kz] : 0.0;
  }
}

static int grid_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (int)b;
}

// Builds one table (kind 0: H^R, 1: B^R) on the padded octant, Sec. 5.2:
//  1. sample K^R on the k-grid refined by s_f (nf = s_f Mt even, s_f >= 1 + sqrt 6),
//  2. inverse transform (even cosine synthesis) and truncate to the padded box,
//  3. forward transform on the padded grid (even cosine analysis).
static hse_status build_table(hse_plan p, int kind, double* tab) {
  const int Mt = p->g.Mt;
  const double h = p->prm.h;
  const double R = std::sqrt(6.0) * Mt * h;  // diagonal of the Lt x Lt x 2Lt domain
  int nf = (int)std::ceil((1.0 + std::sqrt(6.0)) * Mt);
  if (nf % 2) ++nf;
  const int nfz = 2 * nf;
  const int nh = nf / 2 + 1;
  const int ox = Mt + 1, oz = 2 * Mt + 1;  // octant of the padded box / k-grid
  double *a = nullptr, *b = nullptr;
  size_t na = (size_t)nh * nh * oz, nb = (size_t)nh * ox * oz;
  HSE_CUDA(p, cudaMalloc(&a, na * sizeof(double)));
  cudaError_t e = cudaMalloc(&b, nb * sizeof(double));
  if (e != cudaSuccess) { cudaFree(a); return cuda_check(p, e, "cudaMalloc table scratch"); }
  hse_status st = HSE_OK;
  // Every thread sets the same (device maximum) limit, so plans built
  // concurrently from several threads cannot lower it under each other.
  int dev = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncSetAttribute(k_tab_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  cudaFuncSetAttribute(k_cos_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  do {
    size_t sm1 = sizeof(double) * (nfz / 2 + 1 + nfz);
    if (sm1 > (size_t)smax) {
      st = set_err(p, HSE_ERR_UNSUPPORTED, "grid too large for the table precompute (Mt = %d)", Mt);
      break;
    }
    k_tab_pass1<<<dim3(nh, nh), 256, sm1>>>(kind, nf, nfz, h, R, oz, a);             // a[mx][my][iz]
    if ((st = cuda_check(p, cudaGetLastError(), "k_tab_pass1")) != HSE_OK) break;
    auto pass = [&](const double* in, double* out, int n0, int n1, int n2, int axis, int nout, int np, double sc) {
      int o[3] = {n0, n1, n2};
      o[axis] = nout;
      int64_t tot = (int64_t)o[0] * o[1] * o[2];
      size_t smb = sizeof(double) * np;
      k_cos_pass<<<grid_blocks(tot, 256), 256, smb>>>(in, out, n0, n1, n2, axis, nout, np, sc);
      return cuda_check(p, cudaGetLastError(), "k_cos_pass");
    };
    // synthesis along y then x; 1/(nf nf nfz) is the discrete inverse normalisation
    if ((st = pass(a, b, nh, nh, oz, 1, ox, nf, 1.0)) != HSE_OK) break;                 // b[mx][iy][iz]
    if ((st = pass(b, a, nh, ox, oz, 0, ox, nf, 1.0 / ((double)nf * nf * nfz))) != HSE_OK) break;  // a[ix][iy][iz]
    // analysis on the padded grid (Nx = 2Mt, Nz = 4Mt): z, y, x
    if ((st = pass(a, b, ox, ox, oz, 2, oz, 4 * Mt, 1.0)) != HSE_OK) break;
    if ((st = pass(b, a, ox, ox, oz, 1, ox, 2 * Mt, 1.0)) != HSE_OK) break;
    if ((st = pass(a, tab, ox, ox, oz, 0, ox, 2 * Mt, 1.0)) != HSE_OK) break;
    double inv_np = 1.0 / ((double)p->g.Nx * p->g.Ny * p->g.Nz);
    int64_t tot = (int64_t)ox * ox * oz;
    k_tab_finish<<<grid_blocks(tot, 256), 256>>>(tab, Mt, h, p->prm.xi, p->prm.eta, kind == 1, inv_np);
    if ((st = cuda_check(p, cudaGetLastError(), "k_tab_finish")) != HSE_OK) break;
    st = cuda_check(p, cudaDeviceSynchronize(), "table precompute");
  } while (0);
  cudaFree(a);
  cudaFree(b);
  return st;
}

void free_grids(hse_plan p) {
  if (p->have_fft) {
    cufftDestroy(p->fwd2d);
    cufftDestroy(p->inv2d);
    cufftDestroy(p->fftx);
    p->have_fft = false;
  }
  cudaFree(p->fft_work);
  fft64_destroy(p);
  cudaFree(p->spec);
  cudaFree(p->tabB);
  cudaFree(p->tabH);
  cudaFree(p->tabLow);
  cudaFree(p->tabB_df);
  cudaFree(p->tabH_df);
  p->tabLow = p->tabB_df = p->tabH_df = nullptr;
  p->fft_work = nullptr;
  p->fft_work_bytes = 0;
  p->spec = p->tabB = p->tabH = nullptr;
  p->grid_ready = false;
}

// Float-pair copies of the tables for double-float grids (made once, with
// the df64 transforms)
static hse_status prepare_df_tables(hse_plan p) {
  if (p->tabH_df) return HSE_OK;
  const int Mt = p->prm.Mt;
  const int64_t n = (int64_t)(Mt + 1) * (Mt + 1) * (2 * Mt + 1);
  for (int k = 0; k < 2; ++k) {
    double* src = k == 0 ? p->tabH : p->tabB;
    double** dst = k == 0 ? &p->tabH_df : &p->tabB_df;
    if (!src) continue;
    HSE_CUDA(p, cudaMalloc(dst, n * sizeof(double)));
    k_tab_to_df<<<grid_blocks(n, 256), 256>>>(src, reinterpret_cast<float2*>(*dst), n);
    HSE_CUDA(p, cudaGetLastError());
  }
  HSE_CUDA(p, cudaDeviceSynchronize());
  p->prm.grid_bytes += (size_t)n * sizeof(double) * (p->tabB ? 2 : 1);
  return HSE_OK;
}

// Transforms for the plan's grid.  Double-float transforms carry ~48-bit
// arithmetic (rounding ~1e-14 of the data norm), so the automatic choice keeps
// cuFFT double for tolerances below 1e-12; FP32 plans always use cuFFT single.
constexpr double kDf64MinTol = 1e-12;
// HSE_MIXED plans take cuFFT single unless HSE_FFT_DF64 is asked for (FP32
// real space with a double-float Fourier part).
static int resolve_fft(hse_plan p) {
  const hse_params& q = p->prm;
  const bool ok = fft64_supported(p->g.Nx, p->g.Ny, p->g.Nz);
  if (q.precision != HSE_FP64) return p->fft_mode == HSE_FFT_DF64 ? (ok ? HSE_FFT_DF64 : -1) : HSE_FFT_CUFFT;
  if (p->fft_mode == HSE_FFT_DF64) return ok ? HSE_FFT_DF64 : -1;
  if (p->fft_mode == HSE_FFT_CUFFT) return HSE_FFT_CUFFT;
  return ok && (p->tol <= 0.0 || p->tol >= kDf64MinTol) ? HSE_FFT_DF64 : HSE_FFT_CUFFT;
}

// cuFFT plans of the single-plan path (HSE_FFT_CUFFT, and every HSE_MIXED plan)
static hse_status build_cufft(hse_plan p) {
  if (p->have_fft) return HSE_OK;
  const hse_params& q = p->prm;
  const GridDims& g = p->g;
  const bool mixed = q.precision == HSE_MIXED;
  // cuFFT, in place: the input is zero outside x < Mt, y < Mt, z < 2Mt, so the
  // forward transform is a 2-D (y,z) R2C over the Mt planes x < Mt followed by
  // a 1-D transform along x over every (y, kz) line; the inverse runs the x
  // transform first and the 2-D C2R only over the planes the gather reads.
  const long long nzh = g.Nz / 2 + 1;
  long long n2[2] = {g.Ny, g.Nz};
  long long re[2] = {g.Ny, g.pitch}, ce[2] = {g.Ny, nzh};
  long long nx[1] = {g.Nx}, xe[1] = {g.Nx};
  size_t w1 = 0, w2 = 0, w3 = 0;
  HSE_TRY(cufft_check(p, cufftCreate(&p->fwd2d), "cufftCreate"));
  HSE_TRY(cufft_check(p, cufftCreate(&p->inv2d), "cufftCreate"));
  HSE_TRY(cufft_check(p, cufftCreate(&p->fftx), "cufftCreate"));
  p->have_fft = true;
  cufftSetAutoAllocation(p->fwd2d, 0);
  cufftSetAutoAllocation(p->inv2d, 0);
  cufftSetAutoAllocation(p->fftx, 0);
  const cufftType t_r2c = mixed ? CUFFT_R2C : CUFFT_D2Z, t_c2r = mixed ? CUFFT_C2R : CUFFT_Z2D;
  const cufftType t_c2c = mixed ? CUFFT_C2C : CUFFT_Z2Z;
  HSE_TRY(cufft_check(p, cufftMakePlanMany64(p->fwd2d, 2, n2, re, 1, g.Ny * g.pitch, ce, 1, g.Ny * nzh, t_r2c,
                                             q.Mt, &w1), "cufftMakePlanMany64 R2C (y,z)"));
  HSE_TRY(cufft_check(p, cufftMakePlanMany64(p->inv2d, 2, n2, ce, 1, g.Ny * nzh, re, 1, g.Ny * g.pitch, t_c2r,
                                             q.Mt, &w2), "cufftMakePlanMany64 C2R (y,z)"));
  HSE_TRY(cufft_check(p, cufftMakePlanMany64(p->fftx, 1, nx, xe, g.Ny * nzh, 1, xe, g.Ny * nzh, 1, t_c2c,
                                             g.Ny * nzh, &w3), "cufftMakePlanMany64 C2C (x)"));
  size_t wmax = w1 > w2 ? w1 : w2;
  p->fft_work_bytes = wmax > w3 ? wmax : w3;
  if (p->fft_work_bytes) HSE_CUDA(p, cudaMalloc(&p->fft_work, p->fft_work_bytes));
  HSE_TRY(cufft_check(p, cufftSetWorkArea(p->fwd2d, p->fft_work), "cufftSetWorkArea"));
  HSE_TRY(cufft_check(p, cufftSetWorkArea(p->inv2d, p->fft_work), "cufftSetWorkArea"));
  HSE_TRY(cufft_check(p, cufftSetWorkArea(p->fftx, p->fft_work), "cufftSetWorkArea"));
  return HSE_OK;
}

hse_status build_grids(hse_plan p) {
  free_grids(p);
  hse_params& q = p->prm;
  q.h = q.L / q.M;
  q.Mt = q.M + q.P;
  q.eta = q.P * q.xi * q.xi * q.h * q.h / (kWindowC * kWindowC * kPi);
  if (!(q.eta > 0.0 && q.eta < 1.0))
    return set_err(p, HSE_ERR_INVALID, "eta = %g outside (0,1): increase M (M=%d, P=%d, xi=%g)", q.eta, q.M, q.P,
                   q.xi);
  GridDims& g = p->g;
  g.Mt = q.Mt;
  g.Nx = g.Ny = 2 * q.Mt;
  g.Nz = 4 * q.Mt;
  g.pitch = 2 * (g.Nz / 2 + 1);
  g.nh = (int64_t)g.Nx * g.Ny * (g.Nz / 2 + 1);
  g.buf_doubles = 2 * g.nh;
  p->zA0 = q.Mt - q.P / 2 + 1;
  p->comps = product_components(q.kernel_mask);
  q.n_fft_in = p->comps.n;
  q.n_fft_out = free_space(q.kernel_mask) ? 3 : 4;  // T1 (and phi with a wall)
  q.fft = resolve_fft(p);
  if (q.fft < 0) return set_err(p, HSE_ERR_UNSUPPORTED, "df64 FFT: grid %d x %d x %d", g.Nx, g.Ny, g.Nz);
  // FP32 grids and tables: HSE_MIXED plans on cuFFT single; double-float or
  // FP64 grids otherwise (8-byte elements)
  const bool mixed = q.precision == HSE_MIXED && q.fft != HSE_FFT_DF64;
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  size_t tab_elems = (size_t)(q.Mt + 1) * (q.Mt + 1) * (2 * q.Mt + 1);
  size_t spec_bytes = (size_t)g.buf_doubles * esz * q.n_fft_in;
  HSE_CUDA(p, cudaMalloc(&p->spec, spec_bytes));
  HSE_CUDA(p, cudaMalloc(&p->tabH, tab_elems * sizeof(double)));
  if (q.kernel_mask & (HSE_STOKESLET | HSE_STRESSLET)) HSE_CUDA(p, cudaMalloc(&p->tabB, tab_elems * sizeof(double)));
  HSE_TRY(build_table(p, 0, p->tabH));
  if (p->tabB) HSE_TRY(build_table(p, 1, p->tabB));
  if (mixed) {  // the tables are built in FP64 and rounded to FP32 once
    // except for their low-wave-number corner, kept in FP64 for the scaling
    const int K = kLowK < q.Mt ? kLowK : q.Mt;
    const int nlow = (K + 1) * (K + 1) * (K + 1);
    HSE_CUDA(p, cudaMalloc(&p->tabLow, 2 * nlow * sizeof(double)));
    k_tab_corner<<<grid_blocks(nlow, 256), 256>>>(p->tabH, q.Mt, K, p->tabLow);
    k_tab_corner<<<grid_blocks(nlow, 256), 256>>>(p->tabB, q.Mt, K, p->tabLow + nlow);
    HSE_CUDA(p, cudaGetLastError());
    for (double** tp : {&p->tabH, &p->tabB}) {
      if (!*tp) continue;
      float* f = nullptr;
      HSE_CUDA(p, cudaMalloc(&f, tab_elems * sizeof(float)));
      k_tab_to_float<<<grid_blocks((int64_t)tab_elems, 256), 256>>>(*tp, f, (int64_t)tab_elems);
      cudaError_t e = cudaDeviceSynchronize();
      cudaFree(*tp);
      *tp = reinterpret_cast<double*>(f);
      HSE_CUDA(p, e);
    }
  }
  if (q.fft == HSE_FFT_DF64) HSE_TRY(fft64_prepare(p));
  else HSE_TRY(build_cufft(p));
  q.grid_bytes = spec_bytes + tab_elems * esz * (p->tabB ? 2 : 1) + p->fft_work_bytes;
  if (q.fft == HSE_FFT_DF64) HSE_TRY(prepare_df_tables(p));
  p->grid_ready = true;
  return HSE_OK;
}

// ------------------------------------------------------------------------------
// Parameter choice from a relative RMS tolerance (Sec. 6-7).
// The truncation estimates of Tables 2-3 (absolute RMS errors, with Q the sum
// of squared strengths) are made relative with the RMS velocity model
// |u|_rms ~ sqrt(4 pi Q)/L (uniform sources, stokeslet; the more singular
// stresslet and rotlet fields are larger, so the rule is conservative there):
//   real space  S: sqrt(rc/(pi L)) e^{-xi^2 rc^2}
//               T: sqrt(28 xi^4 rc^3/(9 pi L)) e^{-xi^2 rc^2}
//               W: sqrt(2/(3 pi L rc)) e^{-xi^2 rc^2}
//   Fourier     S: R k^3 e^{-k^2/4xi^2} / (2 pi^1.5 xi^2)
//               T: sqrt(7/6) R k^4 e^{-k^2/4xi^2} / (2 pi^1.5 xi^2)
//               W: sqrt(2 xi^2/(3 pi^2 L k)) e^{-k^2/4xi^2}
// with k = k_inf = pi/h and R = sqrt(6) L~.  Each part is held to tol/3; r_c
// and k_inf are found by bisection, M = ceil(L k_inf / pi).  The support P is
// the smallest even number with exp(-c^2 pi P/2) <= tol/20 (Gaussian
// truncation, Alg. 1 step 4) and xi P h >= sqrt(ln(1/tol) + 4) (the extension
// L~ = L + P h must hold the screened kernel, Sec. 5.2).
// ------------------------------------------------------------------------------
// Real-space truncation estimates of Sec. 6 (Table 2), relative form.  The
// stokeslet estimate there is a free-space one; against the direct half-space
// sum the truncation error of the half-space stokeslet grows faster, about
// like 0.5 xi r_c (the derivative terms of the image system), and more again
// once r_c approaches L.  The factor max(1, 0.5 xi r_c) (1 + 6 (r_c/L)^3) was
// fitted to the direct sum (N = 200 ... 30000, uniform and near-wall, tol
// 1e-5 ... 1e-12), after which the real-space error stays within the share of
// tol the plan gives it.  The stresslet and rotlet estimates already held.
static double est_real(int mask, double xi, double rc, double L) {
  double e = std::exp(-xi * xi * rc * rc), m = 0.0;
  if (mask & HSE_STOKESLET) {
    const double a = rc / L;
    const double wall = free_space(mask) ? 1.0 : std::fmax(1.0, 0.5 * xi * rc) * (1.0 + 6.0 * a * a * a);
    m = std::fmax(m, std::sqrt(rc / (kPi * L)) * wall);
  }
  if (mask & HSE_STRESSLET) m = std::fmax(m, std::sqrt(28.0 * std::pow(xi, 4) * std::pow(rc, 3) / (9.0 * kPi * L)));
  if (mask & HSE_ROTLET) m = std::fmax(m, std::sqrt(2.0 / (3.0 * kPi * L * rc)));
  return m * e;
}

static double est_fourier(int mask, double xi, double k, double L, double R) {
  double e = std::exp(-k * k / (4.0 * xi * xi)), m = 0.0, d = 2.0 * std::pow(kPi, 1.5) * xi * xi;
  if (mask & HSE_STOKESLET) m = std::fmax(m, R * k * k * k / d);
  if (mask & HSE_STRESSLET) m = std::fmax(m, std::sqrt(7.0 / 6.0) * R * k * k * k * k / d);
  if (mask & HSE_ROTLET) m = std::fmax(m, std::sqrt(2.0 * xi * xi / (3.0 * kPi * kPi * L * k)));
  return m * e;
}

// smallest x in [lo, hi] with f(x) <= target, f decreasing there
template <typename F>
static double bisect_down(F f, double lo, double hi, double target) {
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (f(mid) <= target) hi = mid; else lo = mid;
  }
  return hi;
}

// Smallest m >= n whose padded FFT lengths 2m, 4m factor as 2^a times an odd
// part in {1, 3, 5, 9, 15, 25, 27, 45, 75, 81} (measured fast in cuFFT; factors
// 7 and larger primes were markedly slower for these double transforms).
static int fft_friendly(int n) {
  static const int odd[] = {1, 3, 5, 9, 15, 25, 27, 45, 75, 81};
  int best = 1 << 30;
  for (int o : odd)
    for (long long m = o; m < best; m *= 2)
      if (m >= n && m % 4 == 0 && m < best) best = (int)m;
  return best;
}

int fft_friendly_size(int n) { return fft_friendly(n); }

static hse_status choose_params(hse_plan p, double xi, double rc, int P, double tol) {
  hse_params& q = p->prm;
  const int mask = q.kernel_mask;
  const double L = q.L;
  if (xi <= 0.0) {
    if (tol <= 0.0 || rc <= 0.0) return set_err(p, HSE_ERR_INVALID, "xi <= 0 needs tol > 0 and rc > 0");
    double t = bisect_down([&](double x) { return est_real(mask, x, rc, L); }, 0.1 / rc, 20.0 / rc, tol / 3.0);
    xi = t;
  }
  if (rc <= 0.0) {
    if (tol <= 0.0) return set_err(p, HSE_ERR_INVALID, "rc <= 0 needs tol > 0");
    rc = bisect_down([&](double r) { return est_real(mask, xi, r, L); }, 1.0 / xi, 12.0 / xi, tol / 3.0);
  }
  q.xi = xi;
  q.rc = rc;
  // FP64 path: pairs with xi rho above the split use FP32.  The FP32 error of a
  // pair is ~ kappa eps32 |K_R(rho)| |c|; summed over the shell [rc64, rc) it
  // behaves like kappa eps32 times the truncation estimate evaluated at rc64
  // (the same sum, started at rc64), so rc64 is where that estimate reaches
  // kShellShare / (kappa eps32) times its value at rc (eps32 = 2^-24): the
  // shell gets half the error share of the real-space truncation estimate
  // (itself at most tol/3).  kappa = 4: the shell carries the Gaussian's
  // exponent in double-float and compensates its sums, ~1e-7 per term;
  // measured against all-FP64 pairs on the N = 1M near-wall S+W workload
  // (xi = 87, r_c = 0.0552) the shell adds 2.4e-12 at rc64 = 0.032 and
  // 1.5e-11 at 0.028, and the plain FP32 form 8x more.
  constexpr double kShellShare = 0.5, kShellKappa = 4.0;
  q.rc64 = 0.0;
  if (q.precision == HSE_FP64) {
    const double target = est_real(mask, xi, rc, L) * (kShellShare / (kShellKappa * std::ldexp(1.0, -24)));
    const double lo = 1.5 / xi;  // never FP32 for xi rho < 1.5
    if (lo >= rc) q.rc64 = rc;
    else if (est_real(mask, xi, lo, L) <= target) q.rc64 = lo;
    else q.rc64 = bisect_down([&](double r) { return est_real(mask, xi, r, L); }, lo, rc, target);
  }
  int M = 0;
  if (tol > 0.0) {
    double R = std::sqrt(6.0) * 1.2 * L;  // L~ <= 1.2 L for the supports used here
    double k = bisect_down([&](double kk) { return est_fourier(mask, xi, kk, L, R); }, 2.0 * xi, 30.0 * xi,
                           tol / 3.0);
    M = (int)std::ceil(L * k / kPi);
    if (M < 4) M = 4;
  }
  if (P <= 0) {
    if (tol <= 0.0) return set_err(p, HSE_ERR_INVALID, "P <= 0 needs tol > 0");
    double p1 = 2.0 * std::log(20.0 / tol) / (kWindowC * kWindowC * kPi);
    P = (int)std::ceil(p1);
    if (P % 2) ++P;
    if (M > 0) {
      // grow P until the extension condition holds on the FFT-friendly grid
      const double need = std::sqrt(std::log(1.0 / tol) + 4.0);
      for (; P <= kMaxP; P += 2) {
        int Mf = fft_friendly(M + P) - P;
        if (xi * P * (L / Mf) >= need) break;
      }
    }
  }
  if (P % 2) ++P;
  if (P < 4 || P > kMaxP) return set_err(p, HSE_ERR_INVALID, "P = %d outside [4, %d]", P, kMaxP);
  if (M > 0) M = fft_friendly(M + P) - P;  // grow M so that Mt = M + P has a fast FFT size
  q.P = P;
  q.M = M;
  return HSE_OK;
}

// Device bytes a plan with these settings will hold (grids, tables, an FFT
// work area of one buffer), without creating it.  Host-only.
hse_status plan_estimate(int mask, const double box[3], double xi, double tol, int precision, size_t* bytes,
                         int* M_out, int* P_out, int df64_fourier) {
  hse_plan_s tmp;
  hse_params& q = tmp.prm;
  q.kernel_mask = mask;
  q.precision = precision;
  for (int d = 0; d < 3; ++d) q.box[d] = box[d];
  q.L = std::fmax(box[0], std::fmax(box[1], box[2]));
  HSE_TRY(choose_params(&tmp, xi, 0.0, 0, tol));
  int Mt = q.M + q.P;
  size_t esz = precision == HSE_MIXED && !df64_fourier ? 4 : 8;
  size_t buf = (size_t)(2 * Mt) * (2 * Mt) * (2 * (2 * Mt + 1)) * esz;
  size_t tab = (size_t)(Mt + 1) * (Mt + 1) * (2 * Mt + 1) * esz;
  int ncomp = product_components(mask).n;
  *bytes = buf * (ncomp + 1) + 2 * tab;
  if (M_out) *M_out = q.M;
  if (P_out) *P_out = q.P;
  return HSE_OK;
}

}  // namespace hse

using namespace hse;

extern "C" hse_status hse_plan_create(int kernel_mask, const double box[3], double xi, double rc, int P, double tol,
                                      int precision, hse_plan* out) {
  if (!out) return set_err(nullptr, HSE_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!valid_mask(kernel_mask)) return set_err(nullptr, HSE_ERR_INVALID, "kernel_mask %d", kernel_mask);
  if (!box || !(box[0] > 0) || !(box[1] > 0) || !(box[2] > 0) || !std::isfinite(box[0]) || !std::isfinite(box[1]) ||
      !std::isfinite(box[2]))
    return set_err(nullptr, HSE_ERR_INVALID, "box must be finite and positive");
  if (precision != HSE_FP64 && precision != HSE_MIXED)
    return set_err(nullptr, HSE_ERR_INVALID, "precision %d", precision);
  if (precision == HSE_MIXED && tol > 0.0 && tol < 1e-6)
    return set_err(nullptr, HSE_ERR_INVALID, "HSE_MIXED needs tol >= 1e-6 (FP32 arithmetic)");
  if (!(tol < 1.0)) return set_err(nullptr, HSE_ERR_INVALID, "tol must be < 1");
  hse_plan p = new (std::nothrow) hse_plan_s();
  if (!p) return set_err(nullptr, HSE_ERR_OOM, "host allocation");
  hse_params& q = p->prm;
  q.kernel_mask = kernel_mask;
  q.precision = precision;
  q.spread_tile[0] = 2;
  q.spread_tile[1] = 4;
  q.spread_tile[2] = 4;
  p->tol = tol;
  for (int d = 0; d < 3; ++d) q.box[d] = box[d];
  q.L = std::fmax(box[0], std::fmax(box[1], box[2]));
  hse_status st = choose_params(p, xi, rc, P, tol);
  if (st == HSE_OK) {
    for (int d = 0; d < 3; ++d) {
      // cells of side >= r_c / kCellReach: the neighbour scan covers
      // (2 kCellReach + 1)^3 cells, 15.6 r_c^3 of candidates for a reach of 2
      // against 27 r_c^3 with cells of side r_c
      double nc = std::floor(box[d] * kCellReach / q.rc);
      if (nc < 1) nc = 1;
      if (nc > 1024) nc = 1024;
      q.ncell[d] = (int)nc;
      p->inv_cell[d] = (double)q.ncell[d] / box[d];
    }
    p->n_rows = 0;
    if (kernel_mask & HSE_STOKESLET) { p->row_S = p->n_rows; p->n_rows += 3; }
    if (kernel_mask & HSE_STRESSLET) { p->row_T = p->n_rows; p->n_rows += 6; }
    if (kernel_mask & HSE_ROTLET) { p->row_W = p->n_rows; p->n_rows += 3; }
    if (q.M > 0) st = build_grids(p);
  }
  if (st != HSE_OK) {
    g_create_error = p->err;
    free_grids(p);
    delete p;
    return st;
  }
  *out = p;
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_grid(hse_plan p, int M) {
  if (!p) return HSE_ERR_INVALID;
  if (M < 4) return set_err(p, HSE_ERR_INVALID, "M = %d < 4", M);
  p->prm.M = M;
  return build_grids(p);
}

extern "C" hse_status hse_plan_set_rc64(hse_plan p, double rc64) {
  if (!p) return HSE_ERR_INVALID;
  if (!(rc64 >= 0.0) || p->prm.precision != HSE_FP64)
    return set_err(p, HSE_ERR_INVALID, "rc64 needs an HSE_FP64 plan and rc64 >= 0");
  p->prm.rc64 = rc64;
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_rcmid(hse_plan p, double rcmid) {
  if (!p) return HSE_ERR_INVALID;
  if (!(rcmid >= 0.0) || p->prm.precision != HSE_FP64)
    return set_err(p, HSE_ERR_INVALID, "rcmid needs an HSE_FP64 plan and rcmid >= 0");
  p->prm.rcmid = rcmid;
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_fft(hse_plan p, int mode) {
  if (!p) return HSE_ERR_INVALID;
  if (mode != HSE_FFT_AUTO && mode != HSE_FFT_CUFFT && mode != HSE_FFT_DF64)
    return set_err(p, HSE_ERR_INVALID, "fft mode %d", mode);
  const int old_mode = p->fft_mode;
  p->fft_mode = mode;
  if (!p->grid_ready) return HSE_OK;
  if (p->prm.precision == HSE_MIXED) {
    // the grid element changes between FP32 (cuFFT single) and double-float:
    // rebuild grids and tables
    const int f = resolve_fft(p);
    if (f < 0) {
      p->fft_mode = old_mode;
      return set_err(p, HSE_ERR_UNSUPPORTED, "df64 FFT: grid %d x %d x %d", p->g.Nx, p->g.Ny, p->g.Nz);
    }
    if (f != p->prm.fft) return build_grids(p);
    return HSE_OK;
  }
  const int f = resolve_fft(p);
  if (f < 0) {
    p->fft_mode = HSE_FFT_AUTO;
    return set_err(p, HSE_ERR_UNSUPPORTED, "df64 FFT: grid %d x %d x %d", p->g.Nx, p->g.Ny, p->g.Nz);
  }
  const size_t work_before = p->fft_work_bytes;
  if (f == HSE_FFT_DF64) HSE_TRY(fft64_prepare(p));
  else HSE_TRY(build_cufft(p));
  p->prm.fft = f;
  p->prm.grid_bytes += p->fft_work_bytes - work_before;  // a cuFFT work area made now
  if (f == HSE_FFT_DF64) HSE_TRY(prepare_df_tables(p));
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_spread_tile(hse_plan p, int wx, int wy, int wz) {
  if (!p) return HSE_ERR_INVALID;
  auto pow2 = [](int v) { return v >= 1 && v <= 16 && (v & (v - 1)) == 0; };
  if (!pow2(wx) || !pow2(wy) || !pow2(wz) || wx * wy * wz != 32)
    return set_err(p, HSE_ERR_INVALID, "spread tile %d x %d x %d (powers of two up to 16, product 32)", wx, wy, wz);
  p->prm.spread_tile[0] = wx;
  p->prm.spread_tile[1] = wy;
  p->prm.spread_tile[2] = wz;
  return HSE_OK;
}

extern "C" hse_status hse_plan_get_params(hse_plan p, hse_params* out) {
  if (!p || !out) return HSE_ERR_INVALID;
  *out = p->prm;
  return HSE_OK;
}

extern "C" hse_status hse_plan_destroy(hse_plan p) {
  if (!p) return HSE_ERR_INVALID;
  cudaDeviceSynchronize();
  if (p->timing) {
    for (int i = 0; i <= HSE_N_STAGES; ++i) cudaEventDestroy(p->ev[i]);
    cudaEventDestroy(p->ev_real_end);
  }
  if (p->s_real) {
    cudaStreamDestroy(p->s_real);
    cudaStreamDestroy(p->s_four);
    cudaEventDestroy(p->ev_fork);
    cudaEventDestroy(p->ev_real);
    cudaEventDestroy(p->ev_four);
  }
  free_grids(p);
  free_workspace(p);
  delete p;
  return HSE_OK;
}

extern "C" const char* hse_status_string(hse_status s) {
  switch (s) {
    case HSE_OK: return "HSE_OK";
    case HSE_ERR_INVALID: return "HSE_ERR_INVALID";
    case HSE_ERR_OOM: return "HSE_ERR_OOM";
    case HSE_ERR_CUDA: return "HSE_ERR_CUDA";
    case HSE_ERR_CUFFT: return "HSE_ERR_CUFFT";
    case HSE_ERR_TIMEOUT: return "HSE_ERR_TIMEOUT";
    case HSE_ERR_UNSUPPORTED: return "HSE_ERR_UNSUPPORTED";
  }
  return "unknown status";
}

extern "C" const char* hse_last_error(hse_plan p) {
  return p ? p->err.c_str() : g_create_error.c_str();
}
