// hse_fourier.cu -- Fourier-space part of the half-space Spectral Ewald method
// (Alg. 1, steps 5-10; Sec. 5.2).  Grid element type T: double-float (df) for
// FP64 plans on the transform path of hse_fft64.cu, double for FP64 plans on
// cuFFT, float for mixed-precision plans.
//
//  prep    per source: support start (ix0, iy0, iz0), the 1-D Gaussian factors
//          of the window (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 |x - z|^2 / eta)
//          and their derivatives, folded with the strengths into the
//          per-source arrays of every spread component;
//  spread  owner-computes tiles: each thread owns one grid point and sums the
//          windows of the cell-listed sources whose P^3 support covers it.
//          Everything is accumulated at the SOURCE position: an image's window
//          is the mirror (k -> 2 Mt - k) of its source's window, so
//  mirror  forms C1 = A(k) +- A(2Mt - k) and the image-only correction grid
//          D(k) = A(2Mt - k) in place.  The wall corrections of every kernel
//          are one harmonic potential whose source D = Cs W + Cv.grad W -
//          Ct:grad grad W is spread through window derivatives (ik C^ and
//          -k k C^ are the transforms of grad C and grad grad C);
//  FFT     zero-padded by 2 in every direction: the pruned double-float
//          transforms of hse_fft64.cu, or cuFFT D2Z / R2C, in place;
//  scale   per wave vector k: T1^ = K^_F C1^ + e3 phi^ and phi^ = E H^R D^
//          (the merged harmonic corrections), stokeslet A^S = -(k^2 I - k k),
//          stresslet A^T, rotlet A^W = -2 i eps k, tables including
//          exp(-(1-eta)k^2/4xi^2), written in place;
//  IFFT    of the 4 fields T1 (3) and phi (hse_fft64.cu, or cuFFT Z2D / C2R);
//  gather  u_F(x) = h^3 sum over the P^3 support of W(x - x_j) T1(x_j)
//          - x3 h^3 sum of grad W(x - x_j) phi(x_j)  (grad phi through the
//          window's gradient, so no T2 = i k phi^ grids are transformed).
#include <algorithm>
#include <type_traits>

#include "hse_df64.cuh"
#include "hse_internal.cuh"

namespace hse {

// ----------------------------------------------------------------------- prep
template <typename T>
struct PrepArgs {
  int64_t n;
  const double* spos;
  const double* sstr;
  int rowS, rowT, rowW, mask;
  int paper;  // component set: 0 product (C1 + one correction grid D), 1 paper (C1/C2/C3 per kernel)
  int nfac;   // window factor sets per particle: 1 (W), 2 (W, W'), 3 (W, W', W'')
  int nc1;    // product set: number of C1 components
  int P, Mt;
  double h, ox, oz, alpha, pre;
  double c2;      // exp(-2 alpha h^2): step of the window recurrence
  int stride;
  RecLayout lay;  // record layout (rec_layout(nfac, components, P))
  T* prep;
  float* prep32;  // FP64 plans: the same record in FP32 (null otherwise)
  int4* supp;
};

template <typename T>
__device__ __forceinline__ void prep_one(const PrepArgs<T>& a, int64_t i) {
  {
    const int64_t n = a.n;
    double x = a.spos[i], y = a.spos[n + i], z = a.spos[2 * n + i];
    int ix0 = support_start(x, a.ox, a.h, a.P, a.Mt);
    int iy0 = support_start(y, a.ox, a.h, a.P, a.Mt);
    int iz0 = support_start(z, a.oz, a.h, a.P, 2 * a.Mt);
    a.supp[i] = make_int4(ix0, iy0, iz0, 0);
    T* o = a.prep + i * (int64_t)a.stride;
    const int P = a.P;
    // window factors wx (prefactor folded in), wy, wz; for the correction grid
    // also wy', wz' (and wy'', wz''), derivatives with respect to the grid
    // point: W' = -2 alpha d W, W'' = (4 alpha^2 d^2 - 2 alpha) W.  The x
    // derivatives go into the combined arrays XX below.
    // The factors along an axis come from the fast Gaussian gridding
    // recurrence (Greengard & Lee, SIAM Review 46, 2004): with d_t = d_0 + t h,
    // w_{t+1} = w_t r_t, r_t = exp(-alpha (2 d_t h + h^2)), r_{t+1} = r_t
    // exp(-2 alpha h^2): two exponentials per axis instead of P (relative
    // rounding <~ 2 P eps64 after P steps).
    const RecLayout& L = a.lay;
    {  // zero entries around the x, y and z blocks
      const int pad[3] = {L.px, L.py, L.pz}, base[3] = {L.x0, L.y0, L.z0}, ke[3] = {L.kx, L.ky, L.ky};
      for (int k = 0; k < 3; ++k)
        for (int t = 0; t < pad[k]; ++t)
          for (int m = 0; m < ke[k]; ++m) {
            o[base[k] + t * ke[k] + m] = (T)0;
            o[base[k] + (P + pad[k] + t) * ke[k] + m] = (T)0;
          }
    }
    double wr[3], rr[3];
    {
      const double d0[3] = {a.ox + ix0 * a.h - x, a.ox + iy0 * a.h - y, a.oz + iz0 * a.h - z};
      for (int k = 0; k < 3; ++k) {
        wr[k] = exp(-a.alpha * d0[k] * d0[k]) * (k == 0 ? a.pre : 1.0);
        rr[k] = exp(-a.alpha * (2.0 * d0[k] * a.h + a.h * a.h));
      }
    }
    for (int t = 0; t < P; ++t) {
      double d[3] = {a.ox + (ix0 + t) * a.h - x, a.ox + (iy0 + t) * a.h - y, a.oz + (iz0 + t) * a.h - z};
      for (int k = 0; k < 3; ++k) {
        const double wv = wr[k];
        wr[k] *= rr[k];
        rr[k] *= a.c2;
        T* e = k == 0 ? o + L.x0 + (t + L.px) * L.kx : (k == 1 ? o + L.y0 + (t + L.py) * L.ky : o + L.z0 + (t + L.pz) * L.ky);
        const int ke = k == 0 ? L.kx : L.ky;
        for (int m = 1; m < ke; ++m) e[m] = (T)0;  // padding (and the x block's XX, written below)
        e[0] = (T)wv;
        if (k > 0 && a.nfac > 1) e[1] = (T)(-2.0 * a.alpha * d[k] * wv);
        if (k > 0 && a.nfac > 2) e[2] = (T)((4.0 * a.alpha * a.alpha * d[k] * d[k] - 2.0 * a.alpha) * wv);
      }
    }
    const int nxx = a.nfac == 1 ? 0 : (a.nfac == 2 ? 3 : 6);  // combined x arrays
    T* c = o + L.c0;
    c[L.stride - L.c0 - 1] = (T)0;  // padding of an odd component count
    int k = 0;
    double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, q[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
    if (a.mask & HSE_STOKESLET) for (int d = 0; d < 3; ++d) f[d] = a.sstr[(a.rowS + d) * n + i];
    if (a.mask & HSE_STRESSLET)
      for (int d = 0; d < 3; ++d) { g[d] = a.sstr[(a.rowT + d) * n + i]; q[d] = a.sstr[(a.rowT + 3 + d) * n + i]; }
    if (a.mask & HSE_ROTLET) for (int d = 0; d < 3; ++d) tau[d] = a.sstr[(a.rowW + d) * n + i];
    const double hz = z;  // source height y3
    double gI[3] = {g[0], g[1], -g[2]}, qI[3] = {q[0], q[1], -q[2]};
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    double sgq[6], sgqI[6];
    for (int m = 0; m < 6; ++m) {
      sgq[m] = 0.5 * (g[ia[m]] * q[ib[m]] + g[ib[m]] * q[ia[m]]);
      sgqI[m] = 0.5 * (gI[ia[m]] * qI[ib[m]] + gI[ib[m]] * qI[ia[m]]);
    }
    double gdq = g[0] * q[0] + g[1] * q[1] + g[2] * q[2];
    if (a.mask & HSE_FREE_SPACE) {  // Sec. 2: C1 only (same in both component sets)
      if (a.mask & HSE_STOKESLET) for (int d = 0; d < 3; ++d) c[k++] = (T)f[d];
      if (a.mask & HSE_STRESSLET) for (int m = 0; m < 6; ++m) c[k++] = (T)sgq[m];
      if (a.mask & HSE_ROTLET) for (int d = 0; d < 3; ++d) c[k++] = (T)tau[d];
    } else if (!a.paper) {
      // C1, and the correction grid
      //   D = Cs W + Cv . grad W - Ct : grad grad W   (at the image; phi^ = E H^R D^)
      // with Cs = -2 f3 (S); Cv = -2 y3 f^I (S) + 4 g.q e3 (T) + 4 (-tau2, tau1, 0) (W);
      // Ct = 4 y3 sym(g^I q^I) (T).  D is accumulated at the source and mirrored
      // in z (image-only component), so every z-odd term changes sign here.
      if (a.mask & HSE_STOKESLET) for (int d = 0; d < 3; ++d) c[k++] = (T)f[d];
      if (a.mask & HSE_STRESSLET) for (int m = 0; m < 6; ++m) c[k++] = (T)sgq[m];
      if (a.mask & HSE_ROTLET) for (int d = 0; d < 3; ++d) c[k++] = (T)tau[d];
      double cs = 0.0, cv[3] = {0, 0, 0}, ct[6] = {0, 0, 0, 0, 0, 0};
      if (a.mask & HSE_STOKESLET) {
        cs += -2.0 * f[2];
        cv[0] += -2.0 * hz * f[0]; cv[1] += -2.0 * hz * f[1]; cv[2] += 2.0 * hz * f[2];
      }
      if (a.mask & HSE_STRESSLET) {
        cv[2] += 4.0 * gdq;
        for (int m = 0; m < 6; ++m) ct[m] = 4.0 * hz * sgqI[m];  // xx xy xz yy yz zz
      }
      if (a.mask & HSE_ROTLET) { cv[0] += -4.0 * tau[1]; cv[1] += 4.0 * tau[0]; }
      // coefficients of W, dx, dy, dz, dxx, dyy, dzz, dxdy, dxdz, dydz (z-odd
      // terms flipped), folded with the x factors into
      //   D = XX00 wy wz + XX10 wy' wz + XX01 wy wz' + XX20 wy'' wz + XX02 wy wz'' + XX11 wy' wz'
      const double q[10] = {cs, cv[0], cv[1], -cv[2], -ct[0], -ct[3], -ct[5], -2.0 * ct[1], 2.0 * ct[2], 2.0 * ct[4]};
      const double dx0 = a.ox + ix0 * a.h - x;
      double wxr = a.pre * exp(-a.alpha * dx0 * dx0), rxr = exp(-a.alpha * (2.0 * dx0 * a.h + a.h * a.h));
      for (int t = 0; t < P; ++t) {
        T* xx = o + L.x0 + (t + L.px) * L.kx + 1;  // XX_m of entry t
        const double dx = a.ox + (ix0 + t) * a.h - x;
        const double wx = wxr;  // the window along x (recurrence as above)
        wxr *= rxr;
        rxr *= a.c2;
        const double dwx = -2.0 * a.alpha * dx * wx;
        const double ddwx = (4.0 * a.alpha * a.alpha * dx * dx - 2.0 * a.alpha) * wx;
        xx[0] = (T)(q[0] * wx + q[1] * dwx + q[4] * ddwx);
        xx[1] = (T)(q[2] * wx + q[7] * dwx);
        xx[2] = (T)(q[3] * wx + q[8] * dwx);
        if (nxx == 6) {
          xx[3] = (T)(q[5] * wx);
          xx[4] = (T)(q[6] * wx);
          xx[5] = (T)(q[9] * wx);
        }
      }
    } else {
      if (a.mask & HSE_STOKESLET) {
        for (int d = 0; d < 3; ++d) c[k++] = (T)f[d];
        c[k++] = (T)f[2];
        c[k++] = (T)(hz * f[0]); c[k++] = (T)(hz * f[1]); c[k++] = (T)(-hz * f[2]);
      }
      if (a.mask & HSE_STRESSLET) {
        for (int m = 0; m < 6; ++m) c[k++] = (T)sgq[m];
        c[k++] = (T)gdq;
        for (int m = 0; m < 6; ++m) c[k++] = (T)(hz * sgqI[m]);
      }
      if (a.mask & HSE_ROTLET) {
        for (int d = 0; d < 3; ++d) c[k++] = (T)tau[d];
        c[k++] = (T)(-tau[1]); c[k++] = (T)tau[0];
      }
    }
  }
}

template <typename T>
__global__ void k_prep(PrepArgs<T> a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    prep_one(a, i);
    if (a.prep32) {  // FP32 copy of the record for the spread's small-weight part
      const T* o = a.prep + i * (int64_t)a.stride;
      float* o32 = a.prep32 + i * (int64_t)a.stride;
      for (int t = 0; t < a.stride; ++t) o32[t] = head32(o[t]);
    }
  }
}

// --------------------------------------------------------------------- spread
template <typename T>
struct SpreadArgs {
  const int4* supp;
  const T* prep;
  // FP64 spread: (warp, particle) pairs whose weights on the warp's points are
  // all below e^{-lnthr} of the window's peak take the FP32 record
  const float* prep32;   // null: FP64 throughout
  const float* spos32;   // sorted positions (FP32 heads)
  float ah2, lnthr;      // alpha h^2 (window exponent per squared grid step), ln(1/threshold)
  const int32_t* cstart;
  int stride, P, Mt, z0, nz_tiles;
  int y0, z0r, c0;       // offsets of the y and z blocks and of the components in a record
  int pad[3];            // zero entries before each block (warp sub-tile - 1)
  int zlo;               // lowest z index any source support reaches (tiles below only write zeros)
  double h, ox, oz;
  double inv_cell[3];
  int ncell[3];
  T* out;                // component c, point (i,j,k) at out + c*cs + i*xs + j*pitch + k
  int64_t cs, xs, pitch;
  int64_t is;            // batched instances: instance stride of out (blockIdx.z = inst * nz_tiles + tile)
  int ncells_inst;       // cells per instance in the cell list
  int64_t n_src;         // sorted particles (rows of spos32)
  int wl[3];             // log2 of the warp sub-tile along x, y, z (hse_params.spread_tile)
};


// two adjacent record elements with one load (8-byte elements: 16 bytes,
// 4-byte elements: 8 bytes; record entries are aligned to two elements)
__device__ __forceinline__ void ld2(const df* p, df& a, df& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = df(v.x, v.y);
  b = df(v.z, v.w);
}
__device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  a = v.x;
  b = v.y;
}
template <typename T, int N>
__device__ __forceinline__ void ldv(const T* p, T* out) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) ld2(p + 2 * i, out[2 * i], out[2 * i + 1]);
}

// NC plain components (C1, or the paper set), plus with DK != 0 the correction
// grid D from derivative windows: DK bits 1 (W term), 2 (first derivatives),
// 4 (second derivatives).
//
// Each warp owns a wx x wy x wz sub-tile (one grid point per lane; 2 x 4 x 4
// unless the plan sets another shape) of the block's 2wx x 2wy x 2wz tile (8
// warps, 2 per dimension) and works alone, with no block-wide barrier: it scans
// the cell-list rows whose sources can reach its sub-tile, 32 candidates at a
// time (one per lane: does the support cover the sub-tile, and is every weight
// on it below the FP32 threshold), compacts the hits into a warp-private list
// (FP32 small-weight hits from the front, the others from the back, each in
// source order) and accumulates them into separate FP32 and full-precision
// sums.  Per point and class the sources are added in cell-row order and,
// within a row, in sorted order, so the result is deterministic.
// blocks per SM the spread is compiled for, while the accumulators fit without
// spilling (else 2): FP32 4 (64 registers); 8-byte elements 3 (80 registers:
// measured on the N = 1M near-wall S+W workload, 41.3 ms against 44.2 ms at 4
// blocks, where the unrolled loop spills)
template <typename T, int NC, int DK>
constexpr int spread_min_blocks() {
  return NC + (DK != 0) <= 7 && DK != 7 && DK != 6 ? (sizeof(T) == 4 ? 4 : 3) : 2;
}

template <typename T, int NC, int DK>
__global__ void __launch_bounds__(256, spread_min_blocks<T, NC, DK>()) k_spread(SpreadArgs<T> a) {
  // per warp: the hits of the current 32 candidates, with their support
  // starts (w: source index, bit 31 set when the FP32 small-weight record applies)
  __shared__ int4 wlist[8][32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int inst = blockIdx.z / a.nz_tiles, ztile = blockIdx.z - inst * a.nz_tiles;
  const int cbase = inst * a.ncells_inst;
  const int lx = a.wl[0], ly = a.wl[1], lz = a.wl[2];
  const int wx = 1 << lx, wy = 1 << ly, wz = 1 << lz;  // warp sub-tile
  const int bx0 = (2 * wx) * blockIdx.x, by0 = (2 * wy) * blockIdx.y, bz0 = a.z0 + (2 * wz) * ztile;
  const int sx = bx0 + wx * (w & 1), sy = by0 + wy * ((w >> 1) & 1), sz = bz0 + wz * (w >> 2);
  const int px = sx + (lane & (wx - 1)), py = sy + ((lane >> lx) & (wy - 1)), pz = sz + (lane >> (lx + ly));
  const int P = a.P;
  // per-particle record (rec_layout): x entries {wx, XX_0..}, y entries
  // {wy, wy', wy''}, z entries {wz, wz', wz''}, then the NC components
  constexpr int NF = DK == 0 ? 1 : ((DK & 4) ? 3 : 2);
  constexpr int KX = rec_kx(NF), KY = rec_ky(NF);
  T acc[NC];
  T accD = (T)0;
  float acc32[NC];
  float accD32 = 0.f;
#pragma unroll
  for (int c = 0; c < NC; ++c) { acc[c] = (T)0; acc32[c] = 0.f; }
  const bool split = sizeof(T) == 8 && a.prep32 != nullptr;
  const float inv_h = (float)(1.0 / a.h), oxf = (float)a.ox, ozf = (float)a.oz;
  const float fsx = (float)sx, fsy = (float)sy, fsz = (float)sz;  // sub-tile origin
  // positions whose support can reach the sub-tile (one grid step of slack for clamping)
  auto cell_range = [&](int lo_idx, int hi_idx, double o, int d, int& c0, int& c1) {
    double lo = o + (lo_idx - P / 2 - 1) * a.h, hi = o + (hi_idx + P / 2 + 1) * a.h;
    c0 = cell_coord(lo, a.inv_cell[d], a.ncell[d]);
    c1 = cell_coord(hi, a.inv_cell[d], a.ncell[d]);
  };
  int cx0, cx1, cy0, cy1, cz0, cz1;
  cell_range(sx, sx + wx - 1, a.ox, 0, cx0, cx1);
  cell_range(sy, sy + wy - 1, a.ox, 1, cy0, cy1);
  cell_range(sz, sz + wz - 1, a.oz, 2, cz0, cz1);
  const int nx = a.ncell[0], ny = a.ncell[1];
  const unsigned below = (1u << lane) - 1;
  int4* list = wlist[w];
  if (sz + wz <= a.zlo) cz1 = cz0 - 1;  // no support reaches the sub-tile: zeros only
  for (int cz = cz0; cz <= cz1; ++cz)
    for (int cy = cy0; cy <= cy1; ++cy) {
      const int c0 = cbase + (cz * ny + cy) * nx + cx0;
      const int s0 = a.cstart[c0], s1 = a.cstart[c0 + (cx1 - cx0) + 1];
      for (int base = s0; base < s1; base += 32) {
        // lane = candidate: does its support cover the sub-tile, and if so is
        // every weight on it below the FP32 threshold (distance from the
        // source to the sub-tile, less half a step for the FP32 position: if
        // even the nearest point has weight below the threshold, so do all)
        const int j = base + lane;
        bool hit = false, small = false;
        int4 sp = make_int4(0, 0, 0, 0);
        if (j < s1) {
          sp = a.supp[j];
          hit = sp.x <= sx + wx - 1 && sp.x + P - 1 >= sx && sp.y <= sy + wy - 1 && sp.y + P - 1 >= sy &&
                sp.z <= sz + wz - 1 && sp.z + P - 1 >= sz;
          if (hit && split) {
            const int64_t n = a.n_src;
            const float gx = (a.spos32[j] - oxf) * inv_h, gy = (a.spos32[n + j] - oxf) * inv_h;
            const float gz = (a.spos32[2 * n + j] - ozf) * inv_h;
            const float ex = fmaxf(0.f, fmaxf(fsx - gx, gx - (fsx + (float)(wx - 1))) - 0.5f);
            const float ey = fmaxf(0.f, fmaxf(fsy - gy, gy - (fsy + (float)(wy - 1))) - 0.5f);
            const float ez = fmaxf(0.f, fmaxf(fsz - gz, gz - (fsz + (float)(wz - 1))) - 0.5f);
            small = a.ah2 * (ex * ex + ey * ey + ez * ez) >= a.lnthr;
          }
        }
        // FP32 small-weight hits fill the list from the front, the others from
        // the back, each class in source order (fixed per point: deterministic
        // sums)
        const unsigned ms = __ballot_sync(0xffffffffu, hit && small);
        const unsigned mb = __ballot_sync(0xffffffffu, hit && !small);
        if (hit) list[small ? __popc(ms & below) : 31 - __popc(mb & below)] = make_int4(sp.x, sp.y, sp.z, j);
        __syncwarp();
        const int ns = __popc(ms), nb = __popc(mb);
        // Branch-free bodies (a lane outside the source's support reads the
        // record's zero pads), unrolled so that the next source's record
        // loads are in flight while this one accumulates.
#pragma unroll 2
        for (int e = 0; e < ns; ++e) {
          const int4 s = list[e];
          // entry of the lane's grid point in the source's padded blocks (the
          // pads hold zeros for points outside the support)
          const float* o = a.prep32 + (int64_t)s.w * a.stride;
          float xv[KX], yv[KY], zv[KY];
          ldv<float, KX>(o + (px - s.x + a.pad[0]) * KX, xv);
          ldv<float, KY>(o + a.y0 + (py - s.y + a.pad[1]) * KY, yv);
          ldv<float, KY>(o + a.z0r + (pz - s.z + a.pad[2]) * KY, zv);
          float cv[(NC + 1) & ~1];
          ldv<float, (NC + 1) & ~1>(o + a.c0, cv);
          const float wyz = yv[0] * zv[0];
          const float wv = xv[0] * wyz;
#pragma unroll
          for (int c = 0; c < NC; ++c) acc32[c] += wv * cv[c];
          if constexpr (DK != 0) {
            accD32 += xv[1] * wyz + xv[2] * (yv[1] * zv[0]) + xv[3] * (yv[0] * zv[1]);
            if constexpr ((DK & 4) != 0)
              accD32 += xv[4] * (yv[2] * zv[0]) + xv[5] * (yv[0] * zv[2]) + xv[6] * (yv[1] * zv[1]);
          }
        }
#pragma unroll 2
        for (int e = 0; e < nb; ++e) {
          const int4 s = list[31 - e];
          const T* o = a.prep + (int64_t)s.w * a.stride;
          T xv[KX], yv[KY], zv[KY];
          ldv<T, KX>(o + (px - s.x + a.pad[0]) * KX, xv);
          ldv<T, KY>(o + a.y0 + (py - s.y + a.pad[1]) * KY, yv);
          ldv<T, KY>(o + a.z0r + (pz - s.z + a.pad[2]) * KY, zv);
          T cv[(NC + 1) & ~1];
          ldv<T, (NC + 1) & ~1>(o + a.c0, cv);
          const T wyz = mulr(yv[0], zv[0]);
          const T wv = mulr(xv[0], wyz);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = mac(acc[c], wv, cv[c]);
          if constexpr (DK != 0) {
            accD = mac(accD, xv[1], wyz);
            accD = mac(accD, xv[2], mulr(yv[1], zv[0]));
            accD = mac(accD, xv[3], mulr(yv[0], zv[1]));
            if constexpr ((DK & 4) != 0) {
              accD = mac(accD, xv[4], mulr(yv[2], zv[0]));
              accD = mac(accD, xv[5], mulr(yv[0], zv[2]));
              accD = mac(accD, xv[6], mulr(yv[1], zv[1]));
            }
          }
        }
        __syncwarp();
      }
    }
  if (px < a.Mt && py < a.Mt && pz >= 0 && pz < 2 * a.Mt) {
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += from32<T>(acc32[c]);
    accD += from32<T>(accD32);
    T* dst = a.out + inst * a.is + px * a.xs + py * a.pitch + pz;
#pragma unroll
    for (int c = 0; c < NC; ++c) dst[c * a.cs] = acc[c];
    if constexpr (DK != 0) dst[NC * a.cs] = accD;
  }
}

template <typename T, int NC, int DK>
static void launch_spread_t(const SpreadArgs<T>& a, dim3 grid, cudaStream_t s) {
  k_spread<T, NC, DK><<<grid, 256, 0, s>>>(a);
}

// nc plain components; dk: derivative kind of the correction grid (0: none)
template <typename T>
static bool launch_spread(int nc, int dk, const SpreadArgs<T>& a, dim3 grid, cudaStream_t s) {
  switch (dk * 64 + nc) {
    // product set: C1 of the mask (+ D)
    case 0 * 64 + 3: launch_spread_t<T, 3, 0>(a, grid, s); return true;
    case 0 * 64 + 6: launch_spread_t<T, 6, 0>(a, grid, s); return true;
    case 0 * 64 + 9: launch_spread_t<T, 9, 0>(a, grid, s); return true;
    case 0 * 64 + 12: launch_spread_t<T, 12, 0>(a, grid, s); return true;
    case 3 * 64 + 3: launch_spread_t<T, 3, 3>(a, grid, s); return true;   // S
    case 6 * 64 + 6: launch_spread_t<T, 6, 6>(a, grid, s); return true;   // T
    case 2 * 64 + 3: launch_spread_t<T, 3, 2>(a, grid, s); return true;   // W
    case 3 * 64 + 6: launch_spread_t<T, 6, 3>(a, grid, s); return true;   // S+W
    case 7 * 64 + 9: launch_spread_t<T, 9, 7>(a, grid, s); return true;   // S+T
    case 6 * 64 + 9: launch_spread_t<T, 9, 6>(a, grid, s); return true;   // T+W
    case 7 * 64 + 12: launch_spread_t<T, 12, 7>(a, grid, s); return true; // S+T+W
    // paper set (hse_spread_grids)
    case 0 * 64 + 5: launch_spread_t<T, 5, 0>(a, grid, s); return true;
    case 0 * 64 + 7: launch_spread_t<T, 7, 0>(a, grid, s); return true;
    case 0 * 64 + 13: launch_spread_t<T, 13, 0>(a, grid, s); return true;
    case 0 * 64 + 18: launch_spread_t<T, 18, 0>(a, grid, s); return true;
    case 0 * 64 + 20: launch_spread_t<T, 20, 0>(a, grid, s); return true;
    case 0 * 64 + 25: launch_spread_t<T, 25, 0>(a, grid, s); return true;
  }
  return false;
}

// --------------------------------------------------------------------- mirror
template <typename T>
struct MirrorArgs {
  T* buf;
  int64_t cs, xs, pitch;
  int Mt, nc;
  int sign[kMaxComp];
  int n_inst;
  int64_t is;  // instance stride
};

template <typename T>
__global__ void k_mirror(MirrorArgs<T> a) {
  const int Mt = a.Mt;
  const int64_t per = (int64_t)Mt * Mt * (Mt + 1);
  const int64_t total = per * a.nc * a.n_inst;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t ci = e / per;
    int c = (int)(ci % a.nc);
    int64_t inst = ci / a.nc;
    int64_t r = e - ci * per;
    int k = (int)(r % (Mt + 1));
    int64_t ij = r / (Mt + 1);
    int j = (int)(ij % Mt), i = (int)(ij / Mt);
    T* col = a.buf + c * a.cs + inst * a.is + i * a.xs + j * a.pitch;
    int kp = 2 * Mt - k;
    T va = col[k];
    T vb = kp < 2 * Mt ? col[kp] : (T)0;
    int s = a.sign[c];
    if (s != 0) {
      col[k] = va + (T)s * vb;
      if (kp < 2 * Mt && kp != k) col[kp] = vb + (T)s * va;
    } else {
      col[k] = vb;
      if (kp < 2 * Mt && kp != k) col[kp] = va;
    }
  }
}

// ---------------------------------------------------------------------- scale
// T: arithmetic of the scaling (double, float, or df for double-float
// spectra); Tab<T>: element type of the kernel tables it reads
template <typename T> struct Cplx;
template <> struct Cplx<double> { typedef double2 type; };
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<df> { typedef cdf type; };
template <typename T> struct Tab { typedef T type; };
template <> struct Tab<df> { typedef df type; };  // float-pair copies of the FP64 tables

template <typename T>
struct ScaleArgs {
  typename Cplx<T>::type* buf;  // complex view of the spectra
  int64_t cstride;              // complex elements per buffer
  int Mt, mask;
  double h;
  const typename Tab<T>::type* tabB;
  const typename Tab<T>::type* tabH;
  // FP32 spectra: FP64 tables on the corner |kx|, |ky|, kz <= lowK (H, then
  // B), whose k-points are scaled in FP64; null otherwise
  const double* tabLow;
  int lowK;
  int iS, iT, iW, iD;  // first component index of each group (C1 of S, T, W; correction grid), -1 if absent
  int n_inst;
  int64_t istride;     // complex elements between instances of one component
  int64_t xstride;     // complex elements between kx planes of one buffer
  int nout;            // 4 (T1, phi) or 3 (free space: T1 only)
};

template <typename C, typename T>
__device__ __forceinline__ C cmk(T x, T y) { C z; z.x = x; z.y = y; return z; }
template <typename C>
__device__ __forceinline__ C cmul_i(C z) { return cmk<C>(-z.y, z.x); }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C, typename T>
__device__ __forceinline__ C cscale(T s, C z) { return cmk<C>(s * z.x, s * z.y); }

// One k-point of the scaling in the arithmetic R (R = T, or double for the
// lowest wave numbers of FP32 spectra): reads the inputs at complex element e,
// writes T1 (and phi) in place.
template <typename R, typename T>
__device__ __forceinline__ void scale_point(const ScaleArgs<T>& a, int64_t e, const R k[3], R TH, R TB) {
  typedef typename Cplx<R>::type C;
  typedef typename Cplx<T>::type CT;
  const C zero = cmk<C>((R)0, (R)0);
  C T1[3] = {zero, zero, zero}, ph = zero;
  const R k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  auto ld = [&](int c) {
    const CT v = a.buf[c * a.cstride + e];
    return cmk<C>((R)v.x, (R)v.y);
  };
  if (a.iS >= 0) {  // -(k^2 I - k k) (1 + k^2/4xi^2) E B^R C1
    C Cv[3] = {ld(a.iS), ld(a.iS + 1), ld(a.iS + 2)};
    C kc = cadd(cadd(cscale(k[0], Cv[0]), cscale(k[1], Cv[1])), cscale(k[2], Cv[2]));
    for (int d = 0; d < 3; ++d) T1[d] = cadd(T1[d], cscale(-TB, cadd(cscale(k2, Cv[d]), cscale(-k[d], kc))));
  }
  if (a.iT >= 0) {  // -i (1 + k^2/4xi^2) E B^R [(k d + k d + k d) k^2 - 2 k k k] : C
    C c6[6];
    for (int m = 0; m < 6; ++m) c6[m] = ld(a.iT + m);
    const int sidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    C Ck[3], tr = cadd(cadd(c6[0], c6[3]), c6[5]);
    for (int j = 0; j < 3; ++j) {
      Ck[j] = zero;
      for (int m = 0; m < 3; ++m) Ck[j] = cadd(Ck[j], cscale(k[m], c6[sidx[j][m]]));
    }
    C kCk = cadd(cadd(cscale(k[0], Ck[0]), cscale(k[1], Ck[1])), cscale(k[2], Ck[2]));
    for (int j = 0; j < 3; ++j) {
      C v = cadd(cscale(k2, cadd(cscale((R)2, Ck[j]), cscale(k[j], tr))), cscale((R)(-2) * k[j], kCk));
      T1[j] = cadd(T1[j], cscale(-TB, cmul_i(v)));
    }
  }
  if (a.iW >= 0) {  // -2 i E H^R (C x k)
    C Cv[3] = {ld(a.iW), ld(a.iW + 1), ld(a.iW + 2)};
    C cr[3] = {cadd(cscale(k[2], Cv[1]), cscale(-k[1], Cv[2])), cadd(cscale(k[0], Cv[2]), cscale(-k[2], Cv[0])),
               cadd(cscale(k[1], Cv[0]), cscale(-k[0], Cv[1]))};
    for (int d = 0; d < 3; ++d) T1[d] = cadd(T1[d], cscale((R)(-2) * TH, cmul_i(cr[d])));
  }
  // harmonic potential of the wall corrections: phi^ = E H^R D^ (D spread
  // through window derivatives); T1 gains e3 phi, grad(phi) is gathered
  if (a.iD >= 0) {
    ph = cscale(TH, ld(a.iD));
    T1[2] = cadd(T1[2], ph);
  }
  for (int d = 0; d < 3; ++d) a.buf[d * a.cstride + e] = cmk<CT>((T)T1[d].x, (T)T1[d].y);
  if (a.nout == 4) a.buf[3 * a.cstride + e] = cmk<CT>((T)ph.x, (T)ph.y);
}

// 4 resident blocks of 256 threads per SM (64 registers): the pass streams the
// 7 input and 4 output spectra, and the extra warps keep more loads in flight
// (measured on the 1M workload: 9.84 -> 8.93 ms against the 72-register build
// at 3 blocks)
template <typename T>
__global__ void __launch_bounds__(256, 4) k_scale(ScaleArgs<T> a) {
  typedef typename Cplx<T>::type C;
  const int Mt = a.Mt, Nx = 2 * Mt, Ny = 2 * Mt, Nzh = 2 * Mt + 1;
  const int64_t nh = (int64_t)Nx * Ny * Nzh;
  const T dkx = (T)(2.0 * kPi / (Nx * a.h)), dkz = (T)(2.0 * kPi / (4.0 * Mt * a.h));
  const C zero = cmk<C>((T)0, (T)0);
  for (int64_t ee = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ee < nh * a.n_inst;
       ee += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = ee / nh, el = ee - inst * nh;
    int jz = (int)(el % Nzh);
    int64_t t = el / Nzh;
    int iy = (int)(t % Ny), ix = (int)(t / Ny);
    // element of component 0 of this instance
    const int64_t e = inst * a.istride + ix * a.xstride + (int64_t)iy * Nzh + jz;
    if (ix == Mt || iy == Mt || jz == 2 * Mt) {  // Nyquist modes are dropped
      for (int d = 0; d < a.nout; ++d) a.buf[d * a.cstride + e] = zero;
      continue;
    }
    const int wx = ix <= Mt ? ix : ix - Nx, wy = iy <= Mt ? iy : iy - Ny;
    const int ax = abs(wx), ay = abs(wy);
    if constexpr (std::is_same<T, float>::value) {
      const int K = a.lowK;
      if (a.tabLow && ax <= K && ay <= K && jz <= K) {
        // lowest wave numbers in FP64, with FP64 tables: the projections
        // k^2 C - k (k.C) of the smallest k are differences of nearly equal
        // terms, and these modes carry the far field
        const int nlow = (K + 1) * (K + 1) * (K + 1), li = (ax * (K + 1) + ay) * (K + 1) + jz;
        const double dx = 2.0 * kPi / (Nx * a.h), dz = 2.0 * kPi / (4.0 * Mt * a.h);
        const double k[3] = {dx * wx, dx * wy, dz * jz};
        scale_point<double, T>(a, e, k, a.tabLow[li], a.tabB ? a.tabLow[nlow + li] : 0.0);
        continue;
      }
    }
    const T k[3] = {dkx * wx, dkx * wy, dkz * jz};
    const int64_t ti = ((int64_t)ax * (Mt + 1) + ay) * Nzh + jz;
    const T TH = (T)a.tabH[ti];
    const T TB = a.tabB ? (T)a.tabB[ti] : (T)0;
    scale_point<T, T>(a, e, k, TH, TB);
  }
}

// --------------------------------------------------------------------- gather
template <typename T>
struct GatherArgs {
  int64_t n_tgt, n_src;
  const double* tgt;      // explicit targets or null
  const double* spos;     // sorted sources (targets = sources)
  const int32_t* sorig;
  const T* buf;           // fields T1x, T1y, T1z (, phi), buffer stride bs, real layout
  int64_t bs, xs, pitch;
  const int32_t* inst_of; // batched instances: instance of each sorted target (null: one)
  int64_t is;             // instance stride of the fields
  int P, Mt;
  double h, ox, oz, alpha, pre, h3;
  double inv_h;           // 1 / h
  double* out;
  int add;
};

constexpr int kGatherWarps = 4;

// warp sum in FP64 (a double-float butterfly sum measured slower: its FP32
// instructions compete for the issue slots the column sums need)
__device__ __forceinline__ double warp_sum64(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double warp_sum64(df v) { return warp_sum64(v.to_double()); }

// per-column sums of the gather are accumulated in FP64 (double grids) or
// double-float (double-float and FP32 grids)
// (FP32 grids: double-float sums on the FP32 pipe, where FP64 additions and
// float -> double conversions would queue on the narrow FP64 pipe)
template <typename T> struct GAcc { typedef double type; };
template <> struct GAcc<df> { typedef df type; };
template <> struct GAcc<float> { typedef df type; };
__device__ __forceinline__ double gacc(double v) { return v; }
__device__ __forceinline__ df gacc(float v) { return df(v, 0.f); }
__device__ __forceinline__ df gacc(df v) { return v; }

// NF = 3: u = <T1> (free space).  NF = 4: u = <T1> - x3 <grad phi>, the
// gradient taken through the window: <grad phi>(x) = h^3 sum_j grad_x W(x - x_j)
// phi_j, grad_x W = -W' with W' the derivative with respect to the grid point.
template <typename T, int NF>
__global__ void __launch_bounds__(kGatherWarps * 32) k_gather(GatherArgs<T> a) {
  __shared__ T wsm[kGatherWarps][6][kMaxP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* wx = wsm[wib][0];
  T* wy = wsm[wib][1];
  T* wz = wsm[wib][2];
  T* dwx = wsm[wib][3];
  T* dwy = wsm[wib][4];
  T* dwz = wsm[wib][5];
  const int P = a.P;
  const int64_t nwarps = (int64_t)gridDim.x * kGatherWarps;
  for (int64_t w = blockIdx.x * (int64_t)kGatherWarps + wib; w < a.n_tgt; w += nwarps) {
    double x, y, z;
    int64_t dst;
    if (a.tgt) {
      x = a.tgt[w]; y = a.tgt[a.n_tgt + w]; z = a.tgt[2 * a.n_tgt + w];
      dst = w;
    } else {
      x = a.spos[w]; y = a.spos[a.n_src + w]; z = a.spos[2 * a.n_src + w];
      dst = a.sorig[w];
    }
    // the target's P nearest grid points per axis (a product with 1/h: a
    // target within rounding of a grid plane may take the support one point
    // over, an equally valid quadrature; the spread's supports use the
    // correctly rounded quotient, which the oracle's grids reproduce)
    int ix0 = support_start_mul(x, a.ox, a.inv_h, P, a.Mt);
    int iy0 = support_start_mul(y, a.ox, a.inv_h, P, a.Mt);
    int iz0 = support_start_mul(z, a.oz, a.inv_h, P, 2 * a.Mt);
    const T* fields = a.buf + (a.inst_of ? a.inst_of[w] * a.is : 0);
    __syncwarp();
    if (lane < P) {
      const double d[3] = {a.ox + (ix0 + lane) * a.h - x, a.ox + (iy0 + lane) * a.h - y,
                           a.oz + (iz0 + lane) * a.h - z};
      double wv0 = a.pre * exp(-a.alpha * d[0] * d[0]);
      double wv1 = exp(-a.alpha * d[1] * d[1]);
      double wv2 = exp(-a.alpha * d[2] * d[2]);
      wx[lane] = (T)wv0;
      wy[lane] = (T)wv1;
      wz[lane] = (T)wv2;
      if (NF == 4) {
        dwx[lane] = (T)(-2.0 * a.alpha * d[0] * wv0);
        dwy[lane] = (T)(-2.0 * a.alpha * d[1] * wv1);
        dwz[lane] = (T)(-2.0 * a.alpha * d[2] * wv2);
      }
    }
    __syncwarp();
    // acc: <T1> (3), then the three window-derivative sums of phi (FP64, or
    // double-float for double-float grids)
    typename GAcc<T>::type acc[NF == 4 ? 6 : 3];
#pragma unroll
    for (int c = 0; c < (NF == 4 ? 6 : 3); ++c) acc[c] = 0;
    for (int q = lane; q < P * P; q += 32) {
      int jj = q / P, kk = q - jj * P;
      T s[3] = {0, 0, 0}, s0 = 0, s1 = 0;
      const T* col = fields + (int64_t)ix0 * a.xs + (int64_t)(iy0 + jj) * a.pitch + iz0 + kk;
      for (int ii = 0; ii < P; ++ii) {
        const T wv = wx[ii];
        const T* pnt = col + (int64_t)ii * a.xs;
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] = mac(s[c], wv, pnt[c * a.bs]);
        if (NF == 4) {
          const T ph = pnt[3 * a.bs];
          s0 = mac(s0, wv, ph);
          s1 = mac(s1, dwx[ii], ph);
        }
      }
      const T wyz = mulr(wy[jj], wz[kk]);
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += gacc(mulr(wyz, s[c]));
      if (NF == 4) {
        acc[3] += gacc(mulr(wyz, s1));
        acc[4] += gacc(mulr(mulr(dwy[jj], wz[kk]), s0));
        acc[5] += gacc(mulr(mulr(wy[jj], dwz[kk]), s0));
      }
    }
    double accd[NF == 4 ? 6 : 3];
#pragma unroll
    for (int c = 0; c < (NF == 4 ? 6 : 3); ++c) accd[c] = warp_sum64(acc[c]);
    if (lane == 0) {
      for (int d = 0; d < 3; ++d) {
        // grad_x W = -W', so u = <T1> - x3 <grad phi> = h^3 (acc_T1 + x3 acc_W')
        double v;
        if constexpr (NF == 4) v = a.h3 * (accd[d] + z * accd[3 + d]);
        else v = a.h3 * accd[d];
        double* o = a.out + d * a.n_tgt + dst;
        *o = a.add ? *o + v : v;
      }
    }
  }
}

// -------------------------------------------------------------------- drivers
static int blocks_for(int64_t n, int t, int cap) {
  int64_t b = (n + t - 1) / t;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

template <typename T>
static PrepArgs<T> prep_args(hse_plan p, int64_t n, int paper, int ncomp) {
  const hse_params& q = p->prm;
  PrepArgs<T> a;
  a.n = n;
  a.spos = p->ws.spos;
  a.sstr = p->ws.sstr;
  a.rowS = p->row_S; a.rowT = p->row_T; a.rowW = p->row_W;
  a.mask = q.kernel_mask;
  a.paper = paper;
  a.P = q.P;
  a.Mt = q.Mt;
  a.h = q.h;
  a.ox = -0.5 * q.P * q.h;
  a.oz = -(double)q.Mt * q.h;
  a.alpha = 2.0 * q.xi * q.xi / q.eta;
  a.pre = pow(2.0 * q.xi * q.xi / (kPi * q.eta), 1.5);
  a.c2 = std::exp(-2.0 * a.alpha * q.h * q.h);
  const int dk = paper ? 0 : deriv_kind(q.kernel_mask);
  a.nfac = dk == 0 ? 1 : ((dk & 4) ? 3 : 2);
  a.nc1 = c1_count(q.kernel_mask);
  // paper: plain windows and every component; product: derivative windows,
  // the combined x arrays of D and C1
  a.lay = rec_layout(a.nfac, paper ? ncomp : a.nc1, q.P, q.spread_tile);
  a.stride = a.lay.stride;
  a.prep = reinterpret_cast<T*>(p->ws.prep);
  // 8-byte grids split small window weights to FP32 unless an FP64 plan asks
  // for FP64 throughout (rc64 >= rc and no double-float band); the split's
  // error (a few 1e-14 relative) is far below any band's
  const bool split = sizeof(T) == 8 && !paper &&
                     (q.precision == HSE_MIXED || q.rc64 < q.rc || (q.rcmid > 0.0 && q.rcmid < q.rc));
  a.prep32 = split ? p->ws.prep32 : nullptr;
  a.supp = reinterpret_cast<int4*>(p->ws.supp);
  return a;
}

// full_z: the spread's tiles cover z from 0 (not from the lowest z a support
// reaches), so every point of the data region x, y < Mt, z < 2 Mt is written
// (zero where no source reaches) and the grid needs no clearing beforehand.
template <typename T>
static hse_status spread_into(hse_plan p, int64_t n_src, const CompSet& cs, int paper, T* out, int64_t cstride,
                              int64_t xs, int64_t pitch, cudaStream_t s, int n_inst = 1, int64_t istride = 0,
                              bool full_z = false) {
  const hse_params& q = p->prm;
  PrepArgs<T> pa = prep_args<T>(p, n_src, paper, cs.n);
  if (n_src > 0) {
    k_prep<T><<<blocks_for(n_src, 128, 152 * 32), 128, 0, s>>>(pa);
    ++p->n_launch;
    HSE_CUDA(p, cudaGetLastError());
  }
  SpreadArgs<T> a;
  a.supp = pa.supp;
  a.prep = pa.prep;
  a.prep32 = pa.prep32;
  a.spos32 = p->ws.spos32;
  a.n_src = n_src;
  // FP32 below a fraction tau of the window's peak: those terms carry
  // relative errors <~ 4 eps32 tau of the largest contribution of their
  // particle.  Measured on the 1M near-wall S+W workload the velocity changes
  // by ~5e-9 tau (relative RMS) against an all-FP64 spread, so a plan that
  // knows its tolerance takes tau = 2e6 tol (its share stays ~1/100 of tol).
  // Stokeslets spread through the box are worse: their rounding noise is
  // white, and the low wave numbers, where the image system cancels the
  // long-range field, scale it by ~1/k^2, so the Fourier part changes by
  // ~1.6e-9 tau sqrt(N) (uniform sources, N = 79k-135k at tau = 2e-4:
  // 0.9e-10-1.2e-10); stokeslet plans cap tau at tol / (1.6e-8 sqrt(N)) per
  // instance, which keeps that share below tol / 10.  tau stays within
  // [1e-5, 1e-3]; plans with explicit parameters and no tol keep tau = 1e-5.
  a.ah2 = (float)(pa.alpha * q.h * q.h);
  double tau = p->tol > 0.0 ? 2e6 * p->tol : 1e-5;
  if (p->tol > 0.0 && (q.kernel_mask & HSE_STOKESLET) && n_src > 0) {
    const double n_per = (double)n_src / (n_inst > 0 ? n_inst : 1);
    tau = std::fmin(tau, p->tol / (1.6e-8 * std::sqrt(n_per)));
  }
  tau = std::fmin(1e-3, std::fmax(1e-5, tau));
  a.lnthr = (float)std::log(1.0 / tau);

  a.cstart = p->ws.cell_start;
  a.stride = pa.stride;
  a.y0 = pa.lay.y0;
  a.z0r = pa.lay.z0;
  a.c0 = pa.lay.c0;
  a.pad[0] = pa.lay.px;
  a.pad[1] = pa.lay.py;
  a.pad[2] = pa.lay.pz;
  a.P = q.P;
  a.Mt = q.Mt;
  // full_z: tiles on the same z boundaries as from zA0, extended down to the
  // first tile at or below 0 (the same warp sub-tiles, so the same FP32 /
  // higher-precision split of the small weights as without full_z)
  const int tx = 2 * q.spread_tile[0], ty = 2 * q.spread_tile[1], tz = 2 * q.spread_tile[2];  // block tile
  for (int d = 0; d < 3; ++d) {
    int l = 0;
    while ((1 << l) < q.spread_tile[d]) ++l;
    a.wl[d] = l;
  }
  a.z0 = full_z ? p->zA0 - ((p->zA0 + tz - 1) / tz) * tz : p->zA0;
  a.zlo = p->zA0;
  a.h = q.h;
  a.ox = pa.ox;
  a.oz = pa.oz;
  for (int d = 0; d < 3; ++d) { a.inv_cell[d] = p->inv_cell[d]; a.ncell[d] = q.ncell[d]; }
  a.out = out;
  a.cs = cstride;
  a.xs = xs;
  a.pitch = pitch;
  a.is = istride;
  a.ncells_inst = q.ncell[0] * q.ncell[1] * q.ncell[2];
  int nzr = 2 * q.Mt - a.z0;
  a.nz_tiles = (nzr + tz - 1) / tz;
  dim3 grid((q.Mt + tx - 1) / tx, (q.Mt + ty - 1) / ty, a.nz_tiles * n_inst);
  const int dk = paper ? 0 : deriv_kind(q.kernel_mask);
  const int nplain = dk ? cs.n - 1 : cs.n;  // the product set's last component is D
  if (!launch_spread<T>(nplain, dk, a, grid, s))
    return set_err(p, HSE_ERR_UNSUPPORTED, "no spread kernel for %d comps", cs.n);
  ++p->n_launch;
  HSE_CUDA(p, cudaGetLastError());
  if (free_space(q.kernel_mask)) return HSE_OK;  // no images: C1 is the source-located grid
  MirrorArgs<T> m;
  m.buf = out;
  m.cs = cstride;
  m.xs = xs;
  m.pitch = pitch;
  m.Mt = q.Mt;
  m.nc = cs.n;
  m.n_inst = n_inst;
  m.is = istride;
  for (int c = 0; c < cs.n; ++c) m.sign[c] = cs.mirror_sign[c];
  int64_t tot = (int64_t)q.Mt * q.Mt * (q.Mt + 1) * cs.n * n_inst;
  k_mirror<T><<<blocks_for(tot, 256, 152 * 64), 256, 0, s>>>(m);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_mirror");
}

hse_status spread_paper_grids(hse_plan p, int64_t n_src, double* grids, cudaStream_t s) {
  const int Mt = p->prm.Mt;
  CompSet cs = paper_components(p->prm.kernel_mask);
  int64_t per = (int64_t)Mt * Mt * 2 * Mt;
  HSE_CUDA(p, cudaMemsetAsync(grids, 0, sizeof(double) * per * cs.n, s));
  return spread_into<double>(p, n_src, cs, 1, grids, per, (int64_t)Mt * 2 * Mt, 2 * Mt, s);
}

// forward / inverse zero-padded transforms of one buffer (double or float)
static cufftResult fft_forward(hse_plan p, double* b) {
  cufftDoubleComplex* z = reinterpret_cast<cufftDoubleComplex*>(b);
  cufftResult r = cufftExecD2Z(p->fwd2d, b, z);
  return r == CUFFT_SUCCESS ? cufftExecZ2Z(p->fftx, z, z, CUFFT_FORWARD) : r;
}
static cufftResult fft_forward(hse_plan p, float* b) {
  cufftComplex* z = reinterpret_cast<cufftComplex*>(b);
  cufftResult r = cufftExecR2C(p->fwd2d, b, z);
  return r == CUFFT_SUCCESS ? cufftExecC2C(p->fftx, z, z, CUFFT_FORWARD) : r;
}
static cufftResult fft_inverse(hse_plan p, double* b) {
  cufftDoubleComplex* z = reinterpret_cast<cufftDoubleComplex*>(b);
  cufftResult r = cufftExecZ2Z(p->fftx, z, z, CUFFT_INVERSE);
  return r == CUFFT_SUCCESS ? cufftExecZ2D(p->inv2d, z, b) : r;
}
static cufftResult fft_inverse(hse_plan p, float* b) {
  cufftComplex* z = reinterpret_cast<cufftComplex*>(b);
  cufftResult r = cufftExecC2C(p->fftx, z, z, CUFFT_INVERSE);
  return r == CUFFT_SUCCESS ? cufftExecC2R(p->inv2d, z, b) : r;
}

// Scale the spectra of n_inst instances (component c of instance i, mode
// (kx, ky, kz) at c cstride + i istride + kx xstride + ky nzh + kz complex
// elements) in the arithmetic S, in place.
template <typename S>
static hse_status launch_scale(hse_plan p, void* spec, int64_t cstride, int n_inst, int64_t istride, int64_t xstride,
                               cudaStream_t s) {
  const hse_params& q = p->prm;
  const GridDims& g = p->g;
  ScaleArgs<S> sa;
  sa.buf = reinterpret_cast<typename Cplx<S>::type*>(spec);
  sa.cstride = cstride;
  sa.Mt = q.Mt;
  sa.mask = q.kernel_mask;
  sa.h = q.h;
  constexpr bool dft = std::is_same<S, df>::value;
  sa.tabB = reinterpret_cast<const typename Tab<S>::type*>(dft ? p->tabB_df : p->tabB);
  sa.tabH = reinterpret_cast<const typename Tab<S>::type*>(dft ? p->tabH_df : p->tabH);
  sa.tabLow = std::is_same<S, float>::value ? p->tabLow : nullptr;
  sa.lowK = kLowK < q.Mt ? kLowK : q.Mt;
  int k = 0;
  sa.iS = sa.iT = sa.iW = sa.iD = -1;
  if (q.kernel_mask & HSE_STOKESLET) { sa.iS = k; k += 3; }
  if (q.kernel_mask & HSE_STRESSLET) { sa.iT = k; k += 6; }
  if (q.kernel_mask & HSE_ROTLET) { sa.iW = k; k += 3; }
  if (!free_space(q.kernel_mask)) sa.iD = k;
  sa.nout = q.n_fft_out;
  sa.n_inst = n_inst;
  sa.istride = istride;
  sa.xstride = xstride;
  k_scale<S><<<blocks_for(g.nh * n_inst, 256, 152 * 32), 256, 0, s>>>(sa);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_scale");
}

template <typename T>
static hse_status fourier_space_t(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                                  cudaStream_t s, cudaEvent_t gather_after) {
  const hse_params& q = p->prm;
  const GridDims& g = p->g;
  const int nin = p->comps.n;
  T* spec = reinterpret_cast<T*>(p->spec);
  // cuFFT reads the whole padded grid (zeros outside the data region); the
  // double-float transforms read only the data region, which the spread
  // writes in full
  constexpr bool full_z = std::is_same<T, df>::value;
  if (!full_z) HSE_CUDA(p, cudaMemsetAsync(spec, 0, sizeof(T) * g.buf_doubles * nin, s));
  HSE_TRY(spread_into<T>(p, n_src, p->comps, 0, spec, g.buf_doubles, (int64_t)g.Ny * g.pitch, g.pitch, s, 1, 0,
                         full_z));
  stage_mark(p, HSE_STAGE_FFT, s);
  // double-float grids go with the double-float transforms; double and float
  // grids with cuFFT
  constexpr bool df64 = std::is_same<T, df>::value;
  const long long xs = (long long)g.Ny * g.pitch;
  if constexpr (df64) {
    HSE_TRY(fft64_forward(p, reinterpret_cast<double*>(spec), nin, g.buf_doubles, xs, s));
    p->n_fft += nin;
  } else {
    if (cufftSetStream(p->fwd2d, s) != CUFFT_SUCCESS || cufftSetStream(p->inv2d, s) != CUFFT_SUCCESS ||
        cufftSetStream(p->fftx, s) != CUFFT_SUCCESS)
      return set_err(p, HSE_ERR_CUFFT, "cufftSetStream");
    for (int c = 0; c < nin; ++c) {
      cufftResult r = fft_forward(p, spec + c * g.buf_doubles);
      ++p->n_fft;
      if (r != CUFFT_SUCCESS) return set_err(p, HSE_ERR_CUFFT, "forward FFT: %d", (int)r);
    }
  }
  stage_mark(p, HSE_STAGE_SCALE, s);
  const int64_t planec = (int64_t)g.Ny * (g.Nz / 2 + 1);
  HSE_TRY(launch_scale<T>(p, spec, g.nh, 1, 0, planec, s));
  stage_mark(p, HSE_STAGE_IFFT, s);
  if constexpr (df64) {
    HSE_TRY(fft64_inverse(p, reinterpret_cast<double*>(spec), q.n_fft_out, g.buf_doubles, xs, s));
    p->n_fft += q.n_fft_out;
  } else {
    for (int c = 0; c < q.n_fft_out; ++c) {
      cufftResult r = fft_inverse(p, spec + c * g.buf_doubles);
      ++p->n_fft;
      if (r != CUFFT_SUCCESS) return set_err(p, HSE_ERR_CUFFT, "inverse FFT: %d", (int)r);
    }
  }
  stage_mark(p, HSE_STAGE_GATHER, s);
  if (n_tgt == 0) return HSE_OK;
  if (gather_after) HSE_CUDA(p, cudaStreamWaitEvent(s, gather_after, 0));
  GatherArgs<T> ga;
  ga.n_tgt = n_tgt;
  ga.n_src = n_src;
  ga.tgt = tgt;
  ga.spos = p->ws.spos;
  ga.sorig = p->ws.val_a;
  ga.buf = spec;
  ga.bs = g.buf_doubles;
  ga.xs = (int64_t)g.Ny * g.pitch;
  ga.pitch = g.pitch;
  ga.inst_of = nullptr;
  ga.is = 0;
  ga.P = q.P;
  ga.Mt = q.Mt;
  ga.h = q.h;
  ga.ox = -0.5 * q.P * q.h;
  ga.oz = -(double)q.Mt * q.h;
  ga.alpha = 2.0 * q.xi * q.xi / q.eta;
  ga.pre = pow(2.0 * q.xi * q.xi / (kPi * q.eta), 1.5);
  ga.h3 = q.h * q.h * q.h;
  ga.inv_h = 1.0 / q.h;
  ga.out = out;
  ga.add = add ? 1 : 0;
  if (q.n_fft_out == 4) k_gather<T, 4><<<blocks_for(n_tgt, kGatherWarps, 152 * 64), kGatherWarps * 32, 0, s>>>(ga);
  else k_gather<T, 3><<<blocks_for(n_tgt, kGatherWarps, 152 * 64), kGatherWarps * 32, 0, s>>>(ga);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_gather");
}

// Batched instances: n_inst instances sharing the plan's grid, particles sorted
// by (instance, cell) in the plan's workspace, inst_of per sorted particle.
// spec: component-major buffers, component c of instance i at (c n_inst + i)
// buffers; fwd / inv: batched 3-D transforms over n_fft_in * n_inst and
// 6 * n_inst buffers.  Adds the Fourier part of every particle to out
// (concatenated order).
// ------------------------------------------------------- batched transforms
// One exec of a batched plan: kind 0 = 2-D (y,z) R2C over `batch` planes at
// real offset `off`; 1 = 2-D C2R likewise; 2 / 3 = 1-D x transform, forward /
// inverse, over `batch` lines starting at complex offset `off`, element
// stride `stride`.
struct FftExec {
  int kind;
  int64_t off, batch, stride;
};

constexpr int64_t kBatchPlanes = 2048;     // planes per 2-D exec (about 0.3-1 GB of data)
constexpr int64_t kBatchLines = 1 << 20;   // lines per 1-D exec

static std::vector<FftExec> batch_schedule(const GridDims& g, int nc, int n_out, int C, bool forward) {
  const int64_t nzh = g.Nz / 2 + 1, plane = (int64_t)g.Ny * g.pitch, planec = (int64_t)g.Ny * nzh;
  const int64_t nbuf = (int64_t)nc * C, Mt = g.Mt;
  const int64_t gb = std::max<int64_t>(1, std::min<int64_t>(kBatchLines / planec, nbuf));
  std::vector<FftExec> ex;
  if (forward) {
    // 2-D over the data planes x < Mt of every buffer (one contiguous half),
    // then x lines of every buffer
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(kBatchPlanes / nbuf, Mt));
    for (int64_t x0 = 0; x0 < Mt; x0 += gx)
      ex.push_back({0, x0 * nbuf * plane, std::min(gx, Mt - x0) * nbuf, 0});
    for (int64_t j0 = 0; j0 < nbuf; j0 += gb)
      ex.push_back({2, j0 * planec, std::min(gb, nbuf - j0) * planec, nbuf * planec});
  } else {
    // x lines of the n_out output components, then 2-D over the planes x < Mt
    // the gather reads, one x plane at a time (the outputs are contiguous in it)
    const int64_t nout = (int64_t)n_out * C;
    for (int64_t j0 = 0; j0 < nout; j0 += gb)
      ex.push_back({3, j0 * planec, std::min(gb, nout - j0) * planec, nbuf * planec});
    for (int64_t x = 0; x < Mt; ++x) ex.push_back({1, x * nbuf * plane, nout, 0});
  }
  return ex;
}

static cufftHandle find_plan(const BatchFFT& f, int kind, int64_t batch, int64_t stride) {
  const int k = kind == 3 ? 2 : kind;
  for (const auto& e : f.plans)
    if (e.kind == k && e.batch == batch && e.stride == stride) return e.h;
  return 0;
}

hse_status batch_fft_prepare(hse_plan p, BatchFFT& f, int n_inst, char** work, int64_t* work_cap) {
  if (p->prm.fft == HSE_FFT_DF64) return fft64_prepare(p);  // no cuFFT plans, no work area
  const GridDims& g = p->g;
  const bool mixed = p->prm.precision == HSE_MIXED;
  const long long nzh = g.Nz / 2 + 1;
  const long long plane = (long long)g.Ny * g.pitch, planec = (long long)g.Ny * nzh;
  std::vector<FftExec> ex = batch_schedule(g, p->comps.n, p->prm.n_fft_out, n_inst, true);
  std::vector<FftExec> ex2 = batch_schedule(g, p->comps.n, p->prm.n_fft_out, n_inst, false);
  ex.insert(ex.end(), ex2.begin(), ex2.end());
  size_t need = 0;
  for (const FftExec& e : ex) {
    const int kind = e.kind == 3 ? 2 : e.kind;
    bool found = false;
    for (const auto& q : f.plans)
      if (q.kind == kind && q.batch == e.batch && q.stride == e.stride) {
        found = true;
        need = std::max(need, q.work);
      }
    if (found) continue;
    BatchFFT::Entry en{kind, e.batch, e.stride, 0, 0};
    if (cufftCreate(&en.h) != CUFFT_SUCCESS) return set_err(p, HSE_ERR_CUFFT, "cufftCreate");
    cufftSetAutoAllocation(en.h, 0);
    cufftResult r;
    if (kind == 0 || kind == 1) {
      long long n2[2] = {g.Ny, g.Nz}, re[2] = {g.Ny, g.pitch}, ce[2] = {g.Ny, nzh};
      if (kind == 0)
        r = cufftMakePlanMany64(en.h, 2, n2, re, 1, plane, ce, 1, planec, mixed ? CUFFT_R2C : CUFFT_D2Z, e.batch,
                                &en.work);
      else
        r = cufftMakePlanMany64(en.h, 2, n2, ce, 1, planec, re, 1, plane, mixed ? CUFFT_C2R : CUFFT_Z2D, e.batch,
                                &en.work);
    } else {
      long long nx[1] = {g.Nx}, xe[1] = {g.Nx};
      r = cufftMakePlanMany64(en.h, 1, nx, xe, e.stride, 1, xe, e.stride, 1, mixed ? CUFFT_C2C : CUFFT_Z2Z, e.batch,
                              &en.work);
    }
    if (r != CUFFT_SUCCESS) {
      cufftDestroy(en.h);
      return set_err(p, r == CUFFT_ALLOC_FAILED ? HSE_ERR_OOM : HSE_ERR_CUFFT, "batched cuFFT plan (kind %d): %d",
                     kind, (int)r);
    }
    need = std::max(need, en.work);
    f.plans.push_back(en);
  }
  if ((int64_t)need > *work_cap) {
    cudaFree(*work);  // synchronises with work in flight
    *work = nullptr;
    *work_cap = 0;
    HSE_CUDA(p, cudaMalloc(work, need));
    *work_cap = (int64_t)need;
  }
  for (const auto& q : f.plans)
    if (q.work && cufftSetWorkArea(q.h, *work) != CUFFT_SUCCESS)
      return set_err(p, HSE_ERR_CUFFT, "cufftSetWorkArea");
  return HSE_OK;
}

void batch_fft_destroy(BatchFFT& f) {
  for (auto& e : f.plans) cufftDestroy(e.h);
  f.plans.clear();
}

template <typename T>
static hse_status run_schedule(hse_plan p, const BatchFFT& f, const std::vector<FftExec>& ex, T* spec,
                               cudaStream_t s) {
  typedef typename std::conditional<sizeof(T) == 8, cufftDoubleComplex, cufftComplex>::type C;
  for (const FftExec& e : ex) {
    cufftHandle h = find_plan(f, e.kind, e.batch, e.stride);
    if (!h) return set_err(p, HSE_ERR_CUFFT, "batched cuFFT plan missing (kind %d)", e.kind);
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return set_err(p, HSE_ERR_CUFFT, "cufftSetStream");
    cufftResult r;
    if (e.kind == 0) {
      T* x = spec + e.off;
      if (sizeof(T) == 8) r = cufftExecD2Z(h, (double*)x, (cufftDoubleComplex*)x);
      else r = cufftExecR2C(h, (float*)x, (cufftComplex*)x);
    } else if (e.kind == 1) {
      T* x = spec + e.off;
      if (sizeof(T) == 8) r = cufftExecZ2D(h, (cufftDoubleComplex*)x, (double*)x);
      else r = cufftExecC2R(h, (cufftComplex*)x, (float*)x);
    } else {
      C* z = reinterpret_cast<C*>(spec) + e.off;
      const int dir = e.kind == 2 ? CUFFT_FORWARD : CUFFT_INVERSE;
      if (sizeof(T) == 8) r = cufftExecZ2Z(h, (cufftDoubleComplex*)z, (cufftDoubleComplex*)z, dir);
      else r = cufftExecC2C(h, (cufftComplex*)z, (cufftComplex*)z, dir);
    }
    ++p->n_fft;
    if (r != CUFFT_SUCCESS) return set_err(p, HSE_ERR_CUFFT, "batched FFT exec (kind %d): %d", e.kind, (int)r);
  }
  return HSE_OK;
}

// Alg. 1 over C instances at once, on slab-major grids (see BatchFFT).
template <typename T>
static hse_status fourier_space_batch_t(hse_plan p, int64_t n_total, int n_inst, const int32_t* inst_of, void* specv,
                                        const BatchFFT& f, double* out, cudaStream_t s) {
  const hse_params& q = p->prm;
  const GridDims& g = p->g;
  const int nin = p->comps.n;
  T* spec = reinterpret_cast<T*>(specv);
  const int64_t nzh = g.Nz / 2 + 1, plane = (int64_t)g.Ny * g.pitch, planec = (int64_t)g.Ny * nzh;
  const int64_t nbuf = (int64_t)nin * n_inst;
  constexpr bool full_z = std::is_same<T, df>::value;  // as in fourier_space_t
  if (!full_z) HSE_CUDA(p, cudaMemsetAsync(spec, 0, sizeof(T) * g.buf_doubles * nbuf, s));
  HSE_TRY(spread_into<T>(p, n_total, p->comps, 0, spec, plane * n_inst, plane * nbuf, g.pitch, s, n_inst, plane,
                         full_z));
  stage_mark(p, HSE_STAGE_FFT, s);
  constexpr bool df64 = std::is_same<T, df>::value;
  if constexpr (df64) {
    HSE_TRY(fft64_forward(p, reinterpret_cast<double*>(spec), (int)nbuf, plane, plane * nbuf, s));
    p->n_fft += (int)nbuf;
  } else {
    HSE_TRY(run_schedule<T>(p, f, batch_schedule(g, nin, q.n_fft_out, n_inst, true), spec, s));
  }
  stage_mark(p, HSE_STAGE_SCALE, s);
  HSE_TRY(launch_scale<T>(p, spec, planec * n_inst, n_inst, planec, planec * nbuf, s));
  stage_mark(p, HSE_STAGE_IFFT, s);
  if constexpr (df64) {
    HSE_TRY(fft64_inverse(p, reinterpret_cast<double*>(spec), q.n_fft_out * n_inst, plane, plane * nbuf, s));
    p->n_fft += q.n_fft_out * n_inst;
  } else {
    HSE_TRY(run_schedule<T>(p, f, batch_schedule(g, nin, q.n_fft_out, n_inst, false), spec, s));
  }
  stage_mark(p, HSE_STAGE_GATHER, s);
  GatherArgs<T> ga;
  ga.n_tgt = n_total;
  ga.n_src = n_total;
  ga.tgt = nullptr;
  ga.spos = p->ws.spos;
  ga.sorig = p->ws.val_a;
  ga.buf = spec;
  ga.bs = plane * n_inst;
  ga.xs = plane * nbuf;
  ga.pitch = g.pitch;
  ga.inst_of = inst_of;
  ga.is = plane;
  ga.P = q.P;
  ga.Mt = q.Mt;
  ga.h = q.h;
  ga.ox = -0.5 * q.P * q.h;
  ga.oz = -(double)q.Mt * q.h;
  ga.alpha = 2.0 * q.xi * q.xi / q.eta;
  ga.pre = pow(2.0 * q.xi * q.xi / (kPi * q.eta), 1.5);
  ga.h3 = q.h * q.h * q.h;
  ga.inv_h = 1.0 / q.h;
  ga.out = out;
  ga.add = 1;
  if (q.n_fft_out == 4)
    k_gather<T, 4><<<blocks_for(n_total, kGatherWarps, 152 * 64), kGatherWarps * 32, 0, s>>>(ga);
  else k_gather<T, 3><<<blocks_for(n_total, kGatherWarps, 152 * 64), kGatherWarps * 32, 0, s>>>(ga);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "batched k_gather");
}

hse_status fourier_space_batch(hse_plan p, int64_t n_total, int n_inst, const int32_t* inst_of, void* spec,
                               BatchFFT& f, double* out, cudaStream_t s) {
  // double-float grids first: FP64 plans, and HSE_MIXED plans asked for a
  // double-float Fourier part
  if (p->prm.fft == HSE_FFT_DF64) return fourier_space_batch_t<df>(p, n_total, n_inst, inst_of, spec, f, out, s);
  if (p->prm.precision == HSE_MIXED)
    return fourier_space_batch_t<float>(p, n_total, n_inst, inst_of, spec, f, out, s);
  return fourier_space_batch_t<double>(p, n_total, n_inst, inst_of, spec, f, out, s);
}

hse_status fourier_space(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                         cudaStream_t s, cudaEvent_t gather_after) {
  if (p->prm.fft == HSE_FFT_DF64) return fourier_space_t<df>(p, n_src, n_tgt, tgt, out, add, s, gather_after);
  if (p->prm.precision == HSE_MIXED) return fourier_space_t<float>(p, n_src, n_tgt, tgt, out, add, s, gather_after);
  return fourier_space_t<double>(p, n_src, n_tgt, tgt, out, add, s, gather_after);
}

}  // namespace hse
