// hse_real.cu -- real-space part of the Ewald split (Sec. 4, Sec. 5.1).
//
// For each target x, over sources y within r_c (free-space pairs, the target's
// own source excluded) and over images y^I within r_c (always included):
//   S:  S^R(r) f      - S^R(rt) f^I
//   T:  T^R(r)(g q)   - T^R(rt)(g^I q^I)
//   W:  W^R(r) tau    + W^R(rt) tau^I
//   + the real-space parts of the wall corrections -x3 grad(phi) + e3 phi,
//     with G_R = erfc(xi r)/r and its derivatives (Sec. 4, eq. G_R) at rt,
// plus the stokeslet self term -4 xi/sqrt(pi) f (Appendix).
// The kernels are those of the Appendix (eq. kernel_real_parts) written with
// erfc; the last term of T^R carries r (not the unit vector), which is the
// dimensionally consistent form.
//
// Work split: one warp per target.  Lanes test 32 candidates at a time with
// the exact cut-off decision ((dx*dx + dy*dy) + dz*dz < r_c^2, no FMA) and the
// passing ones are compacted into a per-warp queue; whenever 32 are queued,
// every lane evaluates one pair, so the FP64 pipe always runs full warps.
#include "hse_internal.cuh"

namespace hse {

struct RealArgs {
  int64_t n_src, n_tgt;
  const double* spos;      // sorted sources, 3 x n_src
  const double* sstr;      // sorted strengths, rows x n_src
  const int32_t* sorig;    // sorted -> original source index
  const int32_t* cstart;   // cell starts
  const double* tgt;       // explicit targets (3 x n_tgt) or null (targets = sources)
  double* out;             // 3 x n_tgt in caller order
  int add;                 // accumulate into out
  int mask, rowS, rowT, rowW;
  double xi, rc2, rc;
  double inv_cell[3];
  int ncell[3];
};

enum { Q_FREE = 0, Q_IMAGE = 1, Q_SELF = 2 };
constexpr int kWarpsPerBlock = 4;
constexpr int kQueue = 64;

// Contribution of one queued pair to the lane's accumulator.
__device__ __forceinline__ void eval_pair(const RealArgs& a, const double* x, int j, int type, double* u) {
  const int64_t n = a.n_src;
  double y0 = a.spos[j], y1 = a.spos[n + j], y2 = a.spos[2 * n + j];
  double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, q[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
  if (a.mask & HSE_STOKESLET)
    for (int i = 0; i < 3; ++i) f[i] = a.sstr[(a.rowS + i) * n + j];
  if (a.mask & HSE_STRESSLET)
    for (int i = 0; i < 3; ++i) { g[i] = a.sstr[(a.rowT + i) * n + j]; q[i] = a.sstr[(a.rowT + 3 + i) * n + j]; }
  if (a.mask & HSE_ROTLET)
    for (int i = 0; i < 3; ++i) tau[i] = a.sstr[(a.rowW + i) * n + j];
  if (type == Q_SELF) {
    double c = -4.0 * a.xi / kSqrtPi;
    for (int i = 0; i < 3; ++i) u[i] += c * f[i];
    return;
  }
  const double xi = a.xi;
  double r[3] = {x[0] - y0, x[1] - y1, type == Q_IMAGE ? x[2] + y2 : x[2] - y2};
  double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double inv = rsqrt(s);
  double rho = s * inv;
  double t = xi * rho;
  double ec = erfc(t);
  double c = (2.0 / kSqrtPi) * xi * exp(-t * t);  // 2 xi e^{-t^2}/sqrt(pi)
  double i1 = inv, i2 = inv * inv;
  double ecr = ec * i1;
  double a1 = (ecr + c) * i2;  // erfc/r^3 + 2 xi e/(sqrt(pi) r^2)
  if (type == Q_FREE) {
    if (a.mask & HSE_STOKESLET) {
      double sa = ecr - c, sb = (c + ecr) * i2;
      double rf = r[0] * f[0] + r[1] * f[1] + r[2] * f[2];
      for (int i = 0; i < 3; ++i) u[i] += sa * f[i] + sb * r[i] * rf;
    }
    if (a.mask & HSE_STRESSLET) {
      double ta = -2.0 * i2 * i2 * (3.0 * ecr + c * (3.0 + 2.0 * t * t));
      double tb = 2.0 * xi * xi * c;
      double rg = r[0] * g[0] + r[1] * g[1] + r[2] * g[2];
      double rq = r[0] * q[0] + r[1] * q[1] + r[2] * q[2];
      double gq = g[0] * q[0] + g[1] * q[1] + g[2] * q[2];
      for (int i = 0; i < 3; ++i) u[i] += ta * r[i] * rg * rq + tb * (g[i] * rq + q[i] * rg + r[i] * gq);
    }
    if (a.mask & HSE_ROTLET) {
      double wa = 2.0 * a1;
      u[0] += wa * (tau[1] * r[2] - tau[2] * r[1]);
      u[1] += wa * (tau[2] * r[0] - tau[0] * r[2]);
      u[2] += wa * (tau[0] * r[1] - tau[1] * r[0]);
    }
    return;
  }
  // image pair at rt = r, source height h
  const double h = y2, x3 = x[2];
  double g1 = -a1;
  double g2 = 3.0 * ecr * i2 * i2 + c * (3.0 * i2 * i2 + 2.0 * xi * xi * i2);
  double phi = 0.0, gp[3] = {0.0, 0.0, 0.0};
  if (a.mask & HSE_STOKESLET) {
    double fI[3] = {f[0], f[1], -f[2]};
    double sa = ecr - c, sb = (c + ecr) * i2;
    double rf = r[0] * fI[0] + r[1] * fI[1] + r[2] * fI[2];
    for (int i = 0; i < 3; ++i) u[i] -= sa * fI[i] + sb * r[i] * rf;
    double g0 = ecr;
    phi += 2.0 * (-f[2] * g0 - h * g1 * rf);
    for (int i = 0; i < 3; ++i) gp[i] += 2.0 * (-f[2] * g1 * r[i] - h * (g1 * fI[i] + g2 * r[i] * rf));
  }
  if (a.mask & HSE_STRESSLET) {
    double gI[3] = {g[0], g[1], -g[2]}, qI[3] = {q[0], q[1], -q[2]};
    double ta = -2.0 * i2 * i2 * (3.0 * ecr + c * (3.0 + 2.0 * t * t));
    double tb = 2.0 * xi * xi * c;
    double rg = r[0] * gI[0] + r[1] * gI[1] + r[2] * gI[2];
    double rq = r[0] * qI[0] + r[1] * qI[1] + r[2] * qI[2];
    double gq = gI[0] * qI[0] + gI[1] * qI[1] + gI[2] * qI[2];
    for (int i = 0; i < 3; ++i) u[i] -= ta * r[i] * rg * rq + tb * (gI[i] * rq + qI[i] * rg + r[i] * gq);
    double g3 = -15.0 * ecr * i2 * i2 * i2 -
                c * (15.0 * i2 * i2 * i2 + 10.0 * xi * xi * i2 * i2 + 4.0 * xi * xi * xi * xi * i2);
    // phi_T = 4 (gI.qI) d3G - 4 h gI.(grad grad G) qI
    phi += 4.0 * gq * g1 * r[2] - 4.0 * h * (g1 * gq + g2 * rg * rq);
    for (int i = 0; i < 3; ++i) {
      double d3i = g1 * (i == 2 ? 1.0 : 0.0) + g2 * r[2] * r[i];
      double t3 = g2 * (gq * r[i] + gI[i] * rq + qI[i] * rg) + g3 * rg * rq * r[i];
      gp[i] += 4.0 * gq * d3i - 4.0 * h * t3;
    }
  }
  if (a.mask & HSE_ROTLET) {
    double tI[3] = {tau[0], tau[1], -tau[2]};
    double wa = 2.0 * a1;
    u[0] += wa * (tI[1] * r[2] - tI[2] * r[1]);
    u[1] += wa * (tI[2] * r[0] - tI[0] * r[2]);
    u[2] += wa * (tI[0] * r[1] - tI[1] * r[0]);
    double v0 = -tau[1], v1 = tau[0];
    double rv = r[0] * v0 + r[1] * v1;
    phi += 4.0 * g1 * rv;
    gp[0] += 4.0 * (g1 * v0 + g2 * r[0] * rv);
    gp[1] += 4.0 * (g1 * v1 + g2 * r[1] * rv);
    gp[2] += 4.0 * (g2 * r[2] * rv);
  }
  for (int i = 0; i < 3; ++i) u[i] -= x3 * gp[i];
  u[2] += phi;
}

// Iterate the candidate cells of a target and call visit(j, type) for every
// source passing the exact cut-off test (plus the self pair).
template <typename Visit>
__device__ __forceinline__ void for_candidates(const RealArgs& a, const double* x, int64_t own, int lane,
                                               Visit&& visit) {
  int cx = cell_coord(x[0], a.inv_cell[0], a.ncell[0]);
  int cy = cell_coord(x[1], a.inv_cell[1], a.ncell[1]);
  int cz = cell_coord(x[2], a.inv_cell[2], a.ncell[2]);
  const int64_t n = a.n_src;
  const int nx = a.ncell[0], ny = a.ncell[1], nz = a.ncell[2];
  // images only reach targets with x3 < rc, and come from sources with y3 < rc - x3
  bool want_img = x[2] < a.rc;
  int czi_hi = want_img ? cell_coord(a.rc - x[2], a.inv_cell[2], nz) : -1;
  for (int pass = 0; pass < 2; ++pass) {
    int z0 = pass == 0 ? (cz > 0 ? cz - 1 : 0) : 0;
    int z1 = pass == 0 ? (cz < nz - 1 ? cz + 1 : nz - 1) : czi_hi;
    for (int iz = z0; iz <= z1; ++iz)
      for (int iy = (cy > 0 ? cy - 1 : 0); iy <= (cy < ny - 1 ? cy + 1 : ny - 1); ++iy) {
        // x-neighbours are contiguous in the cell numbering
        int xa = cx > 0 ? cx - 1 : 0, xb = cx < nx - 1 ? cx + 1 : nx - 1;
        int c0 = (iz * ny + iy) * nx + xa;
        int s0 = a.cstart[c0], s1 = a.cstart[c0 + (xb - xa) + 1];
        for (int base = s0; base < s1; base += 32) {
          int j = base + lane;
          bool ok = j < s1;
          int type = 0;
          bool hit = false;
          if (ok) {
            double y0 = a.spos[j], y1 = a.spos[n + j], y2 = a.spos[2 * n + j];
            double dx = __dsub_rn(x[0], y0), dy = __dsub_rn(x[1], y1);
            if (pass == 0) {
              double dz = __dsub_rn(x[2], y2);
              bool self = own >= 0 ? (a.sorig[j] == own) : (dx == 0.0 && dy == 0.0 && dz == 0.0);
              if (self) { hit = true; type = Q_SELF; }
              else if (dist2_exact(dx, dy, dz) < a.rc2) { hit = true; type = Q_FREE; }
            } else {
              double dz = __dadd_rn(x[2], y2);
              if (dist2_exact(dx, dy, dz) < a.rc2) { hit = true; type = Q_IMAGE; }
            }
          }
          visit(hit, j, type);
        }
      }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_real(RealArgs a) {
  __shared__ int queue[kWarpsPerBlock][kQueue];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* qu = queue[wib];
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < a.n_tgt; w += nwarps) {
    double x[3];
    int64_t own, dst;
    if (a.tgt) {
      x[0] = a.tgt[w]; x[1] = a.tgt[a.n_tgt + w]; x[2] = a.tgt[2 * a.n_tgt + w];
      own = -1;
      dst = w;
    } else {  // targets are the sources, visited in cell order
      x[0] = a.spos[w]; x[1] = a.spos[a.n_src + w]; x[2] = a.spos[2 * a.n_src + w];
      own = a.sorig[w];
      dst = own;
    }
    double u[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
    for_candidates(a, x, own, lane, [&](bool hit, int j, int type) {
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) qu[cnt + __popc(m & ((1u << lane) - 1))] = j | (type << 29);
      cnt += __popc(m);
      __syncwarp();
      if (cnt >= 32) {
        int e = qu[lane];
        eval_pair(a, x, e & 0x1fffffff, e >> 29, u);
        __syncwarp();
        if (lane < cnt - 32) qu[lane] = qu[32 + lane];
        cnt -= 32;
        __syncwarp();
      }
    });
    if (lane < cnt) {
      int e = qu[lane];
      eval_pair(a, x, e & 0x1fffffff, e >> 29, u);
    }
    __syncwarp();
    for (int i = 0; i < 3; ++i)
      for (int off = 16; off > 0; off >>= 1) u[i] += __shfl_xor_sync(0xffffffffu, u[i], off);
    if (lane == 0) {
      for (int i = 0; i < 3; ++i) {
        double* o = a.out + i * a.n_tgt + dst;
        *o = a.add ? *o + u[i] : u[i];
      }
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_counts(RealArgs a, int32_t* na, int32_t* nb) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < a.n_tgt; w += nwarps) {
    double x[3];
    int64_t own, dst;
    if (a.tgt) {
      x[0] = a.tgt[w]; x[1] = a.tgt[a.n_tgt + w]; x[2] = a.tgt[2 * a.n_tgt + w];
      own = -1;
      dst = w;
    } else {
      x[0] = a.spos[w]; x[1] = a.spos[a.n_src + w]; x[2] = a.spos[2 * a.n_src + w];
      own = a.sorig[w];
      dst = own;
    }
    int cf = 0, ci = 0;
    for_candidates(a, x, own, lane, [&](bool hit, int j, int type) {
      unsigned mf = __ballot_sync(0xffffffffu, hit && type == Q_FREE);
      unsigned mi = __ballot_sync(0xffffffffu, hit && type == Q_IMAGE);
      cf += __popc(mf);
      ci += __popc(mi);
    });
    if (lane == 0) { na[dst] = cf; nb[dst] = ci; }
  }
}

static RealArgs make_args(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add) {
  RealArgs a;
  a.n_src = n_src;
  a.n_tgt = n_tgt;
  a.spos = p->ws.spos;
  a.sstr = p->ws.sstr;
  a.sorig = p->ws.val_a;
  a.cstart = p->ws.cell_start;
  a.tgt = tgt;
  a.out = out;
  a.add = add ? 1 : 0;
  a.mask = p->prm.kernel_mask;
  a.rowS = p->row_S; a.rowT = p->row_T; a.rowW = p->row_W;
  a.xi = p->prm.xi;
  a.rc = p->prm.rc;
  a.rc2 = p->prm.rc * p->prm.rc;
  for (int d = 0; d < 3; ++d) { a.inv_cell[d] = p->inv_cell[d]; a.ncell[d] = p->prm.ncell[d]; }
  return a;
}

static int warp_blocks(int64_t n_tgt) {
  int64_t b = (n_tgt + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (b > 152 * 64) b = 152 * 64;
  return b < 1 ? 1 : (int)b;
}

hse_status real_space(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                      cudaStream_t s) {
  if (n_tgt == 0) return HSE_OK;
  RealArgs a = make_args(p, n_src, n_tgt, tgt, out, add);
  k_real<<<warp_blocks(n_tgt), kWarpsPerBlock * 32, 0, s>>>(a);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_real");
}

hse_status neighbor_counts(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, int32_t* na, int32_t* nb,
                           cudaStream_t s) {
  if (n_tgt == 0) return HSE_OK;
  RealArgs a = make_args(p, n_src, n_tgt, tgt, nullptr, false);
  k_counts<<<warp_blocks(n_tgt), kWarpsPerBlock * 32, 0, s>>>(a, na, nb);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_counts");
}

}  // namespace hse
