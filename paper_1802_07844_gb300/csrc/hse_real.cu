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
// Every radial coefficient follows from four numbers of the pair distance
// rho (t = xi rho, c = 2 xi e^{-t^2}/sqrt(pi), E_r = erfc(t)/rho):
//   a1 = (E_r + c)/rho^2,  g2 = (3 a1 + 2 xi^2 c)/rho^2,  g3 = -(5 g2 + 4 xi^4 c)/rho^2
//   S^R: I (E_r - c) + r r a1          W^R: 2 a1 (tau x r)
//   T^R: -2 g2 r(r.g)(r.q) + 2 xi^2 c (g(r.q) + q(r.g) + r(g.q))
//   G_R: g0 = E_r, grad = -a1 r, grad grad = -a1 I + g2 r r, grad^3 with g2, g3.
//
// FP64 throughput (2 FMA/clk/SM on GB300) bounds this stage, so:
//  * erfc(t) = exp(-t^2) erfcx(t), erfcx by degree-8 polynomials on intervals
//    of width 1/8 (table from gen_special_tables.py), exp by Tang's
//    table-driven reduction and a degree-5 Taylor polynomial;
//  * candidates are screened in FP32 with a proven error margin; only those
//    within the margin of r_c take the exact FP64 test, so the accepted set
//    equals the FP64 rule ((dx*dx + dy*dy) + dz*dz < r_c^2, no contraction);
//  * with targets = sources each unordered pair is evaluated once (the radial
//    part is shared by both directions: r -> -r for free pairs,
//    rt -> (-rt1, -rt2, rt3) for image pairs); the partner's share is added
//    with FP64 atomics.
// Work split: one warp per target; passing candidates are compacted into a
// per-warp queue and evaluated 32 at a time, so FP64 instructions run full warps.
#include "hse_df64.cuh"
#include "hse_internal.cuh"
#include "special_tables.inc"

namespace hse {

__device__ const double d_erfcx_coef[HSE_ERFCX_NINT * (HSE_ERFCX_DEG + 1)] = {HSE_ERFCX_COEFS};
__device__ const double d_exp2_j64[64] = {HSE_EXP2_J64};

struct RealArgs {
  int64_t n_src, n_tgt;
  const double* spos;      // sorted sources, 3 x n_src
  const float* spos32;     // the same in FP32 (candidate screening; head of the FP32 pair)
  const float* spos32lo;   // tail: x - head in FP32
  const double* sstr;      // sorted strengths, rows x n_src
  const float* sstr32;     // the same in FP32
  const int32_t* sorig;    // sorted -> original source index
  const int32_t* cstart;   // cell starts
  const double* tgt;       // explicit targets (3 x n_tgt) or null (targets = sources)
  double* out;             // 3 x n_tgt in caller order (symmetric kernel: sorted order)
  float4* out4;            // symmetric FP32 kernel: partner sums in sorted order
  float4* out4lo;          // FP64 kernel's FP32 shell: rounding errors of the out4 sums (null: none)
  int add;                 // accumulate into out (asymmetric kernel)
  int mask, rowS, rowT, rowW;
  double xi, rc2, rc;
  float rc2_lo, rc2_hi;    // FP32 screening thresholds
  float cull2;             // rows of cells farther than sqrt(cull2) (> r_c by a safety margin) are skipped
  float cell_side[3];      // L_d / ncell_d
  float img64_2;           // FP32 path: image pairs closer than this (squared) are evaluated in FP64
  float far2;              // FP64 symmetric kernel: pairs with FP32 distance^2 >= far2 take the
                           // FP32 evaluation (0: none)
  float mid2;              // pairs with FP32 distance^2 in [mid2, far2) (or [mid2, r_c^2)) go to the
                           // double-float kernel k_real_mid (0: none)
  const float* sstr32lo;   // tails of the sorted strengths (double-float pairs with sstr32)
  float2 dxi, dxi2, dkc, dk2, dk4;  // double-float constants xi, xi^2, 2 xi/sqrt(pi), 2 xi^2, 4 xi^4
  double inv_cell[3];
  int ncell[3];
  // batched instances: instance of each sorted particle (null: one instance)
  // and cells per instance; an instance's cells follow each other in the list
  const int32_t* inst_of;
  int ncells_inst;
};

__device__ __forceinline__ int cell_base(const RealArgs& a, int64_t sorted_idx) {
  return a.inst_of ? a.inst_of[sorted_idx] * a.ncells_inst : 0;
}

// Q_FAR: FP32 outer shell, Q_MID: double-float middle band (flags on FREE / IMAGE)
enum { Q_FREE = 0, Q_IMAGE = 1, Q_SELF = 2, Q_FAR = 4, Q_MID = 8 };
constexpr int kWarpsPerBlock = 4;
constexpr int kQueue = 64;
constexpr int kErfcxN = HSE_ERFCX_NINT * (HSE_ERFCX_DEG + 1);
constexpr int kTabN = kErfcxN + 64 + HSE_ERFCX_NINT;  // erfcx intervals, 2^{j/64}, interval centres

// e^{-x} for 0 <= x (Tang's table-driven method, ACM TOMS 15, 1989):
// -x = m ln2/64 + r, |r| <= ln2/128, m = 64 n + j, e^{-x} = 2^n 2^{j/64} e^r,
// 2^{j/64} from the table t2 (shared memory), e^r from its degree-5 Taylor
// polynomial; 10 FP64 operations.
__device__ __forceinline__ double exp_neg(double x, const double* t2) {
  const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low word
  const double y = -x;
  const double tn = fma(y, k64Log2e, magic);
  const int m = __double2loint(tn);
  const double md = tn - magic;
  double r = fma(-md, kLn2By64Head, y);
  r = fma(-md, kLn2By64Tail, r);
  constexpr double C[6] = {HSE_EXP_TAYLOR5_COEFS};
  double p = C[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) p = fma(p, r, C[k]);
  const double v = t2[m & 63] * p;  // in [2^-1/128, 2^(1+1/128)): scaling by 2^n stays normal
  return __hiloint2double(__double2hiint(v) + (int)((unsigned)(m >> 6) << 20), __double2loint(v));
}

// erfcx(t) = e^{t^2} erfc(t) on [0, 12) from the interval table in shared memory
__device__ __forceinline__ double erfcx_tab(double t, float tf, const double* tab) {
  int k = (int)(tf * (float)HSE_ERFCX_INV_WIDTH);
  k = k < 0 ? 0 : (k > HSE_ERFCX_NINT - 1 ? HSE_ERFCX_NINT - 1 : k);
  const double* c = tab + k * (HSE_ERFCX_DEG + 1);
  // centre 2k + 1 of the interval in units of half its width, from the table
  // (an int -> double conversion would take an FP64 instruction)
  double u = fma(2.0 * HSE_ERFCX_INV_WIDTH, t, -tab[kErfcxN + 64 + k]);
  double p = c[HSE_ERFCX_DEG];
#pragma unroll
  for (int j = HSE_ERFCX_DEG - 1; j >= 0; --j) p = fma(p, u, c[j]);
  return p;
}

template <typename T>
struct Radial {
  T er, c, a1, g2, g3;  // erfc(t)/rho, 2 xi e^{-t^2}/sqrt(pi), a1, g2, g3
};

// FP32 approximation of a positive normal double within the float range, by
// truncation (integer operations only: the FP64 pipe, which bounds the
// real-space kernel, also executes double -> float conversions)
__device__ __forceinline__ float approx_float(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  return __uint_as_float(((hi - 0x38000000u) << 3) | (lo >> 29));
}

// FP64: own exp and erfcx table.  The table interval and the range tests use
// FP32 copies of t (t < 12 on the table; e^{-t^2} needs t < 26), so that the
// FP64 pipe only does the arithmetic.
__device__ __forceinline__ Radial<double> radial(double s, float sf, double xi, const double* tab, const float*,
                                                 bool need_g3) {
  Radial<double> R;
  double inv = rsqrt(s);
  double t = xi * s * inv;
  const float tf = __fmul_rn(approx_float(xi), sqrtf(sf));
  double E = tf < 26.0f ? exp_neg(t * t, tab + kErfcxN) : 0.0;
  double ec;
  if (tf < 11.99f) ec = E * erfcx_tab(t, tf, tab);
  else ec = erfc(t);  // beyond the table: only reached when xi r_c > 12
  double i2 = inv * inv;
  R.c = (2.0 / kSqrtPi) * xi * E;
  R.er = ec * inv;
  R.a1 = (R.er + R.c) * i2;
  R.g2 = i2 * fma(3.0, R.a1, 2.0 * xi * xi * R.c);
  R.g3 = need_g3 ? -i2 * fma(5.0, R.g2, 4.0 * xi * xi * xi * xi * R.c) : 0.0;
  return R;
}

// erfcx(t) in FP32 from the float copy of the interval table (t in [0, 12));
// t - c_k is exact (c_k = (2k + 1)/16 has few bits and lies within a factor 2
// of t), so u carries only t's own rounding
__device__ __forceinline__ float erfcx_tab32(float t, const float* tab) {
  int k = (int)(t * (float)HSE_ERFCX_INV_WIDTH);
  k = k < 0 ? 0 : (k > HSE_ERFCX_NINT - 1 ? HSE_ERFCX_NINT - 1 : k);
  const float* c = tab + k * (HSE_ERFCX_DEG + 1);
  const float u = (t - (float)(2 * k + 1) * (0.5f / HSE_ERFCX_INV_WIDTH)) * (2.0f * HSE_ERFCX_INV_WIDTH);
  float p = c[HSE_ERFCX_DEG];
#pragma unroll
  for (int j = HSE_ERFCX_DEG - 1; j >= 0; --j) p = fmaf(p, u, c[j]);
  return p;
}

// FP32 (mixed precision): the FP32 pipe is ~60x the FP64 one on GB300;
// erfc(t) = e^{-t^2} erfcx(t) with erfcx from the FP32 table tab32
__device__ __forceinline__ Radial<float> radial(float s, float, float xi, const double*, const float* tab32,
                                                bool need_g3) {
  Radial<float> R;
  float inv = rsqrtf(s);
  float t = xi * s * inv;
  float E = expf(-t * t);
  float ec = t < 11.99f ? E * erfcx_tab32(t, tab32) : erfcf(t);
  float i2 = inv * inv;
  R.c = (float)(2.0 / kSqrtPi) * xi * E;
  R.er = ec * inv;
  R.a1 = (R.er + R.c) * i2;
  R.g2 = i2 * fmaf(3.0f, R.a1, 2.0f * xi * xi * R.c);
  R.g3 = need_g3 ? -i2 * fmaf(5.0f, R.g2, 4.0f * xi * xi * xi * xi * R.c) : 0.0f;
  return R;
}

// s + e == a + b exactly (Knuth's two-sum; no ordering of |a|, |b| needed)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Radial coefficients of an outer-shell pair of an FP64 plan, in FP32 but with
// the Gaussian's exponent carried to ~44 bits.  e^{-t^2} and erfc(t) change by
// 2 t^2 times the relative error of rho^2 (t = xi rho, 2 t^2 ~ 15 at the
// shell's inner edge), so the plain FP32 form above loses ~1.5e-6 per term;
// here rho^2 = sum_d (dh_d + dl_d)^2 is formed with exact products and sums,
// t^2 = xi^2 rho^2 = zh + zl with the product's error kept, e^{-t^2} =
// e^{-zh} (1 - zl), and erfc(t) = e^{-t^2} erfcx(t), where erfcx varies slowly
// (its relative error stays that of t).  ~1e-7 per term.
__device__ __forceinline__ Radial<float> radial_shell(const float* dh, const float* dl, float xi, float xi2h,
                                                      float xi2l, bool need_g3, const float* tab32) {
  float p[3], q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    p[d] = __fmul_rn(dh[d], dh[d]);
    q[d] = fmaf(dh[d], dh[d], -p[d]);
  }
  float s1, e1, sh, e2;
  two_sum(p[0], p[1], s1, e1);
  two_sum(s1, p[2], sh, e2);
  const float cross = fmaf(dh[0], dl[0], fmaf(dh[1], dl[1], __fmul_rn(dh[2], dl[2])));
  const float sl = __fadd_rn(__fadd_rn(e1, e2), fmaf(2.0f, cross, __fadd_rn(q[0], __fadd_rn(q[1], q[2]))));
  const float zh = __fmul_rn(xi2h, sh);
  const float zl = __fadd_rn(fmaf(xi2h, sh, -zh), fmaf(xi2h, sl, __fmul_rn(xi2l, sh)));
  const float E = __fmul_rn(expf(-zh), __fsub_rn(1.0f, zl));
  const float s = __fadd_rn(sh, sl);
  const float inv = rsqrtf(s);
  const float t = xi * s * inv;
  Radial<float> R;
  const float i2 = inv * inv;
  R.c = (float)(2.0 / kSqrtPi) * xi * E;
  R.er = E * erfcx_tab32(t, tab32) * inv;
  R.a1 = (R.er + R.c) * i2;
  R.g2 = i2 * fmaf(3.0f, R.a1, 2.0f * xi * xi * R.c);
  R.g3 = need_g3 ? -i2 * fmaf(5.0f, R.g2, 4.0f * xi * xi * xi * xi * R.c) : 0.0f;
  return R;
}

template <typename T>
struct Src {
  T f[3], g[3], q[3], tau[3];
};

// KM: the kernel bits known at compile time (0: read them from a.mask)
template <typename T, int KM = 0>
__device__ __forceinline__ void load_src(const RealArgs& a, const T* str, int64_t j, Src<T>& s) {
  const int64_t n = a.n_src;
  const int mask = KM ? KM : a.mask;
#pragma unroll
  for (int i = 0; i < 3; ++i) { s.f[i] = 0; s.g[i] = 0; s.q[i] = 0; s.tau[i] = 0; }
  if (mask & HSE_STOKESLET)
    for (int i = 0; i < 3; ++i) s.f[i] = str[(a.rowS + i) * n + j];
  if (mask & HSE_STRESSLET)
    for (int i = 0; i < 3; ++i) { s.g[i] = str[(a.rowT + i) * n + j]; s.q[i] = str[(a.rowT + 3 + i) * n + j]; }
  if (mask & HSE_ROTLET)
    for (int i = 0; i < 3; ++i) s.tau[i] = str[(a.rowW + i) * n + j];
}

// free-space contribution of source s at r = x - y (sgn_odd = -1 gives the
// contribution at the source's position from the target's strengths when the
// roles are swapped: S is even in r, T and W odd).  Written as chains of
// multiply-adds into u: the FP64 pipe bounds the real-space kernel, and an
// unfused product and sum take two of its instructions.
template <typename T>
__device__ __forceinline__ void add_free(int mask, const Radial<T>& R, const T* r, const Src<T>& s, T xi, T sgn_odd,
                                         T* u) {
  if (mask & HSE_STOKESLET) {
    // (er - c) f + a1 r (r.f)
    const T sa = R.er - R.c;
    const T rf = fma(r[2], s.f[2], fma(r[1], s.f[1], r[0] * s.f[0]));
    const T arf = R.a1 * rf;
#pragma unroll
    for (int i = 0; i < 3; ++i) u[i] = fma(arf, r[i], fma(sa, s.f[i], u[i]));
  }
  if (mask & HSE_STRESSLET) {
    // ta r (r.g)(r.q) + tb (g (r.q) + q (r.g) + r (g.q)), ta = -2 g2, tb = 2 xi^2 c,
    // as coefficients of r, g, q
    const T tb = (sgn_odd * 2 * xi * xi) * R.c;
    const T rg = fma(r[2], s.g[2], fma(r[1], s.g[1], r[0] * s.g[0]));
    const T rq = fma(r[2], s.q[2], fma(r[1], s.q[1], r[0] * s.q[0]));
    const T gq = fma(s.g[2], s.q[2], fma(s.g[1], s.q[1], s.g[0] * s.q[0]));
    const T cr = fma((sgn_odd * -2) * R.g2 * rg, rq, tb * gq), cg = tb * rq, cq = tb * rg;
#pragma unroll
    for (int i = 0; i < 3; ++i) u[i] = fma(cr, r[i], fma(cg, s.g[i], fma(cq, s.q[i], u[i])));
  }
  if (mask & HSE_ROTLET) {
    // 2 a1 tau x r
    const T wa = (sgn_odd * 2) * R.a1;
    const T w0 = wa * s.tau[0], w1 = wa * s.tau[1], w2 = wa * s.tau[2];
    u[0] = fma(w1, r[2], fma(-w2, r[1], u[0]));
    u[1] = fma(w2, r[0], fma(-w0, r[2], u[1]));
    u[2] = fma(w0, r[1], fma(-w1, r[0], u[2]));
  }
}

// image contribution at a target of height x3 from source s of height h,
// rt = x - y^I.  The wall corrections' gradient is collected as
// grad(phi) = ar r + gv (one coefficient of r shared by every kernel, plus the
// strength-vector terms), which the final u -= x3 grad(phi) applies once;
// phi, ar and gv are accumulated at half their values (the kernels'
// corrections carry factors 2 and 4) and doubled once.
template <typename T>
__device__ __forceinline__ void add_image(int mask, const Radial<T>& R, const T* r, T h, T x3, const Src<T>& s, T xi,
                                          T* u) {
  const T a1 = R.a1, g2 = R.g2;  // g1 = -a1 (gradient coefficient of G_R)
  T phi = 0, ar = 0, gv0 = 0, gv1 = 0, gv2 = 0;  // halves
  if (mask & HSE_STOKESLET) {
    // -S^R(rt) f^I, f^I = (f1, f2, -f3)
    const T sa = R.er - R.c;
    const T rf = fma(-r[2], s.f[2], fma(r[1], s.f[1], r[0] * s.f[0]));  // rt . f^I
    const T arf = a1 * rf;
    u[0] = fma(-arf, r[0], fma(-sa, s.f[0], u[0]));
    u[1] = fma(-arf, r[1], fma(-sa, s.f[1], u[1]));
    u[2] = fma(-arf, r[2], fma(sa, s.f[2], u[2]));
    // phi_S = 2 (-f3 G_R - h grad G_R . f^I) = 2 (h a1 rf - f3 er),
    // grad phi_S = 2 (f3 a1 r + h a1 f^I - h g2 rf r)
    const T ha = h * a1;
    phi = fma(ha, rf, -(s.f[2] * R.er));
    ar = fma(-(h * g2), rf, s.f[2] * a1);
    gv0 = ha * s.f[0];
    gv1 = ha * s.f[1];
    gv2 = -ha * s.f[2];
  }
  if (mask & HSE_STRESSLET) {
    // -T^R(rt)(g^I q^I)
    const T tb = (2 * xi * xi) * R.c;
    const T gI2 = -s.g[2], qI2 = -s.q[2];
    const T rg = fma(r[2], gI2, fma(r[1], s.g[1], r[0] * s.g[0]));
    const T rq = fma(r[2], qI2, fma(r[1], s.q[1], r[0] * s.q[0]));
    const T gq = fma(gI2, qI2, fma(s.g[1], s.q[1], s.g[0] * s.q[0]));
    const T g2rg = g2 * rg;
    const T cr = fma(-2 * g2rg, rq, tb * gq), cg = tb * rq, cq = tb * rg;
    u[0] = fma(-cr, r[0], fma(-cg, s.g[0], fma(-cq, s.q[0], u[0])));
    u[1] = fma(-cr, r[1], fma(-cg, s.g[1], fma(-cq, s.q[1], u[1])));
    u[2] = fma(-cr, r[2], fma(-cg, gI2, fma(-cq, qI2, u[2])));
    // phi_T = 4 (gI.qI) d3 G_R - 4 h gI.(grad grad G_R) qI; halves:
    //   phi/2 = -2 gq a1 r3 - 2 h (g2 rg rq - a1 gq)
    //   (grad phi)/2 = 2 gq (g2 r3 r - a1 e3) - 2 h (g2 (gq r + gI rq + qI rg) + g3 rg rq r)
    const T gq2 = gq + gq, h2 = h + h;
    const T ga = gq2 * a1;
    phi = fma(-ga, r[2], fma(-h2, fma(g2rg, rq, -a1 * gq), phi));
    ar = fma(gq2 * g2, r[2], fma(-h2, fma(g2, gq, R.g3 * rg * rq), ar));
    const T hg = -h2 * g2;
    const T dg = hg * rq, dq = hg * rg;
    gv0 = fma(dg, s.g[0], fma(dq, s.q[0], gv0));
    gv1 = fma(dg, s.g[1], fma(dq, s.q[1], gv1));
    gv2 = fma(dg, gI2, fma(dq, qI2, gv2 - ga));
  }
  if (mask & HSE_ROTLET) {
    // +W^R(rt) tau^I = 2 a1 tau^I x rt, tau^I = (tau1, tau2, -tau3)
    const T wa = 2 * a1;
    const T w0 = wa * s.tau[0], w1 = wa * s.tau[1], w2 = -wa * s.tau[2];
    u[0] = fma(w1, r[2], fma(-w2, r[1], u[0]));
    u[1] = fma(w2, r[0], fma(-w0, r[2], u[1]));
    u[2] = fma(w0, r[1], fma(-w1, r[0], u[2]));
    // phi_W = 4 g1 (rt.v), grad phi_W = 4 (g1 v + g2 rt (rt.v)), v = (-tau2, tau1, 0);
    // halves: -wa rv, wa... : g1 v / 2 * 4 = -wa v
    const T rv = fma(r[1], s.tau[0], -r[0] * s.tau[1]);
    phi = fma(-wa, rv, phi);
    ar = fma(g2 + g2, rv, ar);
    gv0 += w1;   // -wa v0 = wa tau2
    gv1 -= w0;   // -wa v1 = -wa tau1
  }
  // u -= x3 grad(phi) = x3 (ar r + gv); u3 += phi (both from their halves)
  const T xd = x3 + x3;
  const T xa = xd * ar;
  u[0] = fma(-xa, r[0], fma(-xd, gv0, u[0]));
  u[1] = fma(-xa, r[1], fma(-xd, gv1, u[1]));
  u[2] = fma(-xa, r[2], fma(-xd, gv2, u[2] + (phi + phi)));
}

// Target position in the arithmetic type of the pair evaluation.  FP32 keeps
// a head/tail pair so that differences of nearby points stay accurate.
struct TgtPos {
  double d[3];
  float h[3], l[3];
};

// separation to sorted source j (free: x - y; image: x - y^I) and the
// source height, in the pair arithmetic
__device__ __forceinline__ void pair_vec(const RealArgs& a, const TgtPos& x, int64_t j, bool img, double* r,
                                         double* h) {
  const int64_t n = a.n_src;
  double y2 = a.spos[2 * n + j];
  r[0] = x.d[0] - a.spos[j];
  r[1] = x.d[1] - a.spos[n + j];
  r[2] = img ? x.d[2] + y2 : x.d[2] - y2;
  *h = y2;
}
__device__ __forceinline__ void pair_vec(const RealArgs& a, const TgtPos& x, int64_t j, bool img, float* r,
                                         float* h) {
  const int64_t n = a.n_src;
  const float* H = a.spos32;
  const float* L = a.spos32lo;
  r[0] = (x.h[0] - H[j]) + (x.l[0] - L[j]);
  r[1] = (x.h[1] - H[n + j]) + (x.l[1] - L[n + j]);
  r[2] = img ? (x.h[2] + H[2 * n + j]) + (x.l[2] + L[2 * n + j]) : (x.h[2] - H[2 * n + j]) + (x.l[2] - L[2 * n + j]);
  *h = H[2 * n + j] + L[2 * n + j];
}
// The same separation as head + tail per component with the heads' difference
// split exactly (two-sum): r_d = dh_d + dl_d to ~2^-24 of the tails, so that
// the shell's distance^2 keeps ~44 bits; r (FP32) is their rounded sum.
__device__ __forceinline__ void pair_vec_split(const RealArgs& a, const TgtPos& x, int64_t j, bool img, float* dh,
                                               float* dl, float* r, float* h) {
  const int64_t n = a.n_src;
  const float* H = a.spos32;
  const float* L = a.spos32lo;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const bool sum = img && d == 2;
    const float yh = H[d * n + j], yl = L[d * n + j];
    float e;
    two_sum(x.h[d], sum ? yh : -yh, dh[d], e);
    dl[d] = __fadd_rn(e, sum ? __fadd_rn(x.l[d], yl) : __fsub_rn(x.l[d], yl));
    r[d] = __fadd_rn(dh[d], dl[d]);
  }
  *h = H[2 * n + j] + L[2 * n + j];
}

// squared length in a fixed operation order (the close-image classification
// must be identical in the kernels that skip and that take those pairs)
__device__ __forceinline__ float sq3(const float* r) {
  return __fadd_rn(__fadd_rn(__fmul_rn(r[0], r[0]), __fmul_rn(r[1], r[1])), __fmul_rn(r[2], r[2]));
}
__device__ __forceinline__ double sq3(const double* r) { return r[0] * r[0] + r[1] * r[1] + r[2] * r[2]; }

template <typename T> __device__ __forceinline__ const T* strengths_of(const RealArgs& a);
template <> __device__ __forceinline__ const double* strengths_of<double>(const RealArgs& a) { return a.sstr; }
template <> __device__ __forceinline__ const float* strengths_of<float>(const RealArgs& a) { return a.sstr32; }

// Candidate scan: cells around the target (free pairs) and the wall-layer
// cells below its image (image pairs), 32 candidates per step, with the
// FP32 screen and the exact FP64 decision for the rest.  j_min bounds the
// sorted source index from below (half list of the symmetric kernel).
// MIDB: classify the double-float band (Q_MID); compiled out otherwise
template <bool MIDB = false, typename Visit>
__device__ __forceinline__ void for_candidates(const RealArgs& a, const double* x, const float* xf, int64_t own,
                                               int lane, int free_min, int img_min, int base, Visit&& visit) {
  int cx = cell_coord(x[0], a.inv_cell[0], a.ncell[0]);
  int cy = cell_coord(x[1], a.inv_cell[1], a.ncell[1]);
  int cz = cell_coord(x[2], a.inv_cell[2], a.ncell[2]);
  const int64_t n = a.n_src;
  const int nx = a.ncell[0], ny = a.ncell[1], nz = a.ncell[2];
  // images only reach targets with x3 < rc, and come from sources with y3 < rc - x3
  // (none in free space)
  bool want_img = x[2] < a.rc && !(a.mask & HSE_FREE_SPACE);
  int czi_hi = want_img ? cell_coord(a.rc - x[2], a.inv_cell[2], nz) : -1;
  for (int pass = 0; pass < 2; ++pass) {
    constexpr int R = kCellReach;
    int z0 = pass == 0 ? (cz > R - 1 ? cz - R : 0) : 0;
    int z1 = pass == 0 ? (cz < nz - R ? cz + R : nz - 1) : czi_hi;
    int jmin = pass == 0 ? free_min : img_min;
    for (int iz = z0; iz <= z1; ++iz) {
      // rows of cells whose box lies beyond the cut-off are skipped, and each
      // row's end cells likewise (box distances in FP32 against a cut-off
      // widened by 1e-5 L, so no pair within r_c is lost); the image pass
      // measures to the mirrored layer
      const float zl = (float)iz * a.cell_side[2], zh = zl + a.cell_side[2];
      const float dzc = pass == 0 ? fmaxf(0.f, fmaxf(zl - xf[2], xf[2] - zh)) : xf[2] + zl;
      const float rz = a.cull2 - dzc * dzc;
      if (!(rz > 0.f)) continue;
      for (int iy = (cy > R - 1 ? cy - R : 0); iy <= (cy < ny - R ? cy + R : ny - 1); ++iy) {
        const float yl = (float)iy * a.cell_side[1], yh = yl + a.cell_side[1];
        const float dyc = fmaxf(0.f, fmaxf(yl - xf[1], xf[1] - yh));
        const float rem = rz - dyc * dyc;
        if (!(rem > 0.f)) continue;
        // x-neighbours are contiguous in the cell numbering
        int xa = cx > R - 1 ? cx - R : 0, xb = cx < nx - R ? cx + R : nx - 1;
        while (xa < xb) {
          const float d = xf[0] - (float)(xa + 1) * a.cell_side[0];
          if (d > 0.f && d * d >= rem) ++xa;
          else break;
        }
        while (xb > xa) {
          const float d = (float)xb * a.cell_side[0] - xf[0];
          if (d > 0.f && d * d >= rem) --xb;
          else break;
        }
        int c0 = base + (iz * ny + iy) * nx + xa;
        int s0 = a.cstart[c0], s1 = a.cstart[c0 + (xb - xa) + 1];
        if (s0 < jmin) s0 = jmin;
        for (int base = s0; base < s1; base += 32) {
          int j = base + lane;
          int type = 0;
          bool hit = false;
          if (j < s1) {
            float dxf = xf[0] - a.spos32[j], dyf = xf[1] - a.spos32[n + j];
            float dzf = pass == 0 ? xf[2] - a.spos32[2 * n + j] : xf[2] + a.spos32[2 * n + j];
            float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
            bool self = pass == 0 && own >= 0 && j == own;
            if (self) {
              hit = true;
              type = Q_SELF;
            } else if (d2f < a.rc2_hi) {
              bool in = d2f < a.rc2_lo;
              if (!in || (pass == 0 && own < 0 && d2f == 0.0f)) {  // exact FP64 decision / zero test
                double dx = __dsub_rn(x[0], a.spos[j]), dy = __dsub_rn(x[1], a.spos[n + j]);
                double dz = pass == 0 ? __dsub_rn(x[2], a.spos[2 * n + j]) : __dadd_rn(x[2], a.spos[2 * n + j]);
                if (pass == 0 && own < 0 && dx == 0.0 && dy == 0.0 && dz == 0.0) {
                  hit = true;
                  type = Q_SELF;
                  in = false;
                } else {
                  in = dist2_exact(dx, dy, dz) < a.rc2;
                }
              }
              if (in) {
                hit = true;
                // FP32 for the outer shell, unless an end point is within rho/64
                // of the wall: there the free and image contributions of a
                // source cancel to O(height/rho), which would amplify rounding
                const float hmin = fminf(xf[2], a.spos32[2 * n + j]);
                const bool wall = 4096.0f * hmin * hmin < d2f;
                const bool far = a.far2 > 0.0f && d2f >= a.far2 && !wall;
                // double-float band [rcmid, rc64) (same FP32 decision in both kernels)
                const bool mid = MIDB && !far && d2f >= a.mid2 && !wall;
                type = (pass == 0 ? Q_FREE : Q_IMAGE) | (far ? Q_FAR : 0) | (mid ? Q_MID : 0);
              }
            }
          }
          visit(hit, j, type);
        }
      }
    }
  }
}

__device__ __forceinline__ void load_table(double* tab) {
  for (int i = threadIdx.x; i < kTabN; i += blockDim.x)
    tab[i] = i < kErfcxN ? d_erfcx_coef[i] : i < kErfcxN + 64 ? d_exp2_j64[i - kErfcxN] : (double)(2 * (i - kErfcxN - 64) + 1);
  __syncthreads();
}

// Asymmetric kernel: explicit targets (or any target set), every ordered pair.
// T is the pair arithmetic (double, or float with HSE_MIXED); sums over a
// lane's pairs are kept in T and reduced across the warp in FP64.
template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_real(RealArgs a) {
  __shared__ int queue[kWarpsPerBlock][kQueue];
  __shared__ double tab[kTabN];
  __shared__ float tab32[kErfcxN];  // erfcx table in FP32 (FP32 pairs)
  for (int i = threadIdx.x; i < kErfcxN; i += blockDim.x) tab32[i] = (float)d_erfcx_coef[i];
  load_table(tab);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* qu = queue[wib];
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const bool need_g3 = a.mask & HSE_STRESSLET;
  const T xi = (T)a.xi;
  const T* str = strengths_of<T>(a);
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < a.n_tgt; w += nwarps) {
    TgtPos x;
    int64_t own, dst;
    if (a.tgt) {
      for (int d = 0; d < 3; ++d) x.d[d] = a.tgt[d * a.n_tgt + w];
      own = -1;
      dst = w;
    } else {  // targets are the sources, visited in cell order
      for (int d = 0; d < 3; ++d) x.d[d] = a.spos[d * a.n_src + w];
      own = w;
      dst = a.sorig[w];
    }
    for (int d = 0; d < 3; ++d) {
      x.h[d] = (float)x.d[d];
      x.l[d] = (float)(x.d[d] - (double)x.h[d]);
    }
    const T x3 = sizeof(T) == 8 ? (T)x.d[2] : (T)(x.h[2] + x.l[2]);
    T u[3] = {0, 0, 0};
    double uself[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
    auto run = [&](int e) {
      int j = e & 0x1fffffff, type = e >> 29;
      if (type == Q_SELF) {
        if (a.mask & HSE_STOKESLET)
          for (int i = 0; i < 3; ++i) uself[i] += -4.0 * a.xi / kSqrtPi * a.sstr[(a.rowS + i) * a.n_src + j];
        return;
      }
      Src<T> s;
      load_src<T>(a, str, j, s);
      T r[3], h;
      pair_vec(a, x, j, type == Q_IMAGE, r, &h);
      T sd = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      if (sizeof(T) == 4 && type == Q_IMAGE && (float)sq3(r) < a.img64_2) {
        // Close image pairs of near-wall targets: the image kernel and the wall
        // corrections cancel to O(x3/rho) (exactly at leading order for a
        // target's own image, rho = 2 x3), so FP32 would leave noise of
        // eps/rho^2; these few pairs use the FP64 evaluation.
        Src<double> sdbl;
        load_src<double>(a, a.sstr, j, sdbl);
        double rd[3], hd;
        pair_vec(a, x, j, true, rd, &hd);
        double s2 = rd[0] * rd[0] + rd[1] * rd[1] + rd[2] * rd[2];
        Radial<double> Rd = radial(s2, approx_float(s2), a.xi, tab, tab32, need_g3);
        add_image<double>(a.mask, Rd, rd, hd, x.d[2], sdbl, a.xi, uself);
        return;
      }
      Radial<T> R = radial(sd, sizeof(T) == 8 ? approx_float((double)sd) : (float)sd, xi, tab, tab32, need_g3);
      if (type == Q_FREE) add_free<T>(a.mask, R, r, s, xi, (T)1, u);
      else add_image<T>(a.mask, R, r, h, x3, s, xi, u);
    };
    float xf[3] = {x.h[0], x.h[1], x.h[2]};
    const int base = a.tgt ? 0 : cell_base(a, w);
    for_candidates(a, x.d, xf, own, lane, 0, 0, base, [&](bool hit, int j, int type) {
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) qu[cnt + __popc(m & ((1u << lane) - 1))] = j | (type << 29);
      cnt += __popc(m);
      __syncwarp();
      if (cnt >= 32) {
        run(qu[lane]);
        __syncwarp();
        if (lane < cnt - 32) qu[lane] = qu[32 + lane];
        cnt -= 32;
        __syncwarp();
      }
    });
    if (lane < cnt) run(qu[lane]);
    __syncwarp();
    double ud[3];
    for (int i = 0; i < 3; ++i) {
      ud[i] = (double)u[i] + uself[i];
      for (int off = 16; off > 0; off >>= 1) ud[i] += __shfl_xor_sync(0xffffffffu, ud[i], off);
    }
    if (lane == 0) {
      for (int i = 0; i < 3; ++i) {
        double* o = a.out + i * a.n_tgt + dst;
        *o = a.add ? *o + ud[i] : ud[i];
      }
    }
  }
}

// Symmetric kernel (targets = sources): warp of sorted target p takes the
// pairs with sorted source index j > p (free) and j >= p (image, j = p is the
// target's own image); the partner's share goes out by FP64 atomicAdd into the
// sorted-order sums a.out (zeroed before the launch; neighbours sit at nearby
// addresses), which k_unsort then writes in caller order.
// FP64 pairs arithmetic with a.far2 > 0: pairs in the outer shell (FP32
// distance^2 >= far2) are queued separately and evaluated in FP32 -- their
// screened kernels are small, so FP32 rounding stays far below the truncation
// error -- with the partner's share sent by one float4 atomic into a.out4.
// Resident blocks per SM the FP64 symmetric kernel is compiled for: 4 (128
// registers) where the pair arithmetic fits without spilling, which keeps 16
// warps per SM issuing to the FP64 pipe; the masks with two strength tensors need
// more registers (3 blocks, up to 170).  The FP32 kernel is latency-bound
// (candidate scans and float4 atomics): 6 blocks (80 registers, 24 warps per
// SM) where it fits without spilling, 5 for S+T and 4 for S+T+W; measured on
// the N = 1M S+W workload at tol 1e-5, 21.7 ms at 4 blocks (109 registers)
// against 18.9 ms at 6.
template <typename T, int KM>
constexpr int real_min_blocks() {
  return sizeof(T) == 8 ? (KM != 3 && KM != 6 && KM != 7 ? 4 : 3) : (KM == 7 ? 4 : (KM == 3 ? 5 : 6));
}

// MID: the plan has a double-float band, whose pairs k_real_mid evaluates
template <typename T, int KM, bool MID>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, real_min_blocks<T, KM>()) k_real_sym(RealArgs a) {
  __shared__ int queue[kWarpsPerBlock][kQueue];
  __shared__ int queue_far[kWarpsPerBlock][kQueue];
  __shared__ double tab[kTabN];
  __shared__ float tab32[kErfcxN];  // erfcx table in FP32 (shell and FP32 pairs)
  for (int i = threadIdx.x; i < kErfcxN; i += blockDim.x) tab32[i] = (float)d_erfcx_coef[i];
  load_table(tab);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* qu = queue[wib];
  int* qf = queue_far[wib];
  const int64_t n = a.n_src;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const bool need_g3 = KM & HSE_STRESSLET;
  const T xi = (T)a.xi;
  const float xi32 = (float)a.xi;
  const float xi2h = (float)(a.xi * a.xi), xi2l = (float)(a.xi * a.xi - (double)xi2h);
  const T* str = strengths_of<T>(a);
  // Compensated FP32 partner sums of the shell: a source receives thousands of
  // float4 atomics, whose rounding would grow with their number.  atomicAdd
  // returns the old value, so the rounding error of each add is recovered
  // exactly by a two-sum (the atomic rounds to nearest) and added to out4lo.
  // The two-sum of a lane's last atomic is taken at its next shell batch, so
  // the atomic's round trip overlaps the scan.
  float4 pend_old = make_float4(0.f, 0.f, 0.f, 0.f), pend_v = pend_old;
  int64_t pend_j = -1;
  auto flush_pending = [&]() {
    if (pend_j >= 0) {
      float s0, e0, e1, e2;
      two_sum(pend_old.x, pend_v.x, s0, e0);
      two_sum(pend_old.y, pend_v.y, s0, e1);
      two_sum(pend_old.z, pend_v.z, s0, e2);
      atomicAdd(a.out4lo + pend_j, make_float4(e0, e1, e2, 0.f));
      pend_j = -1;
    }
  };
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < n; w += nwarps) {
    TgtPos x;
    for (int d = 0; d < 3; ++d) {
      x.d[d] = a.spos[d * n + w];
      x.h[d] = a.spos32[d * n + w];
      x.l[d] = a.spos32lo[d * n + w];
    }
    const T x3 = sizeof(T) == 8 ? (T)x.d[2] : (T)(x.h[2] + x.l[2]);
    const float x3f = x.h[2] + x.l[2];
    Src<T> sp;
    load_src<T, KM>(a, str, w, sp);
    T u[3] = {0, 0, 0};
    float uf[3] = {0.f, 0.f, 0.f}, ufl[3] = {0.f, 0.f, 0.f};  // FP32 shell pairs, compensated
    double uself[3] = {0.0, 0.0, 0.0};
    if (lane == 0 && (KM & HSE_STOKESLET))
      for (int i = 0; i < 3; ++i) uself[i] = -4.0 * a.xi / kSqrtPi * a.sstr[(a.rowS + i) * n + w];
    int cnt = 0, cntf = 0;
    auto partner_add = [&](int64_t j, double v0, double v1, double v2) {
      if (sizeof(T) == 4) atomicAdd(a.out4 + j, make_float4((float)v0, (float)v1, (float)v2, 0.f));
      else {
        atomicAdd(a.out + j, v0);
        atomicAdd(a.out + n + j, v1);
        atomicAdd(a.out + 2 * n + j, v2);
      }
    };
    auto run = [&](int e) {
      int j = e & 0x1fffffff, type = e >> 29;
      Src<T> s;
      load_src<T, KM>(a, str, j, s);
      T r[3], h;
      pair_vec(a, x, j, type == Q_IMAGE, r, &h);
      T sd = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      // close image pairs are left to k_close_images (FP64), see there
      if (sizeof(T) == 4 && type == Q_IMAGE && (float)sq3(r) < a.img64_2) return;
      Radial<T> R = radial(sd, sizeof(T) == 8 ? approx_float((double)sd) : (float)sd, xi, tab, tab32, need_g3);
      T v[3] = {0, 0, 0};
      if (type == Q_FREE) {
        add_free<T>(KM, R, r, s, xi, (T)1, u);
        add_free<T>(KM, R, r, sp, xi, (T)-1, v);  // at y_j from the target's strengths, r -> -r
      } else {
        add_image<T>(KM, R, r, h, x3, s, xi, u);
        if (j != w) {
          T rp[3] = {-r[0], -r[1], r[2]};  // y_j - x^I
          add_image<T>(KM, R, rp, x3, h, sp, xi, v);
        }
      }
      if (type == Q_FREE || j != w) partner_add(j, v[0], v[1], v[2]);
    };
    // FP32 evaluation of an outer-shell pair (only queued when T is double)
    auto run_far = [&](int e) {
      int j = e & 0x1fffffff, type = e >> 29;
      Src<float> s, spf;
      load_src<float, KM>(a, a.sstr32, j, s);
      load_src<float, KM>(a, a.sstr32, w, spf);
      float r[3], dh[3], dl[3], h;
      pair_vec_split(a, x, j, type == Q_IMAGE, dh, dl, r, &h);
      Radial<float> R = radial_shell(dh, dl, xi32, xi2h, xi2l, need_g3, tab32);
      float v[3] = {0.f, 0.f, 0.f}, t[3] = {0.f, 0.f, 0.f};
      if (type == Q_FREE) {
        add_free<float>(KM, R, r, s, xi32, 1.f, t);
        add_free<float>(KM, R, r, spf, xi32, -1.f, v);
      } else {
        add_image<float>(KM, R, r, h, x3f, s, xi32, t);
        if (j != w) {
          float rp[3] = {-r[0], -r[1], r[2]};
          add_image<float>(KM, R, rp, x3f, h, spf, xi32, v);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float s_, e_;
        two_sum(uf[i], t[i], s_, e_);
        uf[i] = s_;
        ufl[i] += e_;
      }
      flush_pending();
      if (type == Q_FREE || j != w) {
        pend_v = make_float4(v[0], v[1], v[2], 0.f);
        pend_old = atomicAdd(a.out4 + j, pend_v);
        pend_j = j;
      }
    };
    float xf[3] = {x.h[0], x.h[1], x.h[2]};
    for_candidates<MID>(a, x.d, xf, w, lane, (int)w + 1, (int)w, cell_base(a, w), [&](bool hit, int j, int type) {
      // pairs of the double-float band are left to k_real_mid
      const bool use = hit && type != Q_SELF && !(MID && (type & Q_MID));
      const bool far = use && (type & Q_FAR);
      const int t = type & 1;
      unsigned m = __ballot_sync(0xffffffffu, use && !far);
      unsigned mf = __ballot_sync(0xffffffffu, far);
      const unsigned below = (1u << lane) - 1;
      if (use && !far) qu[cnt + __popc(m & below)] = j | (t << 29);
      if (far) qf[cntf + __popc(mf & below)] = j | (t << 29);
      cnt += __popc(m);
      cntf += __popc(mf);
      __syncwarp();
      if (cnt >= 32) {
        run(qu[lane]);
        __syncwarp();
        if (lane < cnt - 32) qu[lane] = qu[32 + lane];
        cnt -= 32;
        __syncwarp();
      }
      if constexpr (sizeof(T) == 8) {  // the FP32 path never queues shell pairs
        if (cntf >= 32) {
          run_far(qf[lane]);
          __syncwarp();
          if (lane < cntf - 32) qf[lane] = qf[32 + lane];
          cntf -= 32;
          __syncwarp();
        }
      }
    });
    if (lane < cnt) run(qu[lane]);
    if constexpr (sizeof(T) == 8)
      if (lane < cntf) run_far(qf[lane]);
    __syncwarp();
    double ud[3];
    for (int i = 0; i < 3; ++i) {
      ud[i] = (double)u[i] + ((double)uf[i] + (double)ufl[i]) + uself[i];
      for (int off = 16; off > 0; off >>= 1) ud[i] += __shfl_xor_sync(0xffffffffu, ud[i], off);
    }
    if (lane == 0) {
      if (sizeof(T) == 4)  // own sum in FP64, partner sums arrive in out4
        for (int i = 0; i < 3; ++i) a.out[i * n + w] = ud[i];
      else
        for (int i = 0; i < 3; ++i) atomicAdd(a.out + i * n + w, ud[i]);
    }
  }
  if constexpr (sizeof(T) == 8) flush_pending();
}

// ------------------------------------------------------ double-float band
// Pairs with distance in [rcmid, rc64) are evaluated in double-float (df64)
// arithmetic on the FP32 pipe: ~1e-11 relative per term (the FP32 shell is
// ~1e-7, FP64 ~1e-15), at a fraction of the FP64 pipe's cost.  Positions
// enter as exact head differences plus tails (pair_vec_split), strengths as
// FP32 heads plus tails; the radial functions are built from:
//   1/rho   an FP32 estimate refined by one Newton step carried in df64;
//   e^{-z}  z = xi^2 rho^2 in df64, z = m ln2/64 - r with a Cody-Waite split
//           of ln2/64 (head of 12 bits: m ln2/64 is exact for |m| < 2^11),
//           e^{-z} = 2^{m/64} e^{r}, 2^{j/64} from a float-pair table and
//           e^{r} - 1 - r_head from its Taylor series in FP32 (|r| <= ln2/128);
//   erfcx   the interval polynomials of the FP64 table: c0 + u (c1 + u c2)
//           in df64, the higher terms (< 1e-4 of the sum) in FP32.
constexpr float kLn2By64HeadF = 2839.0f / 262144.0f;  // ln2/64 rounded to 12 bits
constexpr int kMidTab = 12;  // floats per erfcx interval: c0..c2 as pairs, c3..c8
constexpr float kNegInvLn2By64 = 92.332482616893658f;  // 64 / ln2

__device__ __forceinline__ df two_prod_f(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df(p, fmaf(a, b, -p));
}
__device__ __forceinline__ df dfc(float2 v) { return df(v.x, v.y); }

// the shared tables of k_real_mid: erfcx intervals (kMidTab floats each) and
// 2^{j/64} as float pairs
__device__ __forceinline__ void load_mid_tables(float* et, float2* t2) {
  for (int i = threadIdx.x; i < HSE_ERFCX_NINT; i += blockDim.x) {
    const double* c = d_erfcx_coef + i * (HSE_ERFCX_DEG + 1);
    float* o = et + i * kMidTab;
    for (int k = 0; k < 3; ++k) {
      const float h = (float)c[k];
      o[2 * k] = h;
      o[2 * k + 1] = (float)(c[k] - (double)h);
    }
    for (int k = 3; k <= HSE_ERFCX_DEG; ++k) o[3 + k] = (float)c[k];
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    const float h = (float)d_exp2_j64[i];
    t2[i] = make_float2(h, (float)(d_exp2_j64[i] - (double)h));
  }
  __syncthreads();
}

__device__ __forceinline__ Radial<df> radial_mid(const df* r, const RealArgs& a, const float* et, const float2* t2,
                                                 bool need_g3) {
  // s = |r|^2
  df s = r[0] * r[0];
  s += r[1] * r[1];
  s += r[2] * r[2];
  // inv = 1/sqrt(s): y (1 + e/2), e = 1 - s y^2
  const float y0 = rsqrtf(s.hi);
  const df y2 = two_prod_f(y0, y0);
  const float e = __fsub_rn(fmaf(-s.hi, y2.hi, 1.0f), fmaf(s.hi, y2.lo, __fmul_rn(s.lo, y2.hi)));
  const df inv = df_fast_two_sum(y0, __fmul_rn(0.5f * y0, e));
  // E = e^{-z}, z = xi^2 s
  const df z = dfc(a.dxi2) * s;
  const int m = __float2int_rn(-z.hi * kNegInvLn2By64);
  const float rh = __fsub_rn(-z.hi, __fmul_rn((float)m, kLn2By64HeadF));  // exact
  const float rl = __fsub_rn(-__fmul_rn((float)m, (float)(kLn2By64Head - (double)kLn2By64HeadF + kLn2By64Tail)),
                             z.lo);
  const float rr = __fadd_rn(rh, rl);
  const float qt = fmaf(__fmul_rn(rr, rr), fmaf(rr, fmaf(rr, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f), rl);
  const float2 tj = t2[m & 63];
  const df p = two_prod_f(tj.x, rh);
  const df eh = df_fast_two_sum(tj.x, p.hi);  // |p| <= ln2/128 of tj.x
  df E = df_fast_two_sum(eh.hi, __fadd_rn(__fadd_rn(eh.lo, p.lo),
                                          __fadd_rn(tj.y, fmaf(tj.x, qt, __fmul_rn(tj.y, rh)))));
  const float sc = __int_as_float((127 + (m >> 6)) << 23);  // 2^floor(m/64), m >= -64 * 126
  E = df(__fmul_rn(E.hi, sc), __fmul_rn(E.lo, sc));
  // t = xi rho = xi s inv, erfcx(t)
  const df t = dfc(a.dxi) * (s * inv);
  int k = (int)(t.hi * (float)HSE_ERFCX_INV_WIDTH);
  k = k < 0 ? 0 : (k > HSE_ERFCX_NINT - 1 ? HSE_ERFCX_NINT - 1 : k);
  const float* c = et + k * kMidTab;
  const float uh = __fmul_rn(__fsub_rn(t.hi, (float)(2 * k + 1) * (0.5f / HSE_ERFCX_INV_WIDTH)),
                             2.0f * HSE_ERFCX_INV_WIDTH);  // exact
  const float ul = __fmul_rn(t.lo, 2.0f * HSE_ERFCX_INV_WIDTH);
  float tail = c[3 + HSE_ERFCX_DEG];
#pragma unroll
  for (int j = HSE_ERFCX_DEG - 1; j >= 3; --j) tail = fmaf(tail, uh, c[3 + j]);
  tail = __fmul_rn(tail, __fmul_rn(__fmul_rn(uh, uh), uh));
  tail = fmaf(ul, fmaf(2.0f * c[4], uh, c[2]), tail);  // P'(u) ul
  const df h1 = (df(c[2], c[3]) + df(c[4], c[5]) * uh) * uh;
  const df ex = (df(c[0], c[1]) + h1) + df(tail, 0.f);
  Radial<df> R;
  const df i2 = inv * inv;
  R.c = dfc(a.dkc) * E;
  R.er = (E * ex) * inv;
  R.a1 = (R.er + R.c) * i2;
  R.g2 = i2 * fma(df(3.0f, 0.f), R.a1, dfc(a.dk2) * R.c);
  R.g3 = need_g3 ? -(i2 * fma(df(5.0f, 0.f), R.g2, dfc(a.dk4) * R.c)) : df(0.f, 0.f);
  return R;
}

template <int KM>
__device__ __forceinline__ void load_src_df(const RealArgs& a, int64_t j, Src<df>& s) {
  const int64_t n = a.n_src;
  auto ld = [&](int row) { return df(a.sstr32[row * n + j], a.sstr32lo[row * n + j]); };
#pragma unroll
  for (int i = 0; i < 3; ++i) { s.f[i] = df(0.f, 0.f); s.g[i] = s.f[i]; s.q[i] = s.f[i]; s.tau[i] = s.f[i]; }
  if (KM & HSE_STOKESLET)
    for (int i = 0; i < 3; ++i) s.f[i] = ld(a.rowS + i);
  if (KM & HSE_STRESSLET)
    for (int i = 0; i < 3; ++i) { s.g[i] = ld(a.rowT + i); s.q[i] = ld(a.rowT + 3 + i); }
  if (KM & HSE_ROTLET)
    for (int i = 0; i < 3; ++i) s.tau[i] = ld(a.rowW + i);
}

// Symmetric kernel of the double-float band (targets = sources; the same
// half list, cell scan and pair classification as k_real_sym, which skips
// these pairs): the target's sums go to a.out (FP64 atomics, one per
// component and target), the partner's share to the FP32 partner sums a.out4
// with the exact rounding error of each atomic and the double-float tail in
// a.out4lo.
template <int KM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_real_mid(RealArgs a) {
  __shared__ int queue[kWarpsPerBlock][kQueue];
  __shared__ float et[HSE_ERFCX_NINT * kMidTab];
  __shared__ float2 t2[64];
  load_mid_tables(et, t2);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* qu = queue[wib];
  const int64_t n = a.n_src;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const bool need_g3 = KM & HSE_STRESSLET;
  const df xid = dfc(a.dxi);
  float4 pend_old = make_float4(0.f, 0.f, 0.f, 0.f), pend_v = pend_old, pend_lo = pend_old;
  int64_t pend_j = -1;
  auto flush_pending = [&]() {
    if (pend_j >= 0) {
      float s0, e0, e1, e2;
      two_sum(pend_old.x, pend_v.x, s0, e0);
      two_sum(pend_old.y, pend_v.y, s0, e1);
      two_sum(pend_old.z, pend_v.z, s0, e2);
      atomicAdd(a.out4lo + pend_j,
                make_float4(__fadd_rn(e0, pend_lo.x), __fadd_rn(e1, pend_lo.y), __fadd_rn(e2, pend_lo.z), 0.f));
      pend_j = -1;
    }
  };
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < n; w += nwarps) {
    TgtPos x;
    for (int d = 0; d < 3; ++d) {
      x.d[d] = a.spos[d * n + w];
      x.h[d] = a.spos32[d * n + w];
      x.l[d] = a.spos32lo[d * n + w];
    }
    const df x3 = df_norm(df(x.h[2], x.l[2]));
    Src<df> sp;
    load_src_df<KM>(a, w, sp);
    df u[3] = {df(0.f, 0.f), df(0.f, 0.f), df(0.f, 0.f)};
    int cnt = 0;
    auto run = [&](int e) {
      const int j = e & 0x1fffffff, type = e >> 29;
      Src<df> s;
      load_src_df<KM>(a, j, s);
      float rf[3], dh[3], dl[3], hf;
      pair_vec_split(a, x, j, type == Q_IMAGE, dh, dl, rf, &hf);
      df r[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) r[d] = df_norm(df(dh[d], dl[d]));
      const df h = df_norm(df(a.spos32[2 * n + j], a.spos32lo[2 * n + j]));
      const Radial<df> R = radial_mid(r, a, et, t2, need_g3);
      df v[3] = {df(0.f, 0.f), df(0.f, 0.f), df(0.f, 0.f)};
      if (type == Q_FREE) {
        add_free<df>(KM, R, r, s, xid, df(1.0f, 0.f), u);
        add_free<df>(KM, R, r, sp, xid, df(-1.0f, 0.f), v);
      } else {
        add_image<df>(KM, R, r, h, x3, s, xid, u);
        if (j != w) {
          const df rp[3] = {-r[0], -r[1], r[2]};
          add_image<df>(KM, R, rp, x3, h, sp, xid, v);
        }
      }
      flush_pending();
      if (type == Q_FREE || j != w) {
        pend_v = make_float4(v[0].hi, v[1].hi, v[2].hi, 0.f);
        pend_lo = make_float4(v[0].lo, v[1].lo, v[2].lo, 0.f);
        pend_old = atomicAdd(a.out4 + j, pend_v);
        pend_j = j;
      }
    };
    float xf[3] = {x.h[0], x.h[1], x.h[2]};
    for_candidates<true>(a, x.d, xf, w, lane, (int)w + 1, (int)w, cell_base(a, w), [&](bool hit, int j, int type) {
      const bool use = hit && type != Q_SELF && (type & Q_MID);
      const unsigned m = __ballot_sync(0xffffffffu, use);
      if (use) qu[cnt + __popc(m & ((1u << lane) - 1))] = j | ((type & 1) << 29);
      cnt += __popc(m);
      __syncwarp();
      if (cnt >= 32) {
        run(qu[lane]);
        __syncwarp();
        if (lane < cnt - 32) qu[lane] = qu[32 + lane];
        cnt -= 32;
        __syncwarp();
      }
    });
    if (lane < cnt) run(qu[lane]);
    __syncwarp();
    for (int i = 0; i < 3; ++i) {
      double ud = (double)u[i].hi + (double)u[i].lo;
      for (int off = 16; off > 0; off >>= 1) ud += __shfl_xor_sync(0xffffffffu, ud, off);
      if (lane == 0) atomicAdd(a.out + i * n + w, ud);
    }
  }
  flush_pending();
}

// caller order: out[orig(i)] = sorted[i] (+ the FP32 partner sums, if any)
__global__ void k_unsort(int64_t n, const int32_t* __restrict__ sorig, const double* __restrict__ us,
                         const float4* __restrict__ us4, const float4* __restrict__ us4lo, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = sorig[i];
    const float4 p = us4 ? us4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 q = us4lo ? us4lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    out[o] = us[i] + ((double)p.x + (double)q.x);
    out[n + o] = us[n + i] + ((double)p.y + (double)q.y);
    out[2 * n + o] = us[2 * n + i] + ((double)p.z + (double)q.z);
  }
}

// FP32 path, targets = sources: image pairs closer than sqrt(img64_2) (FP32
// classification identical to k_real_sym<float>, which skips them).  For a
// target near the wall the image kernel and the wall corrections cancel to
// O(x3/rho) -- exactly at leading order for its own image, rho = 2 x3 -- so
// these pairs are evaluated in FP64, each ordered pair by its target's warp,
// and added to the target's FP64 sum after k_real_sym.  Only targets with
// x3^2 < img64_2 can have such pairs (rho >= x3 + y3 > x3).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_close_images(RealArgs a) {
  __shared__ double tab[kTabN];
  load_table(tab);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t n = a.n_src;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const bool need_g3 = a.mask & HSE_STRESSLET;
  const int nx = a.ncell[0], ny = a.ncell[1], nz = a.ncell[2];
  for (int64_t w = blockIdx.x * (int64_t)kWarpsPerBlock + wib; w < n; w += nwarps) {
    TgtPos x;
    for (int d = 0; d < 3; ++d) {
      x.d[d] = a.spos[d * n + w];
      x.h[d] = a.spos32[d * n + w];
      x.l[d] = a.spos32lo[d * n + w];
    }
    float x3f = x.h[2] + x.l[2];
    if (x3f * x3f >= a.img64_2) continue;
    int cx = cell_coord(x.d[0], a.inv_cell[0], nx);
    int cy = cell_coord(x.d[1], a.inv_cell[1], ny);
    int czi_hi = cell_coord(a.rc - x.d[2], a.inv_cell[2], nz);
    const int base = cell_base(a, w);
    double u[3] = {0.0, 0.0, 0.0};
    constexpr int R = kCellReach;
    for (int iz = 0; iz <= czi_hi; ++iz)
      for (int iy = (cy > R - 1 ? cy - R : 0); iy <= (cy < ny - R ? cy + R : ny - 1); ++iy) {
        int xa = cx > R - 1 ? cx - R : 0, xb = cx < nx - R ? cx + R : nx - 1;
        int c0 = base + (iz * ny + iy) * nx + xa;
        int s0 = a.cstart[c0], s1 = a.cstart[c0 + (xb - xa) + 1];
        for (int j = s0 + lane; j < s1; j += 32) {
          float rf[3], hf;
          pair_vec(a, x, j, true, rf, &hf);
          if (!(sq3(rf) < a.img64_2)) continue;
          Src<double> sj;
          load_src<double>(a, a.sstr, j, sj);
          double rd[3], hd;
          pair_vec(a, x, j, true, rd, &hd);
          double s2 = sq3(rd);
          Radial<double> R = radial(s2, approx_float(s2), a.xi, tab, nullptr, need_g3);
          add_image<double>(a.mask, R, rd, hd, x.d[2], sj, a.xi, u);
        }
      }
    for (int i = 0; i < 3; ++i)
      for (int off = 16; off > 0; off >>= 1) u[i] += __shfl_xor_sync(0xffffffffu, u[i], off);
    if (lane == 0)
      for (int i = 0; i < 3; ++i) a.out[i * n + w] += u[i];
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
      own = w;
      dst = a.sorig[w];
    }
    float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    int cf = 0, ci = 0;
    for_candidates(a, x, xf, own, lane, 0, 0, a.tgt ? 0 : cell_base(a, w), [&](bool hit, int j, int type) {
      unsigned mf = __ballot_sync(0xffffffffu, hit && type == Q_FREE);
      unsigned mi = __ballot_sync(0xffffffffu, hit && type == Q_IMAGE);
      cf += __popc(mf);
      ci += __popc(mi);
    });
    if (lane == 0) { na[dst] = cf; nb[dst] = ci; }
  }
}

// FP32 screening margin: the FP32 squared distance of two points inside a box
// of side Lmax differs from the exact one by at most
//   2 sqrt(3) |d| delta + 3 delta^2 + 2^-21 |d|^2,  delta = 1.5 2^-23 Lmax
// (rounding of each coordinate to FP32, of the difference, of the squares and
// sums).  Four times that bound around r_c^2 is sent to the FP64 test.
static RealArgs make_args(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add) {
  RealArgs a{};
  a.n_src = n_src;
  a.n_tgt = n_tgt;
  a.spos = p->ws.spos;
  a.spos32 = p->ws.spos32;
  a.spos32lo = p->ws.spos32lo;
  a.sstr = p->ws.sstr;
  a.sstr32 = p->ws.sstr32;
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
  double lmax = std::fmax(p->prm.box[0], std::fmax(p->prm.box[1], p->prm.box[2]));
  double delta = 1.5 * std::ldexp(1.0, -23) * lmax;
  double rc = p->prm.rc;
  double m = 4.0 * (2.0 * std::sqrt(3.0) * rc * delta + 3.0 * delta * delta + std::ldexp(1.0, -21) * rc * rc);
  a.rc2_lo = (float)std::fmax(0.0, a.rc2 - m) * (1.0f - 1e-6f);
  a.rc2_hi = (float)(a.rc2 + m) * (1.0f + 1e-6f);
  // cell rows are culled by an FP32 box distance: target and cell bounds are
  // rounded to FP32 (~3e-7 L), far inside the 1e-5 L margin
  const double rcull = rc + 1e-5 * lmax;
  a.cull2 = (float)(rcull * rcull);
  for (int d = 0; d < 3; ++d) a.cell_side[d] = (float)(p->prm.box[d] / p->prm.ncell[d]);
  a.img64_2 = (float)(a.rc2 / 256.0);
  a.far2 = 0.0f;
  for (int d = 0; d < 3; ++d) { a.inv_cell[d] = p->inv_cell[d]; a.ncell[d] = p->prm.ncell[d]; }
  a.inst_of = nullptr;
  a.ncells_inst = p->prm.ncell[0] * p->prm.ncell[1] * p->prm.ncell[2];
  a.mid2 = 0.0f;
  a.sstr32lo = p->ws.sstr32lo;
  auto split = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  const double xi = p->prm.xi;
  a.dxi = split(xi);
  a.dxi2 = split(xi * xi);
  a.dkc = split(2.0 * xi / kSqrtPi);
  a.dk2 = split(2.0 * xi * xi);
  a.dk4 = split(4.0 * xi * xi * xi * xi);
  return a;
}

// symmetric kernel specialised on the kernel bits (1..7) and on the
// double-float band (FP64 plans only)
template <typename T, bool MID>
static void launch_real_sym_t(int mask, int blocks, const RealArgs& a, cudaStream_t s) {
  switch (mask & 7) {
    case 1: k_real_sym<T, 1, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    case 2: k_real_sym<T, 2, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    case 3: k_real_sym<T, 3, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    case 4: k_real_sym<T, 4, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    case 5: k_real_sym<T, 5, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    case 6: k_real_sym<T, 6, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
    default: k_real_sym<T, 7, MID><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a); break;
  }
}
template <typename T>
static void launch_real_sym(int mask, int blocks, const RealArgs& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (a.mid2 > 0.0f) {
      launch_real_sym_t<T, true>(mask, blocks, a, s);
      return;
    }
  }
  launch_real_sym_t<T, false>(mask, blocks, a, s);
}

template <int KM>
static void launch_real_mid_t(int blocks, const RealArgs& a, cudaStream_t s) {
  k_real_mid<KM><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
}
static void launch_real_mid(int mask, int blocks, const RealArgs& a, cudaStream_t s) {
  switch (mask & 7) {
    case 1: launch_real_mid_t<1>(blocks, a, s); break;
    case 2: launch_real_mid_t<2>(blocks, a, s); break;
    case 3: launch_real_mid_t<3>(blocks, a, s); break;
    case 4: launch_real_mid_t<4>(blocks, a, s); break;
    case 5: launch_real_mid_t<5>(blocks, a, s); break;
    case 6: launch_real_mid_t<6>(blocks, a, s); break;
    default: launch_real_mid_t<7>(blocks, a, s); break;
  }
}

// FP64 plans: the double-float band [rcmid, min(rc64, rc)) of the symmetric
// kernel (k_real_mid); false when the plan has none
static bool mid_band(hse_plan p, RealArgs& a) {
  const double hi = std::fmin(p->prm.rc64 > 0.0 ? p->prm.rc64 : p->prm.rc, p->prm.rc);
  const double lo = p->prm.rcmid;
  if (p->prm.precision != HSE_FP64 || !(lo > 0.0) || lo >= hi) return false;
  a.mid2 = (float)(lo * lo);
  return true;
}

// FP64 plans: enable the FP32 outer shell [rc64, rc) of the symmetric kernel
static bool shell32(hse_plan p, RealArgs& a) {
  const double r64 = p->prm.rc64;
  if (p->prm.precision != HSE_FP64 || !(r64 > 0.0) || r64 >= p->prm.rc) return false;
  a.far2 = (float)(r64 * r64);
  return true;
}

static int warp_blocks(int64_t n_tgt) {
  int64_t b = (n_tgt + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (b > 152 * 64) b = 152 * 64;
  return b < 1 ? 1 : (int)b;
}

// blocks of the symmetric kernel: one warp per target, grid-stride; with a
// residency cap the grid is persistent (cap x SMs blocks), which leaves the
// rest of each SM's registers to kernels running concurrently on other streams
static int sym_blocks(hse_plan p, int64_t n_tgt) {
  int b = warp_blocks(n_tgt);
  if (p->real_bps > 0 && p->n_sm > 0 && b > p->real_bps * p->n_sm) b = p->real_bps * p->n_sm;
  return b;
}

hse_status real_space(hse_plan p, int64_t n_src, int64_t n_tgt, const double* tgt, double* out, bool add,
                      cudaStream_t s) {
  if (n_tgt == 0) return HSE_OK;
  RealArgs a = make_args(p, n_src, n_tgt, tgt, out, add);
  const bool mixed = p->prm.precision == HSE_MIXED;
  // targets = sources: each unordered pair once (half list), the partner's
  // share by atomics (FP64 path: 3 FP64 atomics; FP32 path: one float4 atomic)
  if (tgt == nullptr && !add) {
    a.out = p->ws.usort;
    a.out4 = p->ws.usort4;
    if (mixed) {
      HSE_CUDA(p, cudaMemsetAsync(a.out4, 0, sizeof(float4) * n_tgt, s));
      launch_real_sym<float>(a.mask, sym_blocks(p, n_tgt), a, s);
      if (!free_space(p->prm.kernel_mask)) {
        k_close_images<<<sym_blocks(p, n_tgt), kWarpsPerBlock * 32, 0, s>>>(a);
        ++p->n_launch;
      }
    } else {
      HSE_CUDA(p, cudaMemsetAsync(a.out, 0, sizeof(double) * 3 * n_tgt, s));
      const bool shell = shell32(p, a), mid = mid_band(p, a);
      if (shell || mid) {
        a.out4lo = a.out4 + n_tgt;
        HSE_CUDA(p, cudaMemsetAsync(a.out4, 0, sizeof(float4) * 2 * n_tgt, s));
      }
      launch_real_sym<double>(a.mask, sym_blocks(p, n_tgt), a, s);
      if (mid) {
        // the band's kernel scans only the cells within min(rc64, rc)
        RealArgs am = a;
        const double hi = std::fmin(p->prm.rc64 > 0.0 ? p->prm.rc64 : p->prm.rc, p->prm.rc);
        const double lmax = std::fmax(p->prm.box[0], std::fmax(p->prm.box[1], p->prm.box[2]));
        const double rcull = hi + 1e-5 * lmax;
        am.cull2 = (float)(rcull * rcull);
        HSE_CUDA(p, cudaGetLastError());
        launch_real_mid(a.mask, sym_blocks(p, n_tgt), am, s);
        ++p->n_launch;
      }
    }
    HSE_CUDA(p, cudaGetLastError());
    int64_t b = (n_tgt + 255) / 256;
    k_unsort<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(
        n_tgt, p->ws.val_a, p->ws.usort, (mixed || a.out4lo) ? p->ws.usort4 : nullptr, a.out4lo, out);
    ++p->n_launch;
  } else {
    if (mixed) k_real<float><<<warp_blocks(n_tgt), kWarpsPerBlock * 32, 0, s>>>(a);
    else k_real<double><<<warp_blocks(n_tgt), kWarpsPerBlock * 32, 0, s>>>(a);
  }
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_real");
}

// Batched instances (targets = sources, every instance sharing the plan's
// parameters): sorted particles of all instances, inst_of per sorted particle,
// cell lists of the instances one after another.  Writes the real-space sums
// of every particle in concatenated (unsorted) order to out.
hse_status real_space_batch(hse_plan p, int64_t n_total, const int32_t* inst_of, double* out, cudaStream_t s) {
  if (n_total == 0) return HSE_OK;
  RealArgs a = make_args(p, n_total, n_total, nullptr, nullptr, false);
  a.inst_of = inst_of;
  const bool mixed = p->prm.precision == HSE_MIXED;
  a.out = p->ws.usort;
  a.out4 = p->ws.usort4;
  if (mixed) {
    HSE_CUDA(p, cudaMemsetAsync(a.out4, 0, sizeof(float4) * n_total, s));
    launch_real_sym<float>(a.mask, warp_blocks(n_total), a, s);
    ++p->n_launch;
    if (!free_space(p->prm.kernel_mask)) {
      k_close_images<<<warp_blocks(n_total), kWarpsPerBlock * 32, 0, s>>>(a);
      ++p->n_launch;
    }
  } else {
    HSE_CUDA(p, cudaMemsetAsync(a.out, 0, sizeof(double) * 3 * n_total, s));
    if (shell32(p, a)) {
      a.out4lo = a.out4 + n_total;
      HSE_CUDA(p, cudaMemsetAsync(a.out4, 0, sizeof(float4) * 2 * n_total, s));
    }
    launch_real_sym<double>(a.mask, warp_blocks(n_total), a, s);
    ++p->n_launch;
  }
  HSE_CUDA(p, cudaGetLastError());
  int64_t b = (n_total + 255) / 256;
  k_unsort<<<(unsigned)(b > 152 * 32 ? 152 * 32 : b), 256, 0, s>>>(
      n_total, p->ws.val_a, p->ws.usort, (mixed || a.far2 > 0.0f) ? p->ws.usort4 : nullptr, a.out4lo, out);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "real_space_batch");
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
