/*
 * hs_oracle.c -- plain, slow FP64 CPU oracle for the half-space Stokes sums of
 * Srinivasan & Tornberg, "Fast Ewald summation for Green's functions of Stokes
 * flow in a half-space" (arXiv 1802.07844).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, the smoke check and the CPU-baseline leg of bench.py
 * use it.  It shares no code, header or constant table with the CUDA library.
 *
 * Units ("8 pi units"): the returned velocity is 8*pi times the physical
 * velocity at unit viscosity.  In these units the free-space kernels are
 *   stokeslet  S8(r) f      = f/r + r (r.f)/r^3                       (Sec. 2, eq. 1a)
 *   stresslet  T8(r) (g x q) = -6 r (r.g)(r.q)/r^5                     (Sec. 2, eq. 1b)
 *   rotlet     W8(r) tau    = 2 tau x r / r^3                         (Appendix, W^R as xi->0)
 * and the harmonic potential used by the wall corrections is G = 1/r (Sec. 3).
 *
 * Half-space sum (Sec. 3, eq. v_sum_halfspace), for target x and source y with
 * image y^I = (y1, y2, -y3), r = x - y, rt = x - y^I, h = y3:
 *   S:  S8(r) f - S8(rt) f^I - x3 grad(phi_S) + e3 phi_S
 *   T:  T8(r)(g x q) - T8(rt)(g^I x q^I) - x3 grad(phi_T) + e3 phi_T
 *   W:  W8(r) tau + W8(rt) tau^I - x3 grad(phi_W) + e3 phi_W
 *       (the paper's -2 W~ (g^I x q^I) equals +W8(rt) tau^I because
 *        g^I x q^I = -(g x q)^I for a reflection)
 * with the harmonic corrections of Sec. 3, eq. (phi), all evaluated at rt:
 *   phi_S = 2(-f3 G - h gradG . f^I)
 *   phi_T = 4 (g^I.q^I) d3G - 4 h g^I . (grad grad G) q^I
 *           (the printed phi_T has coefficients 2 and +2 on these two terms,
 *            which violates the no-slip condition; the coefficients used here
 *            are the unique ones giving zero velocity on the wall)
 *   phi_W = 4 gradG . v,  v = q3 g^I - g3 q^I = (-tau2, tau1, 0)
 * The rotlet strength is supplied as the torque tau = g x q directly.
 *
 * Ewald split (Sec. 4): every kernel K = K_R + K_F.
 *   Real-space parts: S^R, T^R, W^R of the Appendix (eq. kernel_real_parts; the
 *   last term of T^R carries r, not r-hat -- dimensional consistency and the
 *   smoothness of T_F require it) and G_R of Sec. 4, eq. (G_R), written with
 *   erfc so that no cancellation occurs at small r.
 *   Smooth parts: K_F = K - K_R written with erf (f(r) = erf(xi r)/r, Appendix)
 *   through F(s) = erf(xi sqrt(s))/sqrt(s) and its s-derivatives; near r = 0 the
 *   Taylor series in s is used.  Self term (Sec. 4 and Appendix): -4 xi/sqrt(pi) f
 *   for the stokeslet only.
 *
 * Free space (Sec. 2, mask bit OR_FREE = 8): the same sums without the wall --
 * only the free-space kernels S8(r) f, T8(r)(g q), W8(r) tau, no images and no
 * harmonic corrections; the Ewald split, the self term and the cut-off rule are
 * the same as above with the image terms dropped.
 *
 * Layouts: positions and strengths are component-major ("SoA"): x[0..n),
 * y[n..2n), z[2n..3n).  Strength blocks follow the kernel bits in the order
 * S (f: 3n), T (g: 3n then q: 3n), W (tau: 3n).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so that the cut-off and cell decisions match their stated operation order).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_S 1
#define OR_T 2
#define OR_W 4
#define OR_FREE 8

#define PART_DIRECT 0
#define PART_REAL 1
#define PART_SMOOTH 2
#define PART_SELF 3

static const double OR_PI = 3.14159265358979323846;
static const double OR_SQRT_PI = 1.77245385090551602730;

/* ------------------------------------------------------------------ */
/* radial coefficient sets                                              */
/* ------------------------------------------------------------------ */

/* G-type: G = g0, grad G = g1 r, grad grad G = g1 I + g2 r r,
 * grad^3 G = g2 (d r + d r + d r) + g3 r r r.                          */
typedef struct { double g0, g1, g2, g3; } gcoef;
/* kernel radial coefficients:
 *   S f   = sa f + sb r (r.f)
 *   T gq  = ta r (r.g)(r.q) + tb (g (r.q) + q (r.g) + r (g.q))
 *   W tau = wa tau x r                                                 */
typedef struct { double sa, sb, ta, tb, wa; } kcoef;

/* F(s) = erf(xi sqrt s)/sqrt s and its first three s-derivatives.
 * Series: F^(k)(s) = (2 xi/sqrt pi) sum_{n>=k} c_n xi^(2n) n!/(n-k)! s^(n-k),
 * c_n = (-1)^n / (n! (2n+1)); used for xi r < 1, closed forms otherwise.   */
static void fsmooth_derivs(double xi, double s, double F[4]) {
  double t2 = xi * xi * s;
  if (t2 < 1.0) {
    for (int k = 0; k < 4; ++k) {
      /* c_n n!/(n-k)! = (-1)^n / ((n-k)! (2n+1)); a = t2^(n-k)/(n-k)! */
      double sum = 0.0, a = 1.0;
      for (int n = k; n <= k + 40; ++n) {
        double sgn = (n % 2) ? -1.0 : 1.0;
        sum += sgn * a / (2.0 * n + 1.0);
        a *= t2 / (double)(n - k + 1);
      }
      F[k] = 2.0 * xi / OR_SQRT_PI * sum * pow(xi, 2.0 * k);
    }
    return;
  }
  double r = sqrt(s);
  double e = exp(-t2);
  double er = erf(xi * r);
  double a = xi / OR_SQRT_PI * e; /* xi e / sqrt(pi) */
  double x3 = xi * xi * xi / OR_SQRT_PI * e;
  double x5 = xi * xi * xi * xi * xi / OR_SQRT_PI * e;
  F[0] = er / r;
  F[1] = a / (r * r) - er / (2.0 * r * r * r);
  F[2] = -x3 / (r * r) - 1.5 * a / (r * r * r * r) + 0.75 * er / pow(r, 5);
  F[3] = x5 / (r * r) + 2.5 * x3 / pow(r, 4) + 3.75 * a / pow(r, 6) - 1.875 * er / pow(r, 7);
}

/* Coefficients of one part of the split at separation vector length rho (rho^2 = s). */
static void coefs(int part, double xi, double rho, double s, gcoef* g, kcoef* k) {
  if (part == PART_DIRECT) {
    /* plain kernels (Sec. 2, eq. 1; G = 1/r) */
    double i1 = 1.0 / rho, i3 = i1 * i1 * i1, i5 = i3 * i1 * i1, i7 = i5 * i1 * i1;
    g->g0 = i1; g->g1 = -i3; g->g2 = 3.0 * i5; g->g3 = -15.0 * i7;
    k->sa = i1; k->sb = i3; k->ta = -6.0 * i5; k->tb = 0.0; k->wa = 2.0 * i3;
  } else if (part == PART_REAL) {
    /* Sec. 4 eq. (G_R) and Appendix eq. (kernel_real_parts), erfc form */
    double t = xi * rho;
    double ec = erfc(t);
    double e = exp(-t * t);
    double c = 2.0 * xi / OR_SQRT_PI * e; /* 2 xi e^{-t^2}/sqrt(pi) */
    double i1 = 1.0 / rho, i2 = i1 * i1;
    double a1 = ec * i2 * i1 + c * i2;                                  /* 1/r^3 + f'/r         */
    double a2 = 3.0 * ec * i2 * i2 * i1 + c * (3.0 * i2 * i2 + 2.0 * xi * xi * i2);
    double a3 = -15.0 * ec * i2 * i2 * i2 * i1
                - c * (15.0 * i2 * i2 * i2 + 10.0 * xi * xi * i2 * i2 + 4.0 * xi * xi * xi * xi * i2);
    g->g0 = ec * i1; g->g1 = -a1; g->g2 = a2; g->g3 = a3;
    /* S^R = 2(xi e/sqrt pi + erfc/(2r)) (I + rh rh) - 4 xi e/sqrt(pi) I */
    double pre = c + ec * i1;          /* 2(xi e/sqrt pi + erfc/(2r)) */
    k->sa = pre - 2.0 * c;             /* coefficient of I           */
    k->sb = pre * i2;                  /* coefficient of r r         */
    /* T^R = -(2/r)[3 erfc/r + (2xi/sqrt pi)(3 + 2 t^2) e] rh rh rh
     *       + (4 xi^3/sqrt pi) e (d r + d r + d r)                      */
    k->ta = -2.0 * i2 * i2 * (3.0 * ec * i1 + c * (3.0 + 2.0 * t * t));
    k->tb = 2.0 * xi * xi * c;         /* 4 xi^3 e / sqrt(pi)         */
    /* W^R = 2 eps rh (erfc/r^2 + 2 xi e/(sqrt(pi) r)) */
    k->wa = 2.0 * (ec * i2 * i1 + c * i2);
  } else { /* PART_SMOOTH: K - K_R via F(s) */
    double F[4];
    fsmooth_derivs(xi, s, F);
    double e = exp(-xi * xi * s);
    g->g0 = F[0]; g->g1 = 2.0 * F[1]; g->g2 = 4.0 * F[2]; g->g3 = 8.0 * F[3];
    k->sa = 2.0 * F[0] + 2.0 * s * F[1];
    k->sb = -2.0 * F[1];
    k->ta = -8.0 * F[2];
    k->tb = -4.0 * xi * xi * xi / OR_SQRT_PI * e;
    k->wa = -4.0 * F[1];
  }
}

static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Distance squared in the fixed operation order ((dx*dx)+(dy*dy))+(dz*dz). */
static inline double dist2(const double* d) {
  double a = d[0] * d[0];
  double b = d[1] * d[1];
  double c = d[2] * d[2];
  return (a + b) + c;
}

/* Free-space kernel part applied to strengths of source m at displacement r. */
static void add_kernels(int mask, const kcoef* k, const double* r, const double* f, const double* g,
                        const double* q, const double* tau, double sign, double* u) {
  if (mask & OR_S) {
    double rf = dot3(r, f);
    for (int i = 0; i < 3; ++i) u[i] += sign * (k->sa * f[i] + k->sb * r[i] * rf);
  }
  if (mask & OR_T) {
    double rg = dot3(r, g), rq = dot3(r, q), gq = dot3(g, q);
    for (int i = 0; i < 3; ++i)
      u[i] += sign * (k->ta * r[i] * rg * rq + k->tb * (g[i] * rq + q[i] * rg + r[i] * gq));
  }
  if (mask & OR_W) {
    double c[3] = {tau[1] * r[2] - tau[2] * r[1], tau[2] * r[0] - tau[0] * r[2], tau[0] * r[1] - tau[1] * r[0]};
    for (int i = 0; i < 3; ++i) u[i] += sign * k->wa * c[i];
  }
}

/* Wall correction  -x3 grad(phi) + e3 phi  for source at height h, rt = x - y^I. */
static void add_corrections(int mask, const gcoef* G, const double* rt, double x3, double h, const double* f,
                            const double* g, const double* q, const double* tau, double* u) {
  double phi = 0.0, gphi[3] = {0.0, 0.0, 0.0};
  if (mask & OR_S) {
    double fI[3] = {f[0], f[1], -f[2]};
    double rfI = dot3(rt, fI);
    /* phi_S = 2(-f3 G - h gradG.f^I) ; gradG = g1 rt ; grad grad G = g1 I + g2 rt rt */
    phi += 2.0 * (-f[2] * G->g0 - h * G->g1 * rfI);
    for (int i = 0; i < 3; ++i) gphi[i] += 2.0 * (-f[2] * G->g1 * rt[i] - h * (G->g1 * fI[i] + G->g2 * rt[i] * rfI));
  }
  if (mask & OR_T) {
    double gI[3] = {g[0], g[1], -g[2]}, qI[3] = {q[0], q[1], -q[2]};
    double gq = dot3(gI, qI), rg = dot3(rt, gI), rq = dot3(rt, qI);
    /* phi_T = 4 (gI.qI) d3G - 4 h gI.(grad grad G) qI */
    phi += 4.0 * gq * G->g1 * rt[2] - 4.0 * h * (G->g1 * gq + G->g2 * rg * rq);
    for (int i = 0; i < 3; ++i) {
      double d3i = G->g1 * (i == 2 ? 1.0 : 0.0) + G->g2 * rt[2] * rt[i]; /* (grad grad G)_{3i} */
      double t3 = G->g2 * (gq * rt[i] + gI[i] * rq + qI[i] * rg) + G->g3 * rg * rq * rt[i];
      gphi[i] += 4.0 * gq * d3i - 4.0 * h * t3;
    }
  }
  if (mask & OR_W) {
    double v[3] = {-tau[1], tau[0], 0.0};
    double rv = dot3(rt, v);
    /* phi_W = 4 gradG . v */
    phi += 4.0 * G->g1 * rv;
    for (int i = 0; i < 3; ++i) gphi[i] += 4.0 * (G->g1 * v[i] + G->g2 * rt[i] * rv);
  }
  for (int i = 0; i < 3; ++i) u[i] += -x3 * gphi[i];
  u[2] += phi;
}

static void load_strengths(int mask, long n, long m, const double* str, double* f, double* g, double* q,
                           double* tau) {
  long off = 0;
  if (mask & OR_S) { for (int i = 0; i < 3; ++i) f[i] = str[off + i * n + m]; off += 3 * n; }
  if (mask & OR_T) {
    for (int i = 0; i < 3; ++i) g[i] = str[off + i * n + m];
    off += 3 * n;
    for (int i = 0; i < 3; ++i) q[i] = str[off + i * n + m];
    off += 3 * n;
  }
  if (mask & OR_W) { for (int i = 0; i < 3; ++i) tau[i] = str[off + i * n + m]; off += 3 * n; }
}

/*
 * oracle_sum: one part of the half-space sum at every target.
 *   part = 0 (direct): the plain sum, Sec. 3 eq. (v_sum_halfspace); the
 *          free-space pair of a target with itself is skipped (Sec. 2).
 *   part = 1 (real): kernels replaced by their real-space parts; a pair
 *          (free-space or image) is used iff |d|^2 < rc^2 with the squared
 *          distance formed as ((dx*dx)+(dy*dy))+(dz*dz); rc <= 0 means no
 *          cut-off.  Self pairs are skipped like in the direct sum.
 *   part = 2 (smooth): kernels replaced by K - K_R, all pairs including the
 *          target's own source (limit values at r = 0).
 *   part = 3 (self): -4 xi/sqrt(pi) f for every (target, source) pair that is
 *          skipped in parts 0/1 (stokeslet only).
 * Identity (Sec. 4): direct = real(no cut-off) + smooth + self.
 * tgt_is_src != 0: targets are the sources (pair m = p skipped by index);
 * otherwise pairs at exactly zero separation are skipped.
 * out: 3 x n_tgt, component-major, overwritten.                               */
int oracle_sum(int mask, int part, double xi, double rc, long n_src, const double* src, const double* str,
               long n_tgt, const double* tgt, int tgt_is_src, double* out) {
  if (n_src < 0 || n_tgt < 0 || (mask & 7) == 0 || mask > 15) return 1;
  if (tgt_is_src) { tgt = src; n_tgt = n_src; }
  double rc2 = rc * rc;
  int cut = (part == PART_REAL && rc > 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (long p = 0; p < n_tgt; ++p) {
    double x[3] = {tgt[p], tgt[n_tgt + p], tgt[2 * n_tgt + p]};
    double u[3] = {0.0, 0.0, 0.0};
    for (long m = 0; m < n_src; ++m) {
      double y[3] = {src[m], src[n_src + m], src[2 * n_src + m]};
      double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, q[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
      load_strengths(mask, n_src, m, str, f, g, q, tau);
      double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
      double yI2 = -y[2];
      double rt[3] = {x[0] - y[0], x[1] - y[1], x[2] - yI2};
      double h = y[2];
      double s = dist2(r), st = dist2(rt);
      int same = tgt_is_src ? (m == p) : (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0);
      gcoef G;
      kcoef K;
      if (part == PART_SELF) {
        if (same && (mask & OR_S))
          for (int i = 0; i < 3; ++i) u[i] += -4.0 * xi / OR_SQRT_PI * f[i];
        continue;
      }
      /* free-space pair */
      int use = (part == PART_SMOOTH) ? 1 : !same;
      if (cut && !(s < rc2)) use = 0;
      if (use) {
        coefs(part, xi, sqrt(s), s, &G, &K);
        add_kernels(mask, &K, r, f, g, q, tau, 1.0, u);
      }
      /* image pair and wall corrections, both at rt (none in free space) */
      int usei = !(mask & OR_FREE);
      if (cut && !(st < rc2)) usei = 0;
      if (usei) {
        coefs(part, xi, sqrt(st), st, &G, &K);
        double fI[3] = {f[0], f[1], -f[2]}, gI[3] = {g[0], g[1], -g[2]}, qI[3] = {q[0], q[1], -q[2]};
        double tauI[3] = {tau[0], tau[1], -tau[2]};
        /* S: -S(rt) f^I ; T: -T(rt)(g^I x q^I) ; W: +W(rt) tau^I */
        add_kernels(mask & (OR_S | OR_T), &K, rt, fI, gI, qI, tauI, -1.0, u);
        add_kernels(mask & OR_W, &K, rt, fI, gI, qI, tauI, 1.0, u);
        add_corrections(mask, &G, rt, x[2], h, f, g, q, tau, u);
      }
    }
    out[p] = u[0];
    out[n_tgt + p] = u[1];
    out[2 * n_tgt + p] = u[2];
  }
  return 0;
}

/* Radial coefficients of one part at rho, for unit tests of the formulas.
 * out: g0 g1 g2 g3 sa sb ta tb wa                                           */
void oracle_coefs(int part, double xi, double rho, double* out) {
  gcoef G;
  kcoef K;
  coefs(part, xi, rho, rho * rho, &G, &K);
  out[0] = G.g0; out[1] = G.g1; out[2] = G.g2; out[3] = G.g3;
  out[4] = K.sa; out[5] = K.sb; out[6] = K.ta; out[7] = K.tb; out[8] = K.wa;
}

/* F, F', F'', F''' of the smooth split (for unit tests). */
void oracle_fsmooth(double xi, double s, double* out) { fsmooth_derivs(xi, s, out); }

/*
 * oracle_cells: cell list for the real-space neighbour search (Sec. 5.1).
 * Cell of a point: c_d = clamp((int)floor((x_d - origin_d) * inv_cell_d), 0, ncell_d - 1),
 * id = (c_z * ncell_y + c_y) * ncell_x + c_x.  perm lists the points sorted by
 * (id, original index) -- a stable counting sort done sequentially.
 * cell_start has ncell_x*ncell_y*ncell_z + 1 entries.                        */
int oracle_cells(long n, const double* pos, const double* origin, const double* inv_cell, const int* ncell,
                 int* cell_id, int* perm, int* cell_start) {
  long nc = (long)ncell[0] * ncell[1] * ncell[2];
  for (long i = 0; i < n; ++i) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      double t = (pos[d * n + i] - origin[d]) * inv_cell[d];
      double fl = floor(t);
      int ci;
      if (fl < 0.0) ci = 0;
      else if (fl > (double)(ncell[d] - 1)) ci = ncell[d] - 1;
      else ci = (int)fl;
      c[d] = ci;
    }
    cell_id[i] = (c[2] * ncell[1] + c[1]) * ncell[0] + c[0];
  }
  for (long c = 0; c <= nc; ++c) cell_start[c] = 0;
  for (long i = 0; i < n; ++i) cell_start[cell_id[i] + 1]++;
  for (long c = 0; c < nc; ++c) cell_start[c + 1] += cell_start[c];
  int* fill = (int*)malloc(sizeof(int) * (nc > 0 ? nc : 1));
  for (long c = 0; c < nc; ++c) fill[c] = cell_start[c];
  for (long i = 0; i < n; ++i) perm[fill[cell_id[i]]++] = (int)i;
  free(fill);
  return 0;
}

/*
 * oracle_neighbor_counts: brute-force count, per target, of free-space pairs
 * and of image pairs within the cut-off (|d|^2 < rc^2, same operation order as
 * the real-space part), self pair skipped as in oracle_sum.                  */
int oracle_neighbor_counts(long n_src, const double* src, long n_tgt, const double* tgt, int tgt_is_src,
                           double rc, int* n_pairs, int* n_images) {
  if (tgt_is_src) { tgt = src; n_tgt = n_src; }
  double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 16)
  for (long p = 0; p < n_tgt; ++p) {
    int a = 0, b = 0;
    double x[3] = {tgt[p], tgt[n_tgt + p], tgt[2 * n_tgt + p]};
    for (long m = 0; m < n_src; ++m) {
      double y[3] = {src[m], src[n_src + m], src[2 * n_src + m]};
      double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
      double yI2 = -y[2];
      double rt[3] = {x[0] - y[0], x[1] - y[1], x[2] - yI2};
      int same = tgt_is_src ? (m == p) : (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0);
      if (!same && dist2(r) < rc2) ++a;
      if (dist2(rt) < rc2) ++b;
    }
    n_pairs[p] = a;
    n_images[p] = b;
  }
  return 0;
}

/*
 * Grid geometry of the Fourier part (Alg. 1, steps 2-4), as read here:
 *   spacing h, support P (even), extended size Mt = M + P;
 *   grid of Mt x Mt x 2Mt points, point (i,j,k) at
 *   (-P h/2 + i h, -P h/2 + j h, -Mt h + k h), so the wall z = 0 is the plane
 *   k = Mt and index k mirrors to 2 Mt - k.
 * Support of a Gaussian centred at c along one axis: the P indices starting at
 *   i0 = clamp(floor((c - o) / h) - P/2 + 1, 0, n - P).
 * An image point uses the mirror of its source's z-support (the P indices
 * 2 Mt - k for k in the source's support), so source and image supports are
 * exact reflections of one another.
 * Window (Alg. 1 step 5, with the square on the distance that its Fourier
 * transform requires): (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 |x - z|^2 / eta),
 * eta = P xi^2 h^2 / (c^2 pi), c = 0.95 (Alg. 1 step 4).
 */
static int support_start(double c, double o, double h, int P, int n) {
  double t = floor((c - o) / h);
  long i0 = (long)t - P / 2 + 1;
  if (i0 < 0) i0 = 0;
  if (i0 > n - P) i0 = n - P;
  return (int)i0;
}

static void splat(double* grid, int Mt, int P, double h, double xi, double eta, const double* z, int ix0, int iy0,
                  int iz0, const double* val, int nval, long comp_stride) {
  double pre = pow(2.0 * xi * xi / (OR_PI * eta), 1.5);
  double ox = -0.5 * P * h, oz = -(double)Mt * h;
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < P; ++b)
      for (int c = 0; c < P; ++c) {
        int i = ix0 + a, j = iy0 + b, k = iz0 + c;
        double gx = ox + i * h, gy = ox + j * h, gz = oz + k * h;
        double d2 = (gx - z[0]) * (gx - z[0]) + (gy - z[1]) * (gy - z[1]) + (gz - z[2]) * (gz - z[2]);
        double w = pre * exp(-2.0 * xi * xi * d2 / eta);
        long idx = ((long)i * Mt + j) * (2L * Mt) + k;
        for (int v = 0; v < nval; ++v) grid[v * comp_stride + idx] += w * val[v];
      }
}

/*
 * oracle_spread: the gridded source terms of Alg. 1 step 5, for each kernel in
 * mask order (S, T, W):
 *   S: C1 = F over the 2N points (f at y, -f^I at y^I)        [3 components]
 *      C2 = f3 at y^I                                          [1]
 *      C3 = y3 f^I at y^I                                      [3]
 *   T: C1 = sym(g q) at y, -sym(g^I q^I) at y^I                [6: xx xy xz yy yz zz]
 *      C2 = g.q at y^I                                         [1]
 *      C3 = y3 sym(g^I q^I) at y^I                             [6]
 *   W: C1 = tau at y, +tau^I at y^I                            [3]
 *      C2 = v = (-tau2, tau1) at y^I                           [2]
 * In free space (mask bit OR_FREE) only C1 at the sources y:
 *   S: f [3]    T: sym(g q) [6]    W: tau [3]
 * grids: ncomp x Mt x Mt x 2Mt (z fastest), zeroed here.  Returns ncomp.     */
int oracle_spread(int mask, long n, const double* src, const double* str, double xi, double h, int P, int Mt,
                  double* grids) {
  double eta = P * xi * xi * h * h / (0.95 * 0.95 * OR_PI);
  long cs = (long)Mt * Mt * 2 * Mt;
  const int free_space = (mask & OR_FREE) != 0;
  int ncomp = free_space ? ((mask & OR_S) ? 3 : 0) + ((mask & OR_T) ? 6 : 0) + ((mask & OR_W) ? 3 : 0)
                         : ((mask & OR_S) ? 7 : 0) + ((mask & OR_T) ? 13 : 0) + ((mask & OR_W) ? 5 : 0);
  memset(grids, 0, sizeof(double) * cs * ncomp);
  double ox = -0.5 * P * h, oz = -(double)Mt * h;
  for (long m = 0; m < n; ++m) {
    double y[3] = {src[m], src[n + m], src[2 * n + m]};
    double yI[3] = {y[0], y[1], -y[2]};
    double f[3] = {0, 0, 0}, g[3] = {0, 0, 0}, q[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
    load_strengths(mask, n, m, str, f, g, q, tau);
    int ix0 = support_start(y[0], ox, h, P, Mt);
    int iy0 = support_start(y[1], ox, h, P, Mt);
    int iz0 = support_start(y[2], oz, h, P, 2 * Mt);
    int izI = 2 * Mt - (iz0 + P - 1);
    double* gp = grids;
    if (free_space) {
      if (mask & OR_S) {
        splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, f, 3, cs);
        gp += 3 * cs;
      }
      if (mask & OR_T) {
        double sg[6];
        int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; ++c) sg[c] = 0.5 * (g[ia[c]] * q[ib[c]] + g[ib[c]] * q[ia[c]]);
        splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, sg, 6, cs);
        gp += 6 * cs;
      }
      if (mask & OR_W) splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, tau, 3, cs);
      continue;
    }
    if (mask & OR_S) {
      double fI[3] = {f[0], f[1], -f[2]};
      double c1[3] = {f[0], f[1], f[2]};
      double c1I[3] = {-fI[0], -fI[1], -fI[2]};
      double cI[4] = {f[2], y[2] * fI[0], y[2] * fI[1], y[2] * fI[2]};
      splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, c1, 3, cs);
      splat(gp, Mt, P, h, xi, eta, yI, ix0, iy0, izI, c1I, 3, cs);
      splat(gp + 3 * cs, Mt, P, h, xi, eta, yI, ix0, iy0, izI, cI, 4, cs);
      gp += 7 * cs;
    }
    if (mask & OR_T) {
      double gI[3] = {g[0], g[1], -g[2]}, qI[3] = {q[0], q[1], -q[2]};
      double s[6], sI[6];
      int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
      for (int c = 0; c < 6; ++c) {
        s[c] = 0.5 * (g[ia[c]] * q[ib[c]] + g[ib[c]] * q[ia[c]]);
        sI[c] = 0.5 * (gI[ia[c]] * qI[ib[c]] + gI[ib[c]] * qI[ia[c]]);
      }
      double c1I[6], cI[7];
      for (int c = 0; c < 6; ++c) c1I[c] = -sI[c];
      cI[0] = dot3(gI, qI);
      for (int c = 0; c < 6; ++c) cI[1 + c] = y[2] * sI[c];
      splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, s, 6, cs);
      splat(gp, Mt, P, h, xi, eta, yI, ix0, iy0, izI, c1I, 6, cs);
      splat(gp + 6 * cs, Mt, P, h, xi, eta, yI, ix0, iy0, izI, cI, 7, cs);
      gp += 13 * cs;
    }
    if (mask & OR_W) {
      double tI[3] = {tau[0], tau[1], -tau[2]};
      double v[2] = {-tau[1], tau[0]};
      splat(gp, Mt, P, h, xi, eta, y, ix0, iy0, iz0, tau, 3, cs);
      splat(gp, Mt, P, h, xi, eta, yI, ix0, iy0, izI, tI, 3, cs);
      splat(gp + 3 * cs, Mt, P, h, xi, eta, yI, ix0, iy0, izI, v, 2, cs);
      gp += 5 * cs;
    }
  }
  return ncomp;
}
