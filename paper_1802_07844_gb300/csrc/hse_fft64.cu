// hse_fft64.cu -- zero-padded 3-D transforms of the FP64 path in double-float
// (df64) arithmetic on the FP32 pipe.
//
// The Fourier part of the method (Sec. 4: spread, zero-padded 3-D FFT, scale,
// inverse FFT, gather) spends most of its FP64 time in the transforms, and on
// GB300 cuFFT's double kernels are bound by the FP64 pipe (2 instructions per
// SM and clock).  These transforms do the same linear maps with ~48-bit
// double-float arithmetic on the 64x wider FP32 pipe; their rounding error
// (~1e-14 of the data norm) is far below the tolerances the FP64 path serves.
//
// Storage: the real grids hold df64 values (8 bytes, {hi, lo}) and a complex
// df64 value occupies 16 bytes ({re.hi, re.lo, im.hi, im.lo}), so the grids
// keep the layout of double grids.  The spread writes df64 values, the forward
// z pass turns them into half spectra in place, every later pass and the
// scaling stay df64, and the inverse z pass writes df64 values for the gather:
// no pass converts to or from FP64.
//
// Each pass is a batched 1-D transform of lines.  A block holds LPB lines in
// shared memory (element e of line l at e * LPB + l) and runs a mixed-radix
// Stockham autosort transform over them (radices 8, 4, 2, 5, 3), alternating
// between two shared buffers so that each radix pass needs one barrier; the
// twiddle table sits in shared memory, and the line passes queue the next
// line set's loads (cp.async) into a third buffer before transforming the
// current one, and store the outputs of their last radix pass straight to
// global memory (inverse passes whose first half is kept end with a radix-2
// pass that forms only that half).
#include <cmath>
#include <mutex>

#include "hse_df64.cuh"
#include "hse_internal.cuh"

namespace hse {

// ---------------------------------------------------------------- schedule
constexpr int kMaxPass = 24;

struct FftSteps {
  int N;                 // line length (complex points)
  int npass;
  int R[kMaxPass];       // radix of each pass
  int Ns[kMaxPass];      // product of the earlier radices
  int step[kMaxPass];    // N / (Ns R): twiddle index step
  unsigned magic[kMaxPass];  // ceil(2^32 / Ns) (exact j / Ns for j, Ns < 2^16)
  float kc[12];          // hi / lo of sin(2pi/3), cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5), cos(pi/4)
};

// two_first: the first pass has radix 2 (used for inputs whose upper half is
// zero: that pass reduces to a copy, done while loading)
// two_last: the last pass has radix 2 (used for inverse lines of which only
// the first half is kept: that pass then computes one output per butterfly)
// eight: radix 8 where 8 divides the rest (the schedules of wide line passes,
// see line_shape; the z passes keep radix 4)
static bool make_steps(int N, FftSteps* st, bool two_first = false, bool two_last = false, bool eight = false) {
  if (N < 2 || N >= 65536 || ((two_first || two_last) && N % 2 != 0) || (two_first && two_last && N % 4 != 0))
    return false;
  FftSteps s{};
  s.N = N;
  int rem = N, Ns = 1;
  while (rem > 1) {
    int R = eight && rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : rem % 5 == 0 ? 5 : rem % 3 == 0 ? 3 : 0;
    if (two_first && s.npass == 0) R = 2;
    if (two_last) {  // keep one factor 2 for the end
      if (R == 8 && (rem / 8) % 2 != 0) R = 4;  // radix 8 only while a factor 2 remains after it
      if (rem == 2) R = 2;
      else if (R == 4 && (rem / 4) % 2 != 0) R = (rem / 2) % 2 == 0 ? 2 : (rem % 5 == 0 ? 5 : (rem % 3 == 0 ? 3 : 2));
      else if (R == 2 && rem != 2 && (rem / 2) % 2 != 0) R = rem % 5 == 0 ? 5 : (rem % 3 == 0 ? 3 : 0);
    }
    if (R == 0 || s.npass == kMaxPass) return false;
    s.R[s.npass] = R;
    s.Ns[s.npass] = Ns;
    s.step[s.npass] = N / (Ns * R);
    s.magic[s.npass] = Ns == 1 ? 0u : (unsigned)((((uint64_t)1 << 32) + Ns - 1) / Ns);
    ++s.npass;
    Ns *= R;
    rem /= R;
  }
  const double c[6] = {std::sin(2 * M_PI / 3), std::cos(2 * M_PI / 5), std::cos(4 * M_PI / 5), std::sin(2 * M_PI / 5),
                       std::sin(4 * M_PI / 5), std::sqrt(0.5)};
  for (int i = 0; i < 6; ++i) {
    float h = (float)c[i];
    s.kc[2 * i] = h;
    s.kc[2 * i + 1] = (float)(c[i] - (double)h);
  }
  *st = s;
  return true;
}

// threads per line: one radix-4 butterfly each when 4 | N, else one radix-2
static int threads_per_line(int N) { return N % 4 == 0 ? N / 4 : N / 2; }
// "wide" line passes: N / 8 threads per line and radix-8 schedules (line_shape)
static bool wide_lines(int N) { return N % 8 == 0 && N >= 512; }

// block shape: at most kFftThreads threads, kFftMinBlocks resident per SM
// (register budget); compile-time tuning knobs
#ifndef HSE_FFT64_THREADS
#define HSE_FFT64_THREADS 512
#endif
#ifndef HSE_FFT64_MIN_BLOCKS
#define HSE_FFT64_MIN_BLOCKS 2
#endif
constexpr int kFftThreads = HSE_FFT64_THREADS, kFftMinBlocks = HSE_FFT64_MIN_BLOCKS;

// lines per block: a power of two, at most kFftThreads threads and 16 lines
static int lines_per_block_log2(int N) {
  int tpl = threads_per_line(N), lsh = 0;
  while (lsh < 4 && (tpl << (lsh + 1)) <= kFftThreads) ++lsh;
  return lsh;
}

// ------------------------------------------------------------- butterflies
// In-register radix-R DFTs (forward: exp(-2 pi i j k / R)) on unnormalised
// inputs; intermediate sums stay unnormalised, and the outputs are normalised
// only by the last pass of a transform (NORM): a df64 pair whose low part
// exceeds half an ulp of its high part by a few units is still accepted by
// every operation here, with the same error bound.
template <bool NORM>
__device__ __forceinline__ cdf out(cdf a) { return NORM ? norm(a) : a; }
template <bool FWD, bool NORM>
__device__ __forceinline__ void dft2(cdf* v) {
  const cdf a = v[0], b = v[1];
  v[0] = out<NORM>(add_raw(a, b));
  v[1] = out<NORM>(sub_raw(a, b));
}
template <bool FWD, bool NORM>
__device__ __forceinline__ void dft4(cdf* v) {
  const cdf a0 = add_raw(v[0], v[2]), a1 = sub_raw(v[0], v[2]);
  const cdf b0 = add_raw(v[1], v[3]), b1 = mul_mi<FWD>(sub_raw(v[1], v[3]));
  v[0] = out<NORM>(add_raw(a0, b0));
  v[2] = out<NORM>(sub_raw(a0, b0));
  v[1] = out<NORM>(add_raw(a1, b1));
  v[3] = out<NORM>(sub_raw(a1, b1));
}
template <bool FWD, bool NORM>
__device__ __forceinline__ void dft3(cdf* v, const float* kc) {
  const df s3(kc[0], kc[1]);
  const cdf t = add_raw(v[1], v[2]);
  const cdf a = sub_raw(v[0], scale_raw(df(0.5f, 0.f), t));
  const cdf b = mul_mi<FWD>(scale_raw(s3, sub_raw(v[1], v[2])));
  v[0] = out<NORM>(add_raw(v[0], t));
  v[1] = out<NORM>(add_raw(a, b));
  v[2] = out<NORM>(sub_raw(a, b));
}
template <bool FWD, bool NORM>
__device__ __forceinline__ void dft5(cdf* v, const float* kc) {
  const df c1(kc[2], kc[3]), c2(kc[4], kc[5]), s1(kc[6], kc[7]), s2(kc[8], kc[9]);
  const cdf t1 = add_raw(v[1], v[4]), t2 = add_raw(v[2], v[3]);
  const cdf t3 = sub_raw(v[1], v[4]), t4 = sub_raw(v[2], v[3]);
  const cdf a1 = add_raw(v[0], add_raw(scale_raw(c1, t1), scale_raw(c2, t2)));
  const cdf a2 = add_raw(v[0], add_raw(scale_raw(c2, t1), scale_raw(c1, t2)));
  const cdf b1 = mul_mi<FWD>(add_raw(scale_raw(s1, t3), scale_raw(s2, t4)));
  const cdf b2 = mul_mi<FWD>(sub_raw(scale_raw(s2, t3), scale_raw(s1, t4)));
  v[0] = out<NORM>(add_raw(v[0], add_raw(t1, t2)));
  v[1] = out<NORM>(add_raw(a1, b1));
  v[4] = out<NORM>(sub_raw(a1, b1));
  v[2] = out<NORM>(add_raw(a2, b2));
  v[3] = out<NORM>(sub_raw(a2, b2));
}

// radix 8 as two radix-4 DFTs of the even and odd inputs: X_k = E_k + w8^k O_k,
// X_{k+4} = E_k - w8^k O_k, with w8 = (1 -+ i) / sqrt(2), w8^2 = -+i and
// w8^3 = w8^2 w8 (upper signs forward); w8 O = (O + w8^2 O) / sqrt(2)
template <bool FWD, bool NORM>
__device__ __forceinline__ void dft8(cdf* v, const float* kc) {
  const df c(kc[10], kc[11]);
  cdf e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft4<FWD, false>(e);
  dft4<FWD, false>(o);
  const cdf p1 = scale_raw(c, add_raw(o[1], mul_mi<FWD>(o[1])));
  const cdf p2 = mul_mi<FWD>(o[2]);
  const cdf p3 = mul_mi<FWD>(scale_raw(c, add_raw(o[3], mul_mi<FWD>(o[3]))));
  v[0] = out<NORM>(add_raw(e[0], o[0]));
  v[4] = out<NORM>(sub_raw(e[0], o[0]));
  v[1] = out<NORM>(add_raw(e[1], p1));
  v[5] = out<NORM>(sub_raw(e[1], p1));
  v[2] = out<NORM>(add_raw(e[2], p2));
  v[6] = out<NORM>(sub_raw(e[2], p2));
  v[3] = out<NORM>(add_raw(e[3], p3));
  v[7] = out<NORM>(sub_raw(e[3], p3));
}

template <bool FWD>
__device__ __forceinline__ cdf twiddle(const float4* __restrict__ tw, int idx) {
  const cdf w = ld_cdf(tw + idx);  // shared-memory copy of the table
  return FWD ? w : conj(w);
}

// One Stockham pass (radix R, Ns = product of the earlier radices) from src
// to dst: butterfly j < N / R reads elements j + t N / R, multiplies element t
// by w_N^{t (j mod Ns) N / (Ns R)} (one exact two-sum per real part, result
// unnormalised), transforms, and writes output t to (j div Ns) Ns R +
// (j mod Ns) + t Ns.  Thread (l, tj) takes butterflies tj, tj + TPL, ... of
// line l.
template <int R, bool FWD, bool NORM>
__device__ __forceinline__ void stockham_pass(const float4* src, float4* dst, int N, int Ns, int step,
                                              unsigned magic, const float* kc, int tpl, int lsh, int l, int tj,
                                              const float4* __restrict__ tw) {
  const int nb = N / R;
  for (int j = tj; j < nb; j += tpl) {
    const int q = Ns == 1 ? j : (int)__umulhi((unsigned)j, magic);
    const int k = j - q * Ns;
    cdf v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = ld_cdf(src + ((j + t * nb) << lsh) + l);
    if (k != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) v[t] = mul_raw(v[t], twiddle<FWD>(tw, t * k * step));
    }
    if (R == 2) dft2<FWD, NORM>(v);
    else if (R == 4) dft4<FWD, NORM>(v);
    else if (R == 8) dft8<FWD, NORM>(v, kc);
    else if (R == 3) dft3<FWD, NORM>(v, kc);
    else dft5<FWD, NORM>(v, kc);
    const int d = q * Ns * R + k;
#pragma unroll
    for (int t = 0; t < R; ++t) st_cdf(dst + ((d + t * Ns) << lsh) + l, v[t]);
  }
}

// All passes, alternating between the block's two shared buffers (a holds the
// input); returns the buffer that holds the result, in natural order.  The
// schedule lives in device memory (uniform loads) so the pass loop can index
// it freely.
template <bool FWD, bool R8 = false>  // R8: schedules may hold radix-8 passes
__device__ __forceinline__ float4* transform_block(float4* a, float4* b, const FftSteps* __restrict__ st, int lsh,
                                                   const float4* __restrict__ tw, int p0 = 0, int p_end = -1) {
  const int tpl = blockDim.x >> lsh;
  const int l = threadIdx.x & ((1 << lsh) - 1), tj = threadIdx.x >> lsh;
  const int N = st->N, npass = st->npass;
  const float* kc = st->kc;
  if (p_end < 0) p_end = npass;
  for (int p = p0; p < p_end; ++p) {
    const int Ns = st->Ns[p], step = st->step[p];
    const unsigned magic = st->magic[p];
    if (p == npass - 1) {  // the last pass stores normalised values
      switch (st->R[p]) {
        case 4: stockham_pass<4, FWD, true>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        case 8:
          if constexpr (R8) stockham_pass<8, FWD, true>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw);
          break;
        case 2: stockham_pass<2, FWD, true>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        case 5: stockham_pass<5, FWD, true>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        default: stockham_pass<3, FWD, true>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
      }
    } else {
      switch (st->R[p]) {
        case 4: stockham_pass<4, FWD, false>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        case 8:
          if constexpr (R8) stockham_pass<8, FWD, false>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw);
          break;
        case 2: stockham_pass<2, FWD, false>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        case 5: stockham_pass<5, FWD, false>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
        default: stockham_pass<3, FWD, false>(a, b, N, Ns, step, magic, kc, tpl, lsh, l, tj, tw); break;
      }
    }
    __syncthreads();
    float4* t = a;
    a = b;
    b = t;
  }
  return a;
}

// The last Stockham pass of a line set (Ns = N / R: butterfly j takes
// elements j + t N/R and writes output t to element j + t N/R) with its
// normalised outputs stored straight to the line in global memory (elements
// e < nstore; start s[l] of line l, stride es), not to shared memory.  With
// R = 2 and nstore = N/2 only the first output of each butterfly is formed.
template <int R, bool FWD>
__device__ __forceinline__ void last_pass_store(const float4* src, float4* __restrict__ data, const long long* s,
                                                long long es, int N, int step, const float* kc, int lsh, int nstore,
                                                const float4* __restrict__ tw) {
  const int tpl = blockDim.x >> lsh;
  const int l = threadIdx.x & ((1 << lsh) - 1), tj = threadIdx.x >> lsh;
  const long long o = s[l];
  if (o < 0) return;
  const int nb = N / R;
  for (int j = tj; j < nb; j += tpl) {
    cdf v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = ld_cdf(src + ((j + t * nb) << lsh) + l);
    if (j != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) v[t] = mul_raw(v[t], twiddle<FWD>(tw, t * j * step));
    }
    if (R == 2 && 2 * nstore == N) {
      st_cdf(data + o + (long long)j * es, norm(add_raw(v[0], v[1])));
      continue;
    }
    if (R == 2) dft2<FWD, true>(v);
    else if (R == 4) dft4<FWD, true>(v);
    else if (R == 8) dft8<FWD, true>(v, kc);
    else if (R == 3) dft3<FWD, true>(v, kc);
    else dft5<FWD, true>(v, kc);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int e = j + t * nb;
      if (e < nstore) st_cdf(data + o + (long long)e * es, v[t]);
    }
  }
}

// ------------------------------------------------------------ line geometry
// Line b (< nlines) of a pass: r = b mod n0, g1 = (b div n0) mod n1,
// g2 = b div (n0 n1); it starts at g2 s2 + g1 s1 + r ls and its elements are
// es apart (units: complex values for C2C passes, doubles for the z passes).
struct LineGeo {
  long long nlines, n0, n1, ls, s1, s2, es;
};

__device__ __forceinline__ long long line_start(const LineGeo& g, long long b) {
  const long long t = b / g.n0, r = b - t * g.n0;
  const long long g2 = t / g.n1, g1 = t - g2 * g.n1;
  return g2 * g.s2 + g1 * g.s1 + r * g.ls;
}

// table of w_N^k = exp(-2 pi i k / N), k < N, rounded from FP64
__global__ void k_twiddles(int N, float4* __restrict__ tw) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)N, &sn, &cs);
    const df c(cs), si(sn);
    tw[k] = make_float4(c.hi, c.lo, si.hi, si.lo);
  }
}

// Asynchronous 16-byte copies global -> shared (the next line set is loaded
// while the current one is transformed)
__device__ __forceinline__ void cp_async16(float4* dst, const float4* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Queue the loads of one line set (starts s[]) into the shared buffer dst.
// half: element e < N/2 goes to positions 2e and 2e + 1 (the radix-2 first
// pass of an input whose upper half is zero is a copy); otherwise elements
// e >= nload are zero.  Lines beyond the last (start -1) are zero.
__device__ __forceinline__ void queue_set(const float4* data, const LineGeo& g, const long long* s, float4* dst,
                                          int lsh, int N, int nload, bool half) {
  const int lpb = 1 << lsh;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (half) {
    for (int i = threadIdx.x; i < (nload << lsh); i += blockDim.x) {
      const long long o = s[i & (lpb - 1)];
      const int e = i >> lsh, l = i & (lpb - 1);
      float4* d0 = dst + ((2 * e) << lsh) + l;
      if (o >= 0) {
        const float4* src = data + o + (long long)e * g.es;
        cp_async16(d0, src);
        cp_async16(d0 + lpb, src);
      } else {
        d0[0] = zero;
        d0[lpb] = zero;
      }
    }
  } else {
    for (int i = threadIdx.x; i < (N << lsh); i += blockDim.x) {
      const long long o = s[i & (lpb - 1)];
      const int e = i >> lsh;
      if (o >= 0 && e < nload) cp_async16(dst + i, data + o + (long long)e * g.es);
      else dst[i] = zero;
    }
  }
  cp_async_commit();
}

// ------------------------------------------------------------ C2C passes
// Elements e >= nload of a line are taken as zero (not read), and only
// elements e < nstore are written back: the data region of a forward pass's
// input and the part of an inverse pass's output that later steps read.
// A block loops over line sets with three shared buffers: the set being
// transformed, its scratch buffer, and the next set, whose loads are queued
// (cp.async) before the current set's passes run.
// WIDE: wide lines (radix-8 butterflies; blocks of N / 4 threads, whose
// residency the three line buffers in shared memory set): up to 128 registers
// (measured on the 1M workload: forward 54.3 -> 52.9 ms, inverse 31.2 -> 30.8
// ms against 64); other shapes keep the 64-register bound of their blocks of
// up to kFftThreads threads.
template <bool FWD, bool WIDE>
__global__ void __launch_bounds__(kFftThreads, WIDE ? 1 : kFftMinBlocks) k_fft_lines(float4* __restrict__ data, LineGeo g,
                                                      const FftSteps* __restrict__ st, int lsh,
                                                      const float4* __restrict__ tw, int nload, int nstore) {
  extern __shared__ float4 sm[];
  __shared__ long long start[3][16];  // line starts of three consecutive sets (one being written)
  const int lpb = 1 << lsh, N = st->N, n = N << lsh;
  float4* stw = sm + 3 * n;  // twiddles in shared memory (read by every pass)
  for (int i = threadIdx.x; i < N; i += blockDim.x) stw[i] = __ldg(tw + i);
  const bool half = nload * 2 == N && st->R[0] == 2;
  const long long step = (long long)gridDim.x * lpb;
  long long b0 = (long long)blockIdx.x * lpb;
  if (b0 >= g.nlines) return;
  auto set_starts = [&](long long b, long long* s) {
    if (threadIdx.x < lpb) s[threadIdx.x] = b + threadIdx.x < g.nlines ? line_start(g, b + threadIdx.x) : -1;
  };
  set_starts(b0, start[0]);
  __syncthreads();
  int cur = 0, nxt = 2;  // buffer of the current set, buffer the next set is loaded into
  queue_set(data, g, start[0], sm + cur * n, lsh, N, nload, half);
  for (int it = 0; b0 < g.nlines; b0 += step, ++it) {
    const long long* sc = start[it % 3];
    long long* sn = start[(it + 1) % 3];
    const long long b1 = b0 + step;
    if (b1 < g.nlines) set_starts(b1, sn);
    cp_async_wait_all();
    __syncthreads();  // the current set has landed; the last set's stores have read their buffer
    const int scr = 3 - cur - nxt;
    if (b1 < g.nlines) queue_set(data, g, sn, sm + nxt * n, lsh, N, nload, half);
    // all passes but the last in shared memory; the last one stores to global
    const int p0 = half ? 1 : 0, pl = st->npass - 1;
    if (pl >= p0) {
      const float4* res = transform_block<FWD, WIDE>(sm + cur * n, sm + scr * n, st, lsh, stw, p0, pl);
      const int step = st->step[pl];
      switch (st->R[pl]) {
        case 4: last_pass_store<4, FWD>(res, data, sc, g.es, N, step, st->kc, lsh, nstore, stw); break;
        case 8:
          if constexpr (WIDE) last_pass_store<8, FWD>(res, data, sc, g.es, N, step, st->kc, lsh, nstore, stw);
          break;
        case 2: last_pass_store<2, FWD>(res, data, sc, g.es, N, step, st->kc, lsh, nstore, stw); break;
        case 5: last_pass_store<5, FWD>(res, data, sc, g.es, N, step, st->kc, lsh, nstore, stw); break;
        default: last_pass_store<3, FWD>(res, data, sc, g.es, N, step, st->kc, lsh, nstore, stw); break;
      }
    } else {  // the whole transform was the load's radix-2 copy
      const float4* res = sm + cur * n;
      for (int i = threadIdx.x; i < (nstore << lsh); i += blockDim.x) {
        const long long o = sc[i & (lpb - 1)];
        if (o >= 0) data[o + (long long)(i >> lsh) * g.es] = res[i];
      }
    }
    const int used = cur;  // both of this set's buffers are free after the next barrier
    cur = nxt;
    nxt = used;
  }
  cp_async_wait_all();
}

// ---------------------------------------------- real <-> half spectrum (z)
// A real line of 2N df64 values x (contiguous) is transformed as the N complex
// values z_n = x_2n + i x_2n+1: with Z = DFT_N z, the half spectrum of x is
// X_k = (Z_k + conj Z_{N-k}) / 2 - i w^k (Z_k - conj Z_{N-k}) / 2, k = 0..N,
// w = exp(-2 pi i / 2N), written in place over the line (2N + 2 doubles hold
// N + 1 complex df64 values).  The inverse forms Z_k = (X_k + conj X_{N-k})
// + i conj(w^k) (X_k - conj X_{N-k}), transforms back (unnormalised, like a
// C2R transform) and writes the first nkeep values of the line.  The forward
// pass reads the first 2 nload real values only (the rest is zero).
template <bool FWD>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) k_fft_z(double* __restrict__ data, LineGeo g, const FftSteps* __restrict__ st,
                                                  int lsh, const float4* __restrict__ tw,
                                                  const float4* __restrict__ tw2, int nkeep, int nload) {
  extern __shared__ float4 sm[];
  __shared__ long long start[16];
  const int lpb = 1 << lsh, N = st->N;
  float4* stw = sm + 2 * (N << lsh);  // twiddles in shared memory (read by every pass)
  for (int i = threadIdx.x; i < N; i += blockDim.x) stw[i] = __ldg(tw + i);
  for (long long b0 = (long long)blockIdx.x * lpb; b0 < g.nlines; b0 += (long long)gridDim.x * lpb) {
    if (threadIdx.x < lpb) start[threadIdx.x] = b0 + threadIdx.x < g.nlines ? line_start(g, b0 + threadIdx.x) : -1;
    __syncthreads();
    // forward with a zero upper half and a radix-2 first pass: that pass is a
    // copy to positions 2k and 2k + 1, done here (as in k_fft_lines)
    const bool half = FWD && nload * 2 == N && st->R[0] == 2;
    for (int l = 0; l < lpb; ++l) {
      const long long o = start[l];
      for (int k = threadIdx.x; k < (half ? nload : N); k += blockDim.x) {
        cdf z = cdf_make(df(0.f, 0.f), df(0.f, 0.f));
        if (o >= 0) {
          if (FWD) {
            if (k < nload) z = ld_cdf(reinterpret_cast<const float4*>(data + o + 2 * k));  // x_2k, x_2k+1
          } else {
            const float4* X = reinterpret_cast<const float4*>(data + o);
            const cdf xk = ld_cdf(X + k), xn = conj(ld_cdf(X + N - k));
            const cdf wk = conj(ldg_cdf(tw2 + k));
            z = (xk + xn) + mul_mi<false>(wk * (xk - xn));
          }
        }
        if (half) {
          st_cdf(sm + ((2 * k) << lsh) + l, z);
          st_cdf(sm + ((2 * k + 1) << lsh) + l, z);
        } else {
          st_cdf(sm + (k << lsh) + l, z);
        }
      }
    }
    __syncthreads();
    const float4* res = transform_block<FWD>(sm, sm + (N << lsh), st, lsh, stw, half ? 1 : 0);
    for (int l = 0; l < lpb; ++l) {
      const long long o = start[l];
      if (o < 0) continue;
      if (FWD) {
        float4* X = reinterpret_cast<float4*>(data + o);
        const df half(0.5f, 0.f);
        for (int k = threadIdx.x; k <= N; k += blockDim.x) {
          const cdf zk = ld_cdf(res + ((k == N ? 0 : k) << lsh) + l);
          const cdf zn = conj(ld_cdf(res + ((k == 0 ? 0 : N - k) << lsh) + l));
          const cdf ev = half * (zk + zn), od = half * (zk - zn);
          st_cdf(X + k, ev + mul_mi<true>(ldg_cdf(tw2 + k) * od));
        }
      } else {
        for (int k = threadIdx.x; 2 * k < nkeep; k += blockDim.x) {
          const cdf z = ld_cdf(res + (k << lsh) + l);
          if (2 * k + 1 < nkeep) st_cdf(reinterpret_cast<float4*>(data + o + 2 * k), z);
          else *reinterpret_cast<float2*>(data + o + 2 * k) = make_float2(z.x.hi, z.x.lo);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ driver
struct Fft64Tables {
  FftSteps sx, sz;           // x / y lines (length Nx = Ny) and z half-lines (Nz / 2)
  FftSteps sxh, szh;         // the same with a radix-2 first pass (forward, zero upper half)
  FftSteps sxl;              // x / y lines with a radix-2 last pass (inverse, first half kept)
  FftSteps* d_steps = nullptr;  // device copies {sx, sz, sxh, szh, sxl}
  float4* tw = nullptr;      // twiddles of lengths Nx, Nz / 2 and Nz, back to back
};

static Fft64Tables* tables(hse_plan p) { return reinterpret_cast<Fft64Tables*>(p->fft64); }

// lengths whose schedule uses radices 2, 3, 4, 5 only and whose line fits
// one block (threads_per_line <= kFftThreads)
bool fft64_supported(int Nx, int Ny, int Nz) {
  FftSteps a, b;
  return Nx == Ny && Nz % 2 == 0 && make_steps(Nx, &a) && make_steps(Nz / 2, &b) &&
         threads_per_line(Nx) <= kFftThreads && threads_per_line(Nz / 2) <= kFftThreads;
}

hse_status fft64_prepare(hse_plan p) {
  if (p->fft64) return HSE_OK;
  const GridDims& g = p->g;
  if (!fft64_supported(g.Nx, g.Ny, g.Nz))
    return set_err(p, HSE_ERR_UNSUPPORTED, "df64 FFT: grid %d x %d x %d", g.Nx, g.Ny, g.Nz);
  Fft64Tables* t = new Fft64Tables();
  make_steps(g.Nx, &t->sx);
  make_steps(g.Nz / 2, &t->sz);
  make_steps(g.Nx, &t->sxh, true, false, wide_lines(g.Nx));  // forward line passes
  make_steps(g.Nz / 2, &t->szh, true);
  if (!make_steps(g.Nx, &t->sxl, false, true, wide_lines(g.Nx))) t->sxl = t->sx;
  const int n1 = g.Nx, nh = g.Nz / 2;
  cudaError_t e = cudaMalloc(&t->tw, sizeof(float4) * (n1 + nh + 2 * nh));
  if (e != cudaSuccess) {
    delete t;
    return cuda_check(p, e, "cudaMalloc(df64 twiddles)");
  }
  p->fft64 = t;
  HSE_CUDA(p, cudaMalloc(&t->d_steps, 5 * sizeof(FftSteps)));
  const FftSteps* hs[5] = {&t->sx, &t->sz, &t->sxh, &t->szh, &t->sxl};
  for (int i = 0; i < 5; ++i)
    HSE_CUDA(p, cudaMemcpy(t->d_steps + i, hs[i], sizeof(FftSteps), cudaMemcpyHostToDevice));
  k_twiddles<<<(n1 + 255) / 256, 256>>>(n1, t->tw);
  k_twiddles<<<(nh + 255) / 256, 256>>>(nh, t->tw + n1);
  k_twiddles<<<(2 * nh + 255) / 256, 256>>>(2 * nh, t->tw + n1 + nh);
  HSE_CUDA(p, cudaGetLastError());
  HSE_CUDA(p, cudaDeviceSynchronize());
  // a block holds up to three buffers of (threads / TPL) lines of N points (at
  // most kFftThreads threads and TPL >= N / 4: 32 KB each for 512 threads) and
  // the N twiddles (plans may be built from several threads: set the limits once)
  static std::once_flag attr;
  std::call_once(attr, [] {
    const int cap = 160 * 1024;  // up to three line buffers (<= 96 KB) and the twiddles (<= 32 KB)
    cudaFuncSetAttribute(k_fft_lines<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_fft_lines<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_fft_lines<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_fft_lines<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_fft_z<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    cudaFuncSetAttribute(k_fft_z<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  });
  return HSE_OK;
}

void fft64_destroy(hse_plan p) {
  Fft64Tables* t = tables(p);
  if (!t) return;
  cudaFree(t->tw);
  cudaFree(t->d_steps);
  delete t;
  p->fft64 = nullptr;
}

static unsigned grid_for(long long nlines, int lsh) {
  long long blocks = (nlines + (1 << lsh) - 1) >> lsh;
  const long long cap = 152LL * 3 * 32;
  return (unsigned)(blocks < cap ? blocks : cap);
}

// Line passes of lengths N >= 512 divisible by 8 ("wide" lines) run N / 8
// threads per line, two lines per block, with radix-8 passes where the
// schedule allows (one radix-8 butterfly per thread and pass, one pass through
// shared memory and one barrier where two radix-4 passes would take two): at
// N = 640 the forward schedule is 2 (the load's copy), 8, 8, 5 and the inverse
// 8, 8, 5, 2 instead of 2, 4, 4, 4, 5 and 4, 4, 4, 5, 2.  Measured on the 1M
// workload: forward 55.1 -> 54.0 ms, inverse 31.9 -> 31.1 ms.  Shorter lines
// divisible by 8 keep radix 4 and N / 8 threads per line forward (two
// butterflies per thread and pass: 56.8 -> 55.2 ms for the forward transforms
// of the 1M workload when that was measured) and N / 4 inverse: at N = 288 or
// 320 the N / 8 shape gives blocks of 72-80 threads, and the N = 1e5
// workloads' inverse transforms were slower with it.  Other lengths run one
// radix-4 (or radix-2) butterfly per thread.
static void line_shape(int N, bool fwd, int* tpl, int* lsh) {
  if (N % 8 == 0 && (fwd || wide_lines(N))) {
    *tpl = N / 8;
    *lsh = (*tpl << 1) <= kFftThreads ? 1 : 0;
  } else {
    *tpl = threads_per_line(N);
    *lsh = lines_per_block_log2(N);
  }
}

static hse_status run_lines(hse_plan p, double* buf, const LineGeo& geo, bool fwd, int nload, int nstore,
                            cudaStream_t s) {
  const Fft64Tables* t = tables(p);
  int tpl = 0, lsh = 0;
  line_shape(t->sx.N, fwd, &tpl, &lsh);
  const unsigned threads = (unsigned)(tpl << lsh);
  const size_t shm = sizeof(float4) * (3 * ((size_t)t->sx.N << lsh) + t->sx.N);  // three line buffers, twiddles
  if (geo.nlines <= 0) return HSE_OK;
  float4* c = reinterpret_cast<float4*>(buf);
  const dim3 grid(grid_for(geo.nlines, lsh));
  // forward passes read a zero upper half: the radix-2-first schedule; inverse
  // passes keeping the first half: the radix-2-last schedule
  const FftSteps* st = t->d_steps + (fwd ? 2 : (2 * nstore == t->sx.N ? 4 : 0));
  const bool wide = wide_lines(t->sx.N);
  if (fwd && wide) k_fft_lines<true, true><<<grid, threads, shm, s>>>(c, geo, st, lsh, t->tw, nload, nstore);
  else if (fwd) k_fft_lines<true, false><<<grid, threads, shm, s>>>(c, geo, st, lsh, t->tw, nload, nstore);
  else if (wide) k_fft_lines<false, true><<<grid, threads, shm, s>>>(c, geo, st, lsh, t->tw, nload, nstore);
  else k_fft_lines<false, false><<<grid, threads, shm, s>>>(c, geo, st, lsh, t->tw, nload, nstore);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), "k_fft_lines");
}

static hse_status run_z(hse_plan p, double* buf, const LineGeo& geo, bool fwd, int nkeep, int nload,
                        cudaStream_t s) {
  const Fft64Tables* t = tables(p);
  const int N = t->sz.N, lsh = lines_per_block_log2(N);
  const unsigned threads = (unsigned)(threads_per_line(N) << lsh);
  const size_t shm = sizeof(float4) * (2 * ((size_t)N << lsh) + N);  // two line buffers, twiddles
  if (geo.nlines <= 0) return HSE_OK;
  const float4* tw = t->tw + t->sx.N;
  const float4* tw2 = tw + N;
  if (fwd)  // radix-2-first schedule, as for the forward line passes
    k_fft_z<true><<<grid_for(geo.nlines, lsh), threads, shm, s>>>(buf, geo, t->d_steps + 3, lsh, tw, tw2, nkeep,
                                                                    nload);
  else
    k_fft_z<false><<<grid_for(geo.nlines, lsh), threads, shm, s>>>(buf, geo, t->d_steps + 1, lsh, tw, tw2, nkeep,
                                                                     nload);
  ++p->n_launch;
  return cuda_check(p, cudaGetLastError(), fwd ? "k_fft_z<fwd>" : "k_fft_z<inv>");
}

// Geometry of the grids: buffer b's real element (x, y, z) at
// x * xs + b * bs + y * pitch + z (8-byte units), nb buffers transformed together.
// Data occupy x < Mt, y < Mt, z < 2 Mt; the rest of the real grid is never
// read (taken as zero), so it needs no clearing.  As complex values the half
// spectrum (kx, ky, kz) of buffer b sits at (kx * xs + b * bs) / 2 + ky * nzh + kz.
hse_status fft64_forward(hse_plan p, double* base, int nb, long long bs, long long xs, cudaStream_t s) {
  const GridDims& g = p->g;
  const long long Mt = g.Mt, nzh = g.Nz / 2 + 1, pitch = g.pitch;
  const int N = (int)g.Nx, mt = (int)Mt;
  // z: lines (x < Mt, b, y < Mt), data at z < 2 Mt (Mt complex pairs)
  HSE_TRY(run_z(p, base, LineGeo{Mt * nb * Mt, Mt, nb, pitch, bs, xs, 1}, true, 0, mt, s));
  // y: lines (x < Mt, b, kz), elements y (data at y < Mt)
  HSE_TRY(run_lines(p, base, LineGeo{Mt * nb * nzh, nzh, nb, 1, bs / 2, xs / 2, nzh}, true, mt, N, s));
  // x: lines (b, y, kz) of every buffer, elements x (data at x < Mt)
  return run_lines(p, base, LineGeo{(long long)nb * g.Ny * nzh, (long long)g.Ny * nzh, nb, 1, bs / 2, 0, xs / 2},
                   true, mt, N, s);
}

// Inverse (unnormalised): df64 half spectra -> df64 values at x < Mt, y < Mt,
// z < 2 Mt of each of the nb buffers (the rest is left undefined).
hse_status fft64_inverse(hse_plan p, double* base, int nb, long long bs, long long xs, cudaStream_t s) {
  const GridDims& g = p->g;
  const long long Mt = g.Mt, nzh = g.Nz / 2 + 1, pitch = g.pitch;
  const int N = (int)g.Nx, mt = (int)Mt;
  // x: every line, written back for x < Mt (the planes the later passes read)
  HSE_TRY(run_lines(p, base, LineGeo{(long long)nb * g.Ny * nzh, (long long)g.Ny * nzh, nb, 1, bs / 2, 0, xs / 2},
                    false, N, mt, s));
  // y: the planes x < Mt, written back for y < Mt
  HSE_TRY(run_lines(p, base, LineGeo{Mt * nb * nzh, nzh, nb, 1, bs / 2, xs / 2, nzh}, false, N, mt, s));
  return run_z(p, base, LineGeo{Mt * nb * Mt, Mt, nb, pitch, bs, xs, 1}, false, (int)(2 * Mt), (int)(Mt), s);
}

}  // namespace hse
