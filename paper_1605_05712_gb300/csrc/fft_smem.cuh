// fft_smem.cuh -- in-place shared-memory FFT stages for the pattern FFT (sm_103a).
//
// The pattern FFT of Sec. 2.2 is an ordinary d_M-dimensional DFT over the
// elementary divisors; every 1-D piece of it runs here on lines held in
// shared memory.  Forward transforms leave the spectrum in bit-reversed order
// and inverse transforms take bit-reversed input to natural output, so
// forward -> pointwise Green operator -> inverse needs no permutation pass: the
// pointwise step decodes each frequency with __brev.
//
// Binary32 and double-float kernels: the forward transform is decimation in
// frequency (Sande-Tukey), the inverse its exact adjoint (decimation in time);
// radix-4 stages are two radix-2 stages fused (so the order stays plain bit
// reversal), an odd log2 length adds one radix-2 stage.  Binary64 kernels run
// decimation in time both ways with fused multiply-add butterflies (fft_fwd_fma,
// fft_inv_fma below).  Butterflies are in place, a thread keeps only the
// values of the butterflies it is working on, and stages are separated by
// __syncthreads().
//
// Line addressing: a line l = l_hi * nlo + l_lo (nlo a power of two) has its element idx at
//   l_hi * L * nlo + idx * nlo + l_lo,
// which covers contiguous rows (nlo = 1) and tiles of columns (nlo = tile
// width x inner axes) alike, stored at slot tpos() of that index (the padded
// tile layout).  Butterfly numbering puts l_lo fastest, so neighbouring
// threads touch neighbouring shared-memory words.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "df64.cuh"

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<dfloat> { typedef dcplx type; };

template <typename C> __device__ __forceinline__ C cmake(double x, double y);
template <> __device__ __forceinline__ double2 cmake<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 cmake<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <> __device__ __forceinline__ dcplx cmake<dcplx>(double x, double y) {
  dcplx r;
  r.x = dfloat(x);
  r.y = dfloat(y);
  return r;
}
// complex from two reals of the kernel's precision (no round trip through binary64)
template <typename C, typename R> __device__ __forceinline__ C cpair(R x, R y) { C r; r.x = x; r.y = y; return r; }

// read-only loads of complex table entries
template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ dcplx ldg_c<dcplx>(const dcplx* p) { return ldg_dc(p); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
// i * a
template <typename C> __device__ __forceinline__ C cmuli(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }

// slot of tile element i (one pad slot after every 128 bytes of values; see tile_span in kernels.cuh)
template <typename C> __device__ __forceinline__ int tpos(int i) { return i + (i >> (sizeof(C) == 8 ? 4 : 3)); }

__device__ __forceinline__ uint32_t bitrev(uint32_t p, int log2L) {
  return log2L == 0 ? 0u : (__brev(p) >> (32 - log2L));
}

// twiddle W_L^j = exp(-2 pi i j / L) from the table of W_N^t, N = 2^tw_log2 >= L
template <typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int tw_log2, int log2L, uint32_t j) {
  return ldg_c(&tw[j << (tw_log2 - log2L)]);
}

// the three twiddles W_L^j, W_L^{2j}, W_L^{3j} of a radix-4 butterfly.  Binary32 kernels load W_L^j and
// form the powers by complex multiplication (two products instead of two table loads, whose latency the
// binary32 passes wait on; about one rounding more, inside the mixed-precision tolerance); binary64 and
// pair kernels load all three (their arithmetic pipes, not the loads, bound them)
template <typename C>
__device__ __forceinline__ void twid3(const C* __restrict__ tw, int tw_log2, int log2L, uint32_t j, C& w1, C& w2,
                                      C& w3) {
  w1 = twid(tw, tw_log2, log2L, j);
  if constexpr (sizeof(C) == 8) {   // float2
    w2 = cmul(w1, w1);
    w3 = cmul(w1, w2);
  } else {
    w2 = twid(tw, tw_log2, log2L, 2 * j);
    w3 = twid(tw, tw_log2, log2L, 3 * j);
  }
}

// one radix-4 DIF butterfly (two radix-2 levels) in registers: block 2^lgb, position j of the first value
template <typename C>
__device__ __forceinline__ void r4_dif(C& a0, C& a1, C& a2, C& a3, uint32_t j, int lgb, const C* __restrict__ tw,
                                       int tw_log2) {
  const C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  const C id13 = cmuli(d13);
  a0 = cadd(s02, s13);
  if (j == 0) {
    a1 = csub(s02, s13);
    a2 = csub(d02, id13);
    a3 = cadd(d02, id13);
  } else {
    C w1, w2, w3;
    twid3(tw, tw_log2, lgb, j, w1, w2, w3);
    a1 = cmul(csub(s02, s13), w2);
    a2 = cmul(csub(d02, id13), w1);
    a3 = cmul(cadd(d02, id13), w3);
  }
}
// its adjoint (the radix-4 DIT butterfly with conjugate twiddles)
template <typename C>
__device__ __forceinline__ void r4_dit(C& a0, C& a1, C& a2, C& a3, uint32_t j, int lgb, const C* __restrict__ tw,
                                       int tw_log2) {
  C p1 = a1, p2 = a2, p3 = a3;
  if (j != 0) {
    C w1, w2, w3;
    twid3(tw, tw_log2, lgb, j, w1, w2, w3);
    p1 = cmulc(p1, w2);
    p2 = cmulc(p2, w1);
    p3 = cmulc(p3, w3);
  }
  const C a = cadd(a0, p1), bb = csub(a0, p1), sp = cadd(p2, p3), dp = cmuli(csub(p2, p3));
  a0 = cadd(a, sp);
  a2 = csub(a, sp);
  a1 = cadd(bb, dp);
  a3 = csub(bb, dp);
}

// Two consecutive radix-4 stages fused in registers: blocks of N = 2^lg and then their quarters.  A thread
// holds the 16 values x[u][t] at j2 + u N/4 + t N/16 of one block (j2 < N/16): the first stage's
// butterflies j2 + t N/16 (t < 4) act on x[.][t], the second stage's butterfly j2 of quarter u on x[u][.].
// The arithmetic is that of the two separate stages; one shared-memory round trip and barrier less.
// INV: the adjoint pair (quarters first, conjugate twiddles), as fft_dit_inv runs it.
template <typename C, bool INV>
__device__ void r16_stage(C* s, int log2L, int lgnlo, int nhi, int lg, const C* __restrict__ tw, int tw_log2) {
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  const int lg16 = lg - 4, lgg_line = log2L - 4;   // groups per block and per line
  const unsigned total = (unsigned)nhi << (lgnlo + lgg_line);
  const int q1 = 1 << (lg - 2 + lgnlo), q2 = 1 << (lg16 + lgnlo);
  for (unsigned b = threadIdx.x; b < total; b += nthr) {
    const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
    const unsigned r = rest & ((1u << lgg_line) - 1u), l_hi = rest >> lgg_line;
    const unsigned blk = r >> lg16, j2 = r & ((1u << lg16) - 1u);
    const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + ((blk << lg) << lgnlo) + (j2 << lgnlo));
    C x[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) x[u][t] = s[tpos<C>(e0 + u * q1 + t * q2)];
    if (!INV) {
#pragma unroll
      for (int t = 0; t < 4; ++t) r4_dif(x[0][t], x[1][t], x[2][t], x[3][t], j2 + ((uint32_t)t << lg16), lg, tw, tw_log2);
#pragma unroll
      for (int u = 0; u < 4; ++u) r4_dif(x[u][0], x[u][1], x[u][2], x[u][3], j2, lg - 2, tw, tw_log2);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) r4_dit(x[u][0], x[u][1], x[u][2], x[u][3], j2, lg - 2, tw, tw_log2);
#pragma unroll
      for (int t = 0; t < 4; ++t) r4_dit(x[0][t], x[1][t], x[2][t], x[3][t], j2 + ((uint32_t)t << lg16), lg, tw, tw_log2);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) s[tpos<C>(e0 + u * q1 + t * q2)] = x[u][t];
  }
  __syncthreads();
}

// ---------------------------------------------------------------- binary64: fused multiply-add butterflies
// The binary64 passes are bound by the binary64 arithmetic pipe, so their cost is the number of binary64
// instructions.  A twiddled radix-4 butterfly written as three complex products and sixteen additions takes
// 28 of them.  Taking the real (or imaginary) part of each twiddle out of its product as a common factor
// (Linzer and Feig's method, in the radix-4 arrangement Goedecker gave it) turns every product into the
// multiplier of a fused multiply-add: 22 instructions.  With b' = (b.x - tau b.y, b.y + tau b.x):
//   form A (Re w != 0): tau = Im w / Re w,   w b = Re w (b'.x, b'.y)
//   form B (Im w != 0): tau = -Re w / Im w,  w b = (-Im w b'.y, Im w b'.x)
// The butterfly's twiddles are w1 = W_N^j, w2 = w1^2, w3 = w1^3 with 0 <= j < N/4, so w1 and w3 are always
// in form A (their angles stay off pi/2 and 3 pi/2 for power-of-two N); w2 takes whichever form has the
// larger divisor.  Per twiddle index t (N = 2^tw_log2, t < N/4): t1 = tau(w1), t3 = tau(w3), tau2 = tau(w2),
// s1 = Re w1, sx2 (the first scale of w2 b; the second is sy2 = sx2 in form A, -sx2 in form B) and
// r = Re w3 / Re w1 with its lowest mantissa bit replaced by the form of w2 (1: form B; <= 1 ulp of r).
// Then w1 a + w3 b = s1 (a' + r b'), and every sum of a value and a scaled product is one fused multiply-add.
// Index 0 holds the identity twiddles (tau = 0, scales and r = 1), which reproduce the plain additions
// exactly, so no lane needs a branch of its own.
// Layout (lf): two copies of six arrays of n = max(N/4, 1) words, [t1 | t3 | tau2 | s1 | sx2 | r]; the first
// copy in natural order of t, the second in bit-reversed order (position u holds t = bitrev(u) over log2 n
// bits), so that lanes with neighbouring indices read neighbouring words in both transforms.
struct FmaTw {
  double t1, t3, tau2, s1, sx2, sy2, r;
  bool swap;
};
__device__ __forceinline__ FmaTw fma_tw(const double* __restrict__ base, int n, uint32_t e) {
  FmaTw w;
  w.t1 = __ldg(base + e);
  w.t3 = __ldg(base + n + e);
  w.tau2 = __ldg(base + 2 * n + e);
  w.s1 = __ldg(base + 3 * n + e);
  w.sx2 = __ldg(base + 4 * n + e);
  w.r = __ldg(base + 5 * n + e);
  w.swap = (__double_as_longlong(w.r) & 1) != 0;
  // sy2 = -sx2 in form B: a sign flip by integer operations (no binary64 instruction)
  w.sy2 = __longlong_as_double(__double_as_longlong(w.sx2) ^ ((long long)w.swap << 63));
  return w;
}
__device__ __forceinline__ int fma_tw_n(int tw_log2) { return tw_log2 >= 2 ? 1 << (tw_log2 - 2) : 1; }

// radix-4 decimation-in-time butterfly: a0..a3 at block positions j, j + N/4, j + N/2, j + 3N/4 of a block of
// N = 2^lg, twiddles w2, w1, w3 on a1, a2, a3 (INV: their conjugates, the inverse transform)
template <bool INV>
__device__ __forceinline__ void r4_plain(double2& a0, double2& a1, double2& a2, double2& a3) {
  const double2 A = cadd(a0, a1), B = csub(a0, a1), sp = cadd(a2, a3), dm = csub(a2, a3);
  a0 = cadd(A, sp);
  a2 = csub(A, sp);
  // forward: B -/+ i dm; inverse: B +/- i dm
  if (!INV) {
    a1 = make_double2(B.x + dm.y, B.y - dm.x);
    a3 = make_double2(B.x - dm.y, B.y + dm.x);
  } else {
    a1 = make_double2(B.x - dm.y, B.y + dm.x);
    a3 = make_double2(B.x + dm.y, B.y - dm.x);
  }
}
template <bool INV>
__device__ __forceinline__ void r4_fma(double2& a0, double2& a1, double2& a2, double2& a3, const FmaTw& w) {
  double Ax, Ay, Bx, By, X2, Y2, X3, Y3;
  if (!INV) {
    // w2 a1 = (sx2 P, sy2 Q)
    const double bx = fma(-w.tau2, a1.y, a1.x), by = fma(w.tau2, a1.x, a1.y);
    const double P = w.swap ? by : bx, Q = w.swap ? bx : by;
    Ax = fma(w.sx2, P, a0.x);
    Ay = fma(w.sy2, Q, a0.y);
    Bx = fma(-w.sx2, P, a0.x);
    By = fma(-w.sy2, Q, a0.y);
    X2 = fma(-w.t1, a2.y, a2.x);
    Y2 = fma(w.t1, a2.x, a2.y);
    X3 = fma(-w.t3, a3.y, a3.x);
    Y3 = fma(w.t3, a3.x, a3.y);
  } else {
    // conj(w2) a1 = conj(w2 conj(a1)) = (sx2 P, -sy2 Q)
    const double bx = fma(w.tau2, a1.y, a1.x), by = fma(w.tau2, a1.x, -a1.y);
    const double P = w.swap ? by : bx, Q = w.swap ? bx : by;
    Ax = fma(w.sx2, P, a0.x);
    Ay = fma(-w.sy2, Q, a0.y);
    Bx = fma(-w.sx2, P, a0.x);
    By = fma(w.sy2, Q, a0.y);
    X2 = fma(w.t1, a2.y, a2.x);
    Y2 = fma(-w.t1, a2.x, a2.y);
    X3 = fma(w.t3, a3.y, a3.x);
    Y3 = fma(-w.t3, a3.x, a3.y);
  }
  // w1 a2 +/- w3 a3 = s1 (SP or DM)
  const double SPx = fma(w.r, X3, X2), SPy = fma(w.r, Y3, Y2);
  const double DMx = fma(-w.r, X3, X2), DMy = fma(-w.r, Y3, Y2);
  a0 = make_double2(fma(w.s1, SPx, Ax), fma(w.s1, SPy, Ay));
  a2 = make_double2(fma(-w.s1, SPx, Ax), fma(-w.s1, SPy, Ay));
  if (!INV) {   // B -/+ i s1 DM
    a1 = make_double2(fma(w.s1, DMy, Bx), fma(-w.s1, DMx, By));
    a3 = make_double2(fma(-w.s1, DMy, Bx), fma(w.s1, DMx, By));
  } else {      // B +/- i s1 DM
    a1 = make_double2(fma(-w.s1, DMy, Bx), fma(w.s1, DMx, By));
    a3 = make_double2(fma(w.s1, DMy, Bx), fma(-w.s1, DMx, By));
  }
}
// the butterfly at slots i0..i3 of the tile: plain additions (blocks of 4, or twiddle index 0 where every
// lane of the warp has the same index), else the fused multiply-add form with twiddles w
template <bool INV>
__device__ __forceinline__ void r4_slots(double2* s, int i0, int i1, int i2, int i3, bool plain, const FmaTw& w) {
  double2 a0 = s[i0], a1 = s[i1], a2 = s[i2], a3 = s[i3];
  if (plain) r4_plain<INV>(a0, a1, a2, a3);
  else r4_fma<INV>(a0, a1, a2, a3, w);
  s[i0] = a0;
  s[i1] = a1;
  s[i2] = a2;
  s[i3] = a3;
}

// Stage plan shared by both binary64 transforms: an odd log2 length first takes one twiddle-free radix-2
// stage (span 1 of the bit-reversed-input algorithm), then radix-4 stages on blocks of 2^lg, lg = lg0 + 2,
// lg0 + 4, ..., log2L, one shared-memory round trip each.  The nhi line groups are nrep equal sets (the
// tensor components, outermost) with the same twiddles: a thread loads a butterfly's twiddles once and
// applies them in every set (nrep times fewer table loads).
//
// The inverse (bit-reversed in, natural out) is the decimation-in-time algorithm as it stands.  The forward
// transform (natural in, bit-reversed out) is the same algorithm with every memory position p relabelled
// bitrev(p): a butterfly of block 2^lg at (block b, position j) moves to group G = bitrev(j) and offset
// i = bitrev(b) of span H = 2^(log2L - lg), its four values at G 4H + v H + i with v = bitrev2(u), and its
// twiddles stay those of j.  So both run twiddle-before-butterfly (decimation in time), the order the
// fused multiply-adds need, and the forward output is the bit-reversed spectrum the decimation-in-frequency
// kernels produce.
static __device__ void fft_fwd_fma(double2* s, int log2L, int lgnlo, int nhi, const double* __restrict__ lf, int tw_log2,
                                   int nrep) {
  if (log2L == 0) return;
  const int n = fma_tw_n(tw_log2);
  const int nh1 = nhi / nrep, rep_off = nh1 << (log2L + lgnlo);
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  const int lg0 = log2L & 1;
  if (lg0) {   // span L/2, no twiddles
    const int lgh = log2L - 1;
    const unsigned total = (unsigned)nhi << (lgnlo + lgh);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned k = rest & ((1u << lgh) - 1u), l_hi = rest >> lgh;
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + (k << lgnlo));
      const int i0 = tpos<double2>(e0), i1 = tpos<double2>(e0 + (int)((1u << lgh) << lgnlo));
      const double2 a = s[i0], c = s[i1];
      s[i0] = cadd(a, c);
      s[i1] = csub(a, c);
    }
    __syncthreads();
  }
  int lg = lg0 + 2;
  for (; lg <= log2L; lg += 2) {
    // block 2^lg relabelled: groups G of 4H values, H = 2^(log2L - lg); value u at G 4H + bitrev2(u) H + i.
    // Its twiddle index bitrev(G) over lg - 2 bits, shifted to the table's N, is bitrev(G) over log2 n bits:
    // position G of the bit-reversed table copy, the same at every stage
    const int lgH = log2L - lg, lgg = lg - 2;
    const unsigned total = (unsigned)nh1 << (lgnlo + log2L - 2);
    const bool uni = lgH + lgnlo >= 5;
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned i = rest & ((1u << lgH) - 1u), G = (rest >> lgH) & ((1u << lgg) - 1u);
      const unsigned l_hi = rest >> (log2L - 2);
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + (((G << (lgH + 2)) | i) << lgnlo));
      const int h = 1 << (lgH + lgnlo);
      const bool plain = lg == 2 || (uni && G == 0);
      FmaTw w = {};
      if (!plain) w = fma_tw(lf + 6 * n, n, G);
      for (int c = 0; c < nrep; ++c) {
        const int ec = e0 + c * rep_off;
        r4_slots<false>(s, tpos<double2>(ec), tpos<double2>(ec + 2 * h), tpos<double2>(ec + h),
                        tpos<double2>(ec + 3 * h), plain, w);
      }
    }
    __syncthreads();
  }
}

static __device__ void fft_inv_fma(double2* s, int log2L, int lgnlo, int nhi, const double* __restrict__ lf, int tw_log2,
                                   int nrep) {
  if (log2L == 0) return;
  const int n = fma_tw_n(tw_log2);
  const int nh1 = nhi / nrep, rep_off = nh1 << (log2L + lgnlo);
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  const int lg0 = log2L & 1;
  const bool uni = lgnlo >= 5;   // neighbouring lanes differ in the line, not in the block position
  if (lg0) {   // span 1, no twiddles
    const int lgh = log2L - 1;
    const unsigned total = (unsigned)nhi << (lgnlo + lgh);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned k = rest & ((1u << lgh) - 1u), l_hi = rest >> lgh;
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + ((2u * k) << lgnlo));
      const int i0 = tpos<double2>(e0), i1 = tpos<double2>(e0 + (1 << lgnlo));
      const double2 a = s[i0], c = s[i1];
      s[i0] = cadd(a, c);
      s[i1] = csub(a, c);
    }
    __syncthreads();
  }
  int lg = lg0 + 2;
  for (; lg <= log2L; lg += 2) {
    const int lgq = lg - 2;
    const unsigned total = (unsigned)nh1 << (lgnlo + log2L - 2);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned j = rest & ((1u << lgq) - 1u), blk = (rest >> lgq) & ((1u << (log2L - lg)) - 1u);
      const unsigned l_hi = rest >> (log2L - 2);
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + ((((blk << lg) | j)) << lgnlo));
      const int q = 1 << (lgq + lgnlo);
      const bool plain = lg == 2 || (uni && j == 0);
      FmaTw w = {};
      if (!plain) w = fma_tw(lf, n, j << (tw_log2 - lg));
      for (int c = 0; c < nrep; ++c) {
        const int ec = e0 + c * rep_off;
        r4_slots<true>(s, tpos<double2>(ec), tpos<double2>(ec + q), tpos<double2>(ec + 2 * q),
                       tpos<double2>(ec + 3 * q), plain, w);
      }
    }
    __syncthreads();
  }
}

// Forward DIF FFT (sign -1, unnormalized) of nhi * nlo lines of length 2^log2L, nlo = 2^lgnlo.
// Output in bit-reversed order.  Must be called by all threads of the block.
// FUSE: run pairs of radix-4 stages in registers (r16_stage), as the binary32 kernels do.
// nrep (binary64 only): the lines form nrep equal sets, outermost, that share their twiddles.
// Binary64 (C = double2) runs fft_fwd_fma with the fused multiply-add table lf instead (FUSE unused).
template <typename C, bool FUSE = (sizeof(C) == 8)>
__device__ void fft_dif(C* s, int log2L, int lgnlo, int nhi, const C* __restrict__ tw, int tw_log2,
                        const double* __restrict__ lf, int nrep = 1) {
  if constexpr (std::is_same<C, double2>::value) {
    fft_fwd_fma(s, log2L, lgnlo, nhi, lf, tw_log2, nrep);
    return;
  }
  if (log2L == 0) return;
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  int lg = log2L;  // log2 of current block size N
  if (lg & 1) {    // one radix-2 stage on the full length
    const int lgh = log2L - 1;
    const unsigned total = (unsigned)nhi << (lgnlo + lgh);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned j = rest & ((1u << lgh) - 1u), l_hi = rest >> lgh;
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + (j << lgnlo));
      const int i0 = tpos<C>(e0), i1 = tpos<C>(e0 + (int)((1u << lgh) << lgnlo));
      const C a = s[i0], c = s[i1];
      s[i0] = cadd(a, c);
      s[i1] = cmul(csub(a, c), twid(tw, tw_log2, log2L, j));
    }
    __syncthreads();
    lg -= 1;
  }
  // pairs of radix-4 stages fused in registers while at least two remain (16 complex values per thread)
  if constexpr (FUSE)
    for (; lg >= 4; lg -= 4) r16_stage<C, false>(s, log2L, lgnlo, nhi, lg, tw, tw_log2);
  const int lgq_line = log2L - 2;  // radix-4 butterflies per line = L/4
  for (; lg >= 2; lg -= 2) {
    const int lgq = lg - 2;
    const unsigned total = (unsigned)nhi << (lgnlo + lgq_line);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned r = rest & ((1u << lgq_line) - 1u), l_hi = rest >> lgq_line;
      const unsigned blk = r >> lgq, j = r & ((1u << lgq) - 1u);
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + ((blk << lg) << lgnlo) + (j << lgnlo));
      const int q = (int)(1u << (lgq + lgnlo));
      const int i0 = tpos<C>(e0), i1 = tpos<C>(e0 + q), i2 = tpos<C>(e0 + 2 * q), i3 = tpos<C>(e0 + 3 * q);
      const C x0 = s[i0], x1 = s[i1], x2 = s[i2], x3 = s[i3];
      const C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
      const C id13 = cmuli(d13);
      s[i0] = cadd(s02, s13);
      if (j == 0) {  // all three twiddles are 1
        s[i1] = csub(s02, s13);
        s[i2] = csub(d02, id13);
        s[i3] = cadd(d02, id13);
      } else {
        C w1, w2, w3;
        twid3(tw, tw_log2, lg, j, w1, w2, w3);
        s[i1] = cmul(csub(s02, s13), w2);
        s[i2] = cmul(csub(d02, id13), w1);
        s[i3] = cmul(cadd(d02, id13), w3);
      }
    }
    __syncthreads();
  }
}

// Inverse DIT FFT (sign +1, unnormalized): the adjoint of fft_dif.
// Input in bit-reversed order, output natural.  All threads must call.
// Binary64 runs fft_inv_fma (same result up to rounding).
template <typename C, bool FUSE = (sizeof(C) == 8)>
__device__ void fft_dit_inv(C* s, int log2L, int lgnlo, int nhi, const C* __restrict__ tw, int tw_log2,
                            const double* __restrict__ lf, int nrep = 1) {
  if constexpr (std::is_same<C, double2>::value) {
    fft_inv_fma(s, log2L, lgnlo, nhi, lf, tw_log2, nrep);
    return;
  }
  if (log2L == 0) return;
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  const int lgq_line = log2L - 2;
  // the DIF ran its radix-4 stages on block sizes 2^(log2L - (log2L&1)) ... 4; mirror them: a lone
  // smallest stage when their number is odd, then pairs fused in registers (adjoint order inside a pair)
  const int lgmax = log2L - (log2L & 1);
  const int lone = FUSE ? (((lgmax / 2) & 1) ? 2 : 0) : lgmax;
  for (int lg = 2; lg <= lone; lg += 2) {
    const int lgq = lg - 2;
    const unsigned total = (unsigned)nhi << (lgnlo + lgq_line);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned r = rest & ((1u << lgq_line) - 1u), l_hi = rest >> lgq_line;
      const unsigned blk = r >> lgq, j = r & ((1u << lgq) - 1u);
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + ((blk << lg) << lgnlo) + (j << lgnlo));
      const int q = (int)(1u << (lgq + lgnlo));
      const int i0 = tpos<C>(e0), i1 = tpos<C>(e0 + q), i2 = tpos<C>(e0 + 2 * q), i3 = tpos<C>(e0 + 3 * q);
      const C c0 = s[i0];
      C p1 = s[i1], p2 = s[i2], p3 = s[i3];
      if (j != 0) {  // conj twiddles u^2, u^1, u^3 with u = conj(W_N^j)
        C w1, w2, w3;
        twid3(tw, tw_log2, lg, j, w1, w2, w3);
        p1 = cmulc(p1, w2);
        p2 = cmulc(p2, w1);
        p3 = cmulc(p3, w3);
      }
      const C a = cadd(c0, p1), bb = csub(c0, p1), sp = cadd(p2, p3), dp = cmuli(csub(p2, p3));
      s[i0] = cadd(a, sp);
      s[i2] = csub(a, sp);
      s[i1] = cadd(bb, dp);
      s[i3] = csub(bb, dp);
    }
    __syncthreads();
  }
  if constexpr (FUSE)
    for (int lg = lone + 4; lg <= lgmax; lg += 4) r16_stage<C, true>(s, log2L, lgnlo, nhi, lg, tw, tw_log2);
  if (log2L & 1) {   // adjoint of the leading radix-2 stage, applied last
    const int lgh = log2L - 1;
    const unsigned total = (unsigned)nhi << (lgnlo + lgh);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned j = rest & ((1u << lgh) - 1u), l_hi = rest >> lgh;
      const int e0 = (int)(((l_hi << (log2L + lgnlo)) | l_lo) + (j << lgnlo));
      const int i0 = tpos<C>(e0), i1 = tpos<C>(e0 + (int)((1u << lgh) << lgnlo));
      const C a = s[i0];
      const C c = cmulc(s[i1], twid(tw, tw_log2, log2L, j));
      s[i0] = cadd(a, c);
      s[i1] = csub(a, c);
    }
    __syncthreads();
  }
}
