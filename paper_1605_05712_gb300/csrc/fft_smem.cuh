// fft_smem.cuh -- in-place shared-memory FFT stages for the pattern FFT (sm_103a).
//
// The pattern FFT of Sec. 2.2 is an ordinary d_M-dimensional DFT over the
// elementary divisors; every 1-D piece of it runs here on lines held in
// shared memory.  Forward transforms are decimation-in-frequency (Sande-Tukey)
// and leave the spectrum in bit-reversed order; inverse transforms are the
// exact adjoint (decimation-in-time) and take bit-reversed input to natural
// output.  Forward -> pointwise Green operator -> inverse therefore needs no
// permutation pass: the pointwise step decodes each frequency with __brev.
//
// Radix-4 stages are two radix-2 DIF stages fused (so the order stays plain
// bit reversal); an odd log2 length adds one radix-2 stage.  Butterflies are
// in place, a thread keeps only the 4 values of the butterfly it is working
// on, and stages are separated by __syncthreads().
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

// Forward DIF FFT (sign -1, unnormalized) of nhi * nlo lines of length 2^log2L, nlo = 2^lgnlo.
// Output in bit-reversed order.  Must be called by all threads of the block.
// FUSE: run pairs of radix-4 stages in registers (r16_stage); binary32 kernels always, the 16-byte types
// where the kernel's register budget holds 16 complex values (the six-component passes, 128 registers)
template <typename C, bool FUSE = (sizeof(C) == 8)>
__device__ void fft_dif(C* s, int log2L, int lgnlo, int nhi, const C* __restrict__ tw, int tw_log2) {
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
template <typename C, bool FUSE = (sizeof(C) == 8)>
__device__ void fft_dit_inv(C* s, int log2L, int lgnlo, int nhi, const C* __restrict__ tw, int tw_log2) {
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
