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
// width x inner axes) alike.  Butterfly numbering puts l_lo fastest, so
// neighbouring threads touch neighbouring shared-memory words.
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

// Forward DIF FFT (sign -1, unnormalized) of nhi * nlo lines of length 2^log2L, nlo = 2^lgnlo.
// Output in bit-reversed order.  Must be called by all threads of the block.
template <typename C>
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
      C* base = s + ((l_hi << (log2L + lgnlo)) | l_lo);
      C* p0 = base + (j << lgnlo);
      C* p1 = base + ((j + (1u << lgh)) << lgnlo);
      const C a = *p0, c = *p1;
      *p0 = cadd(a, c);
      *p1 = cmul(csub(a, c), twid(tw, tw_log2, log2L, j));
    }
    __syncthreads();
    lg -= 1;
  }
  const int lgq_line = log2L - 2;  // radix-4 butterflies per line = L/4
  for (; lg >= 2; lg -= 2) {
    const int lgq = lg - 2;
    const unsigned total = (unsigned)nhi << (lgnlo + lgq_line);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned r = rest & ((1u << lgq_line) - 1u), l_hi = rest >> lgq_line;
      const unsigned blk = r >> lgq, j = r & ((1u << lgq) - 1u);
      C* base = s + ((l_hi << (log2L + lgnlo)) | l_lo) + ((blk << lg) << lgnlo);
      C* p0 = base + (j << lgnlo);
      const unsigned q = 1u << (lgq + lgnlo);
      const C x0 = p0[0], x1 = p0[q], x2 = p0[2 * q], x3 = p0[3 * q];
      const C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
      const C id13 = cmuli(d13);
      p0[0] = cadd(s02, s13);
      if (j == 0) {  // all three twiddles are 1
        p0[q] = csub(s02, s13);
        p0[2 * q] = csub(d02, id13);
        p0[3 * q] = cadd(d02, id13);
      } else {
        C w1, w2, w3;
        twid3(tw, tw_log2, lg, j, w1, w2, w3);
        p0[q] = cmul(csub(s02, s13), w2);
        p0[2 * q] = cmul(csub(d02, id13), w1);
        p0[3 * q] = cmul(cadd(d02, id13), w3);
      }
    }
    __syncthreads();
  }
}

// Inverse DIT FFT (sign +1, unnormalized): the adjoint of fft_dif.
// Input in bit-reversed order, output natural.  All threads must call.
template <typename C>
__device__ void fft_dit_inv(C* s, int log2L, int lgnlo, int nhi, const C* __restrict__ tw, int tw_log2) {
  if (log2L == 0) return;
  const unsigned nthr = blockDim.x, nlo_m = (1u << lgnlo) - 1u;
  const int lgq_line = log2L - 2;
  // the DIF ran its radix-4 stages on block sizes 2^(log2L - (log2L&1)) ... 4; mirror them
  const int lgmax = log2L - (log2L & 1);
  for (int lg = 2; lg <= lgmax; lg += 2) {
    const int lgq = lg - 2;
    const unsigned total = (unsigned)nhi << (lgnlo + lgq_line);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned r = rest & ((1u << lgq_line) - 1u), l_hi = rest >> lgq_line;
      const unsigned blk = r >> lgq, j = r & ((1u << lgq) - 1u);
      C* base = s + ((l_hi << (log2L + lgnlo)) | l_lo) + ((blk << lg) << lgnlo);
      C* p0 = base + (j << lgnlo);
      const unsigned q = 1u << (lgq + lgnlo);
      const C c0 = p0[0];
      C p1 = p0[q], p2 = p0[2 * q], p3 = p0[3 * q];
      if (j != 0) {  // conj twiddles u^2, u^1, u^3 with u = conj(W_N^j)
        C w1, w2, w3;
        twid3(tw, tw_log2, lg, j, w1, w2, w3);
        p1 = cmulc(p1, w2);
        p2 = cmulc(p2, w1);
        p3 = cmulc(p3, w3);
      }
      const C a = cadd(c0, p1), bb = csub(c0, p1), sp = cadd(p2, p3), dp = cmuli(csub(p2, p3));
      p0[0] = cadd(a, sp);
      p0[2 * q] = csub(a, sp);
      p0[q] = cadd(bb, dp);
      p0[3 * q] = csub(bb, dp);
    }
    __syncthreads();
  }
  if (log2L & 1) {   // adjoint of the leading radix-2 stage, applied last
    const int lgh = log2L - 1;
    const unsigned total = (unsigned)nhi << (lgnlo + lgh);
    for (unsigned b = threadIdx.x; b < total; b += nthr) {
      const unsigned l_lo = b & nlo_m, rest = b >> lgnlo;
      const unsigned j = rest & ((1u << lgh) - 1u), l_hi = rest >> lgh;
      C* base = s + ((l_hi << (log2L + lgnlo)) | l_lo);
      C* p0 = base + (j << lgnlo);
      C* p1 = base + ((j + (1u << lgh)) << lgnlo);
      const C a = *p0;
      const C c = cmulc(*p1, twid(tw, tw_log2, log2L, j));
      *p0 = cadd(a, c);
      *p1 = csub(a, c);
    }
    __syncthreads();
  }
}
