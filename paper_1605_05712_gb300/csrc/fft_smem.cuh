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
// Line addressing: a line l = l_hi * nlo + l_lo has its element idx at
//   l_hi * L * nlo + idx * nlo + l_lo,
// which covers contiguous rows (nlo = 1) and tiles of columns (nlo = tile
// width x inner axes) alike.  Butterfly numbering puts l_lo fastest, so
// neighbouring threads touch neighbouring shared-memory words.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };

template <typename C> __device__ __forceinline__ C cmake(double x, double y);
template <> __device__ __forceinline__ double2 cmake<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 cmake<float2>(double x, double y) { return make_float2((float)x, (float)y); }

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
  return __ldg(&tw[j << (tw_log2 - log2L)]);
}

// Forward DIF FFT (sign -1, unnormalized) of nhi * nlo lines of length 2^log2L.
// Output in bit-reversed order.  Must be called by all threads of the block.
template <typename C>
__device__ void fft_dif(C* s, int log2L, int nlo, int nhi, const C* __restrict__ tw, int tw_log2) {
  if (log2L == 0) return;
  const int L = 1 << log2L;
  const int nthr = blockDim.x;
  int lg = log2L;  // log2 of current block size N
  if (lg & 1) {    // one radix-2 stage on the full length
    const int half = L >> 1;
    const long total = (long)nhi * nlo * half;
    for (long b = threadIdx.x; b < total; b += nthr) {
      int l_lo = (int)(b % nlo);
      long rest = b / nlo;
      int j = (int)(rest % half);
      int l_hi = (int)(rest / half);
      C* base = s + (long)l_hi * L * nlo + l_lo;
      C a = base[(long)j * nlo], c = base[(long)(j + half) * nlo];
      C w = twid(tw, tw_log2, log2L, j);
      base[(long)j * nlo] = cadd(a, c);
      base[(long)(j + half) * nlo] = cmul(csub(a, c), w);
    }
    __syncthreads();
    lg -= 1;
  }
  for (; lg >= 2; lg -= 2) {
    const int N = 1 << lg, q = N >> 2;
    const long per_line = L >> 2;
    const long total = (long)nhi * nlo * per_line;
    for (long b = threadIdx.x; b < total; b += nthr) {
      int l_lo = (int)(b % nlo);
      long rest = b / nlo;
      int r = (int)(rest % per_line);
      int l_hi = (int)(rest / per_line);
      int blk = r >> (lg - 2), j = r & (q - 1);
      C* base = s + (long)l_hi * L * nlo + l_lo + (long)blk * N * nlo;
      C x0 = base[(long)j * nlo], x1 = base[(long)(j + q) * nlo];
      C x2 = base[(long)(j + 2 * q) * nlo], x3 = base[(long)(j + 3 * q) * nlo];
      C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
      C w1 = twid(tw, tw_log2, lg, j), w2 = twid(tw, tw_log2, lg, 2 * j), w3 = twid(tw, tw_log2, lg, 3 * j);
      C id13 = cmuli(d13);
      base[(long)j * nlo] = cadd(s02, s13);
      base[(long)(j + q) * nlo] = cmul(csub(s02, s13), w2);
      base[(long)(j + 2 * q) * nlo] = cmul(csub(d02, id13), w1);
      base[(long)(j + 3 * q) * nlo] = cmul(cadd(d02, id13), w3);
    }
    __syncthreads();
  }
}

// Inverse DIT FFT (sign +1, unnormalized): the adjoint of fft_dif.
// Input in bit-reversed order, output natural.  All threads must call.
template <typename C>
__device__ void fft_dit_inv(C* s, int log2L, int nlo, int nhi, const C* __restrict__ tw, int tw_log2) {
  if (log2L == 0) return;
  const int L = 1 << log2L;
  const int nthr = blockDim.x;
  // the DIF ran its radix-4 stages on block sizes 2^(log2L - (log2L&1)) ... 4; mirror them
  const int lgmax = log2L - (log2L & 1);
  for (int lg = 2; lg <= lgmax; lg += 2) {
    const int N = 1 << lg, q = N >> 2;
    const long per_line = L >> 2;
    const long total = (long)nhi * nlo * per_line;
    for (long b = threadIdx.x; b < total; b += nthr) {
      int l_lo = (int)(b % nlo);
      long rest = b / nlo;
      int r = (int)(rest % per_line);
      int l_hi = (int)(rest / per_line);
      int blk = r >> (lg - 2), j = r & (q - 1);
      C* base = s + (long)l_hi * L * nlo + l_lo + (long)blk * N * nlo;
      C c0 = base[(long)j * nlo], c1 = base[(long)(j + q) * nlo];
      C c2 = base[(long)(j + 2 * q) * nlo], c3 = base[(long)(j + 3 * q) * nlo];
      // conj twiddles: u^1, u^2, u^3 with u = conj(W_N^j)
      C p1 = cmulc(c1, twid(tw, tw_log2, lg, 2 * j));
      C p2 = cmulc(c2, twid(tw, tw_log2, lg, j));
      C p3 = cmulc(c3, twid(tw, tw_log2, lg, 3 * j));
      C a = cadd(c0, p1), bb = csub(c0, p1), sp = cadd(p2, p3), dp = cmuli(csub(p2, p3));
      base[(long)j * nlo] = cadd(a, sp);
      base[(long)(j + 2 * q) * nlo] = csub(a, sp);
      base[(long)(j + q) * nlo] = cadd(bb, dp);
      base[(long)(j + 3 * q) * nlo] = csub(bb, dp);
    }
    __syncthreads();
  }
  if (log2L & 1) {   // adjoint of the leading radix-2 stage, applied last
    const int half = L >> 1;
    const long total = (long)nhi * nlo * half;
    for (long b = threadIdx.x; b < total; b += nthr) {
      int l_lo = (int)(b % nlo);
      long rest = b / nlo;
      int j = (int)(rest % half);
      int l_hi = (int)(rest / half);
      C* base = s + (long)l_hi * L * nlo + l_lo;
      C a = base[(long)j * nlo];
      C c = cmulc(base[(long)(j + half) * nlo], twid(tw, tw_log2, log2L, j));
      base[(long)j * nlo] = cadd(a, c);
      base[(long)(j + half) * nlo] = csub(a, c);
    }
    __syncthreads();
  }
}
