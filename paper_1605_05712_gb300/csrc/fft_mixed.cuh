// fft_mixed.cuh -- mixed-radix FFT of lines held in shared memory, natural order in and out.
//
// Sec. 2.2 of arXiv 1605.05712: the pattern DFT is an ordinary d_M-dimensional DFT over the elementary
// divisors e_j of M, whatever they are.  The power-of-two kernels (fft_smem.cuh) cover divisors 2^k;
// these stages cover every other length L = r_1 r_2 ... r_t (radix 4, 2, 3, 5 as register butterflies,
// any other prime p as a direct p-point DFT of O(p) work per output).
//
// Stockham autosort form (derived for this file): after s stages the buffer holds, at p * M + q,
//   X_s[p][q] = sum_{n < L_s} x[q + n M] W_{L_s}^{n p},   L_s = r_1 ... r_s,  M = L / L_s,
// so X_0 = x and X_t = DFT(x) in natural order.  A stage of radix r (L' = L_s r, M' = M / r) reads
//   X_s[p][q' + j M'] (j < r), multiplies by W_{L'}^{j p} = W_L^{j p M'} and writes the r-point DFT of
// those values to X_{s+1}[p + L_s k][q'] (k < r).  Each stage reads one buffer and writes the other
// (ping-pong), separated by __syncthreads(); the inverse uses the conjugate roots (no scaling).
//
// Line addressing as in fft_smem.cuh: w (a power of two) interleaved lines per group, so element p of
// line (lh, ll) is at lh * L * w + p * w + ll; rows use w = 1, column tiles w = tile width.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_smem.cuh"

// W_L^t (or its conjugate for the inverse) from the axis table of W_L^t, t < L
template <typename C, bool INV>
__device__ __forceinline__ C mroot(const C* __restrict__ tw, int t) {
  const C w = ldg_c(tw + t);
  return INV ? cconj(w) : w;
}

// one radix-r butterfly: inputs x[in0 + j * in_step] (j < r) times W_L^{j p M'}, outputs y[out0 + k * out_step]
template <typename C, bool INV>
__device__ __forceinline__ void mixed_butterfly(const C* x, C* y, int r, int L, int in0, int in_step, int out0,
                                                int out_step, int tstep, const C* __restrict__ tw) {
  // tstep = p M': the twiddle of input j is W_L^{j tstep} (j tstep < L)
  if (r == 2) {
    const C a0 = x[in0];
    C a1 = x[in0 + in_step];
    if (tstep) a1 = cmul(a1, mroot<C, INV>(tw, tstep));
    y[out0] = cadd(a0, a1);
    y[out0 + out_step] = csub(a0, a1);
  } else if (r == 4) {
    const C a0 = x[in0];
    C a1 = x[in0 + in_step], a2 = x[in0 + 2 * in_step], a3 = x[in0 + 3 * in_step];
    if (tstep) {
      a1 = cmul(a1, mroot<C, INV>(tw, tstep));
      a2 = cmul(a2, mroot<C, INV>(tw, 2 * tstep));
      a3 = cmul(a3, mroot<C, INV>(tw, 3 * tstep));
    }
    const C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    const C id13 = cmuli(d13);
    y[out0] = cadd(s02, s13);
    y[out0 + 2 * out_step] = csub(s02, s13);
    // forward root W_4 = -i: y1 = d02 - i d13; the inverse flips the sign of i
    y[out0 + out_step] = INV ? cadd(d02, id13) : csub(d02, id13);
    y[out0 + 3 * out_step] = INV ? csub(d02, id13) : cadd(d02, id13);
  } else if (r == 3) {
    const C a0 = x[in0];
    C a1 = x[in0 + in_step], a2 = x[in0 + 2 * in_step];
    if (tstep) {
      a1 = cmul(a1, mroot<C, INV>(tw, tstep));
      a2 = cmul(a2, mroot<C, INV>(tw, 2 * tstep));
    }
    const C w3 = mroot<C, INV>(tw, L / 3);            // W_3 (conjugated for the inverse)
    const C s = cadd(a1, a2), d = csub(a1, a2);
    const C t = cadd(a0, cscale(s, w3.x));
    const C u = cmuli(cscale(d, w3.y));
    y[out0] = cadd(a0, s);
    y[out0 + out_step] = cadd(t, u);
    y[out0 + 2 * out_step] = csub(t, u);
  } else if (r == 5) {
    const C a0 = x[in0];
    C a1 = x[in0 + in_step], a2 = x[in0 + 2 * in_step], a3 = x[in0 + 3 * in_step], a4 = x[in0 + 4 * in_step];
    if (tstep) {
      a1 = cmul(a1, mroot<C, INV>(tw, tstep));
      a2 = cmul(a2, mroot<C, INV>(tw, 2 * tstep));
      a3 = cmul(a3, mroot<C, INV>(tw, 3 * tstep));
      a4 = cmul(a4, mroot<C, INV>(tw, 4 * tstep));
    }
    const C c1 = mroot<C, INV>(tw, L / 5), c2 = mroot<C, INV>(tw, 2 * (L / 5));   // W_5, W_5^2
    const C s1 = cadd(a1, a4), d1 = csub(a1, a4), s2 = cadd(a2, a3), d2 = csub(a2, a3);
    // y_1, y_4 = a0 + c1x s1 + c2x s2 +- i (c1y d1 + c2y d2);  y_2, y_3 = a0 + c2x s1 + c1x s2 +- i (c2y d1 - c1y d2)
    const C A1 = cadd(a0, cadd(cscale(s1, c1.x), cscale(s2, c2.x)));
    const C B1 = cmuli(cadd(cscale(d1, c1.y), cscale(d2, c2.y)));
    const C A2 = cadd(a0, cadd(cscale(s1, c2.x), cscale(s2, c1.x)));
    const C B2 = cmuli(csub(cscale(d1, c2.y), cscale(d2, c1.y)));
    y[out0] = cadd(a0, cadd(s1, s2));
    y[out0 + out_step] = cadd(A1, B1);
    y[out0 + 4 * out_step] = csub(A1, B1);
    y[out0 + 2 * out_step] = cadd(A2, B2);
    y[out0 + 3 * out_step] = csub(A2, B2);
  } else {
    // any other radix: the r-point DFT term by term, roots W_r^{jk} = W_L^{(jk mod r) L / r}
    const int Lr = L / r;
    for (int k = 0; k < r; ++k) {
      C acc = x[in0];
      int jk = 0;
      for (int j = 1; j < r; ++j) {
        jk += k;
        if (jk >= r) jk -= r;
        C a = x[in0 + j * in_step];
        if (tstep) a = cmul(a, mroot<C, INV>(tw, j * tstep));
        acc = cadd(acc, cmul(a, mroot<C, INV>(tw, jk * Lr)));
      }
      y[out0 + k * out_step] = acc;
    }
  }
}

// Transform nhi groups of w (= 2^lgw) interleaved lines of length L with the radices rad[0..nst).  Reads
// x, ping-pongs through y; returns the buffer that holds the result (x if nst is even, else y).  All
// threads of the block must call; the buffers are published on return.
template <typename C, bool INV>
__device__ C* fft_mixed(C* x, C* y, int L, const uint16_t* rad, int nst, int lgw, int nhi,
                        const C* __restrict__ tw) {
  const int w = 1 << lgw;
  int M = L, Lc = 1;
  for (int s = 0; s < nst; ++s) {
    const int r = rad[s];
    const int Mn = M / r, nb = L / r;
    const int total = (nhi * nb) << lgw;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int ll = b & (w - 1), rest = b >> lgw;
      const int lh = rest / nb, bf = rest - lh * nb;
      const int p = bf / Mn, q = bf - p * Mn;
      const int base = lh * L * w + ll;
      mixed_butterfly<C, INV>(x, y, r, L, base + (p * M + q) * w, Mn * w, base + (p * Mn + q) * w, Lc * Mn * w,
                              p * Mn, tw);
    }
    __syncthreads();
    C* t = x;
    x = y;
    y = t;
    M = Mn;
    Lc *= r;
  }
  return x;
}
