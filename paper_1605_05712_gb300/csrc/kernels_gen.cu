// kernels_gen.cu -- the Basic Scheme iteration on lattices whose elementary divisors are not all powers of
// two (Sec. 2.2: the pattern DFT is the d_M-dimensional DFT over the divisors e_j, for every regular M).
//
// Same pass structure as kernels.cu, with mixed-radix transforms (fft_mixed.cuh) in natural order and
// the full complex spectrum (no real-to-complex packing: a row of odd length has no half-length
// complex form).  Per item the spectrum T holds n_c planes of m complex values in spectral order, the
// row axis last.  One iteration of Algorithm 1 (Sec. 3.2):
//   gen_row_kernel : inverse FFT of the previous spectrum along the row -> eps^(n+1) (its real part),
//                    Cauchy residual (Sec. 5.2) against eps^(n), eps written, polarization
//                    tau = (C_y - C0) : eps, forward FFT along the row (Green operator here when the row
//                    is the only axis);
//   gen_col_kernel : one logical axis per launch on tiles of columns: four-step twiddle, forward FFT,
//                    the Green operator (axis 0), inverse FFT, inverse twiddle.
// Binary64, double-float pairs and binary32 (the mixed path: increment form on a strain held as pairs, and
// its binary64-accurate restart on pairs, as the power-of-two kernels do it).
#include <math.h>

#include <algorithm>

#include "fft_mixed.cuh"
#include "kernels_dev.cuh"

// strain slot of one point: binary64, or a double-float pair (hi, lo) during a pair or mixed solve
template <typename Real>
__device__ __forceinline__ Real eps_ld1(const double* p) {
  if constexpr (is_df<Real>) {
    const float2 o = *(const float2*)p;
    return dfloat(o.x, o.y);
  } else if constexpr (is_f32<Real>) {
    const float2 o = *(const float2*)p;
    return o.x + o.y;
  } else {
    return *p;
  }
}
// per-precision copies of the item's tables: binary64, binary32 (mixed) or pairs
template <typename Real>
__device__ __forceinline__ const Real* tab_of(const double* d, const float* f, const dfloat* df) {
  if constexpr (is_df<Real>) return (const Real*)df;
  else if constexpr (is_f32<Real>) return (const Real*)f;
  else return (const Real*)d;
}
template <typename Real>
__device__ __forceinline__ void eps_st1(double* p, Real v) {
  if constexpr (is_df<Real>) *(float2*)p = make_float2(v.hi, v.lo);
  else *p = v;
}

// the two-level table of W_e^j of the four-step split: W_e^{(j >> s) << s} W_e^{j & (2^s - 1)}
template <typename C>
__device__ __forceinline__ C gen_split_tw(const LatDev& dv, int64_t j) {
  const C* st = (const C*)dv.stw;
  const int sh = dv.split_lo_log2;
  return cmul(ldg_c(st + (j >> sh)), ldg_c(st + dv.stw_hi_n + (j & ((int64_t(1) << sh) - 1))));
}

// ------------------------------------------------------------------ row pass
template <typename Real, int NC>
__global__ void __launch_bounds__(256) gen_row_kernel(LatDev dv, RowArgs a) {
  typedef typename cplx_of<Real>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n_c = NC, D = (NC == 6) ? 3 : 2;
  const int R = dv.Rlen, rpc = a.rpc, nlines = n_c * rpc;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const bool update = (a.flags & ROW_UPDATE) != 0;
  if (a.flags & ROW_ONLY_PAUSED) {   // the restart passes of a mixed solve (pairs)
    if (*(volatile const int*)&isc->done != ITEM_PAUSED) return;
  } else if (update && *(volatile const int*)&isc->done != ITEM_ACTIVE) {
    return;   // finished (or paused) earlier
  }
  C* buf0 = (C*)smem_raw;
  C* buf1 = buf0 + (size_t)nlines * R;
  double* red = (double*)(buf1 + (size_t)nlines * R);
  __shared__ int s_last;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t m = dv.m, r0 = (int64_t)blockIdx.x * rpc;
  C* T = (C*)a.T + item_i * a.t_stride;
  const int ra = dv.nax - 1;
  const C* tw = (const C*)dv.tw + dv.ax_twoff[ra];
  double* eps = item->eps;
  const uint8_t* phase = item->phase;
  C* cur = buf0;
  if (a.flags & ROW_LOAD_EPS) {
    for (int idx = tid; idx < nlines * R; idx += nthr) {
      const int line = idx / R, n = idx - line * R;
      const int c = line / rpc, row = line - c * rpc;
      buf0[idx] = cpair<C>(eps_ld1<Real>(eps + (c * m + (r0 + row) * R + n)), Real(0));
    }
    __syncthreads();
  } else {
    for (int idx = tid; idx < nlines * R; idx += nthr) {
      const int line = idx / R, n = idx - line * R;
      const int c = line / rpc, row = line - c * rpc;
      cp_async_elem(buf0 + idx, T + (c * m + (r0 + row) * R + n));
    }
    cp_async_wait_all();
    __syncthreads();
    cur = fft_mixed<C, true>(buf0, buf1, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, nlines, tw);
  }
  C* other = (cur == buf0) ? buf1 : buf0;
  // pointwise: update, residual, polarization (the inverse transform's real part is eps^(n+1), or the
  // increment eps^(n+1) - eps^(n) in the binary32 increment form)
  constexpr bool DBL = std::is_same<Real, double>::value;
  const bool tau_of_delta = !DBL && update && (a.flags & (ROW_INCREMENT | ROW_TAU_DELTA)) != 0;
  const bool incr = !DBL && update && (a.flags & ROW_INCREMENT) != 0 &&
                    ((a.flags & ROW_INCR_FIRST) != 0 || *(volatile const int*)&isc->iter > 0);
  double dsum = 0.0;
  dfloat dd_acc(0.f, 0.f), dd_shear(0.f, 0.f);
  DF dfs = {0.f, 0.f}, dfs_shear = {0.f, 0.f};
  for (int idx = tid; idx < rpc * R; idx += nthr) {
    const int row = idx / R, n = idx - row * R;
    const int64_t g = (r0 + row) * R + n;
    Real e[NC];
#pragma unroll
    for (int c = 0; c < n_c; ++c) e[c] = cur[((size_t)c * rpc + row) * R + n].x;
    const bool field = (a.flags & ROW_FIELD) != 0;
    const int ph = field ? 0 : phase[g];
    if (!field && update && a.mat.scheme == LAT_SCHEME_EYRE_MILTON) {
      // the transform returned u = (C + C0) eps: eps = (C_p + C0)^{-1} u
      const Real* W = tab_of<Real>(item->Wtab, item->Wtab_f, item->Wtab_df) + ph * n_c * n_c;
      Real u[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) u[c] = e[c];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        Real t = Real(0);
#pragma unroll
        for (int q = 0; q < n_c; ++q) t += ldg_r(W + c * n_c + q) * u[q];
        e[c] = t;
      }
    }
    if (update) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        double* pe = eps + (c * m + g);
        if constexpr (is_f32<Real>) {
          // binary32: the strain is a double-float pair; no binary64 arithmetic
          float2 o = *(float2*)pe;
          float d;
          if (incr) {   // T carried the increment itself
            d = e[c];
            df_acc(o.x, o.y, d);
          } else {      // T carried the new strain
            d = df_diff(e[c], o.x, o.y);
            o = make_float2(e[c], 0.f);
          }
          *(float2*)pe = o;
          if (c >= D) df_add_sq(dfs_shear, d);
          else df_add_sq(dfs, d);
          if (tau_of_delta) e[c] = d;
        } else {
          const Real d = e[c] - eps_ld1<Real>(pe);
          if constexpr (is_df<Real>) {
            if (c >= D) df_acc_sq(dd_shear, d);
            else df_acc_sq(dd_acc, d);
          } else {
            dsum += (c >= D ? 2.0 : 1.0) * (d * d);
          }
          eps_st1<Real>(pe, e[c]);
          if (tau_of_delta) e[c] = d;   // the pair restart: polarization of the exact increment
        }
      }
    }
    if (field) {   // per-point stiffness field: tau = C_y : eps - C0 : eps
      const GreenK<Real> gk = green_consts<Real>(item, a.mat);
      Real t[NC];
      field_polarize<Real, NC>(tab_of<Real>(item->fld, item->fld_f, item->fld_df), m, g, gk.lam0, gk.mu0 + gk.mu0,
                               e, t);
#pragma unroll
      for (int c = 0; c < n_c; ++c) cur[((size_t)c * rpc + row) * R + n] = cpair<C>(t[c], Real(0));
      continue;
    }
    const Real* Dt = tab_of<Real>(item->Dtab, item->Dtab_f, item->Dtab_df) + ph * n_c * n_c;
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      Real t = Real(0);
#pragma unroll
      for (int q = 0; q < n_c; ++q) t += ldg_r(Dt + c * n_c + q) * e[q];
      cur[((size_t)c * rpc + row) * R + n] = cpair<C>(t, Real(0));
    }
  }
  __syncthreads();
  C* out = fft_mixed<C, false>(cur, other, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, nlines, tw);
  if (a.flags & ROW_GAMMA) {  // the row is the only logical axis: its spectrum is the whole spectrum
    const GreenK<Real> gk = green_consts<Real>(item, a.mat);
    for (int idx = tid; idx < rpc * R; idx += nthr) {
      const int row = idx / R, k = idx - row * R;
      C val[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) val[c] = out[((size_t)c * rpc + row) * R + k];
      int kk[LAT_MAX_AX] = {0};
      kk[ra] = k;
      green_at<Real, NC>(dv, a.mat, item, gk, kk, val);
#pragma unroll
      for (int c = 0; c < n_c; ++c) out[((size_t)c * rpc + row) * R + k] = val[c];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nlines * R; idx += nthr) {
    const int line = idx / R, n = idx - line * R;
    const int c = line / rpc, row = line - c * rpc;
    T[c * m + (r0 + row) * R + n] = out[idx];
  }
  if (!update) return;
  double* partials = a.it.partials + item_i * a.it.pstride;
  double tot;
  if constexpr (is_f32<Real>) {
    const dfloat pr = dfloat(dfs.hi, dfs.lo) + dfloat(2.f * dfs_shear.hi, 2.f * dfs_shear.lo);
    if (!item_reduce<1>(&pr, partials, isc, red, &s_last, &tot)) return;
  } else if constexpr (is_df<Real>) {
    const dfloat pr = dd_acc + (dd_shear + dd_shear);
    if (!item_reduce<1>(&pr, partials, isc, red, &s_last, &tot)) return;
  } else {
    if (!item_reduce<1>(&dsum, partials, isc, red, &s_last, &tot)) return;
  }
  if (tid == 0) item_report(sqrt(tot) / item->norm0, isc, item_i, a.it);
}

// ------------------------------------------------------------------ column pass (one logical axis)
// grid: (outer x tiles, items); a tile is w (a power of two) neighbouring columns of the axis a.a0 with
// all n_f planes; columns are the indices of the axes after a0 (row axis included), tiles_main per outer
template <typename Real, int NF>
__global__ void __launch_bounds__(256) gen_col_kernel(LatDev dv, ColArgs a) {
  typedef typename cplx_of<Real>::type C;
  const int item_i = blockIdx.y;
  if (a.scal) {
    const int st = *(volatile const int*)&((const ItemScal*)((const char*)a.scal + (size_t)item_i * 256))->done;
    if (a.only_paused ? st != ITEM_PAUSED : st != ITEM_ACTIVE) return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.G, x = a.a0, w = a.w, lgw = __ffs(w) - 1;
  C* s0 = (C*)smem_raw;
  C* s1 = s0 + (size_t)NF * L * w;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t tiles = a.tiles_main;
  const int64_t o = blockIdx.x / tiles, t = blockIdx.x - o * tiles;
  const int64_t ic = a.inner * a.row_slots;          // columns per outer index
  const int64_t i0 = t * w;
  const int wv = (int)min((int64_t)w, ic - i0);
  const int64_t plane = a.outer * (int64_t)L * ic;
  C* dst = (C*)a.T + item_i * a.t_stride;
  const C* src = a.Tin ? (const C*)a.Tin : dst;
  const int64_t base = o * L * ic + i0;
  for (int idx = tid; idx < NF * L * w; idx += nthr) {
    const int col = idx & (w - 1), g = (idx >> lgw) % L, f = (idx >> lgw) / L;
    if (col < wv) cp_async_elem(s0 + idx, src + (f * plane + base + (int64_t)g * ic + col));
    else s0[idx] = cmake<C>(0.0, 0.0);
  }
  cp_async_wait_all();
  __syncthreads();
  const C* tw = (const C*)dv.tw + dv.ax_twoff[x];
  // four-step twiddle W_e^{n1 k2}: the split's n1 axis is the one before the row, so k2 = column index
  if (a.has_twiddle && a.mode != COL_INV) {
    for (int idx = tid; idx < L * w; idx += nthr) {
      const int col = idx & (w - 1), g = idx >> lgw;
      const C W = gen_split_tw<C>(dv, (int64_t)g * ((i0 + col) % dv.Rlen));
#pragma unroll
      for (int f = 0; f < NF; ++f) s0[(size_t)f * L * w + idx] = cmul(s0[(size_t)f * L * w + idx], W);
    }
    __syncthreads();
  }
  C* cur = s0;
  if (a.mode != COL_INV) cur = fft_mixed<C, false>(s0, s1, L, dv.ax_rad[x], dv.ax_nrad[x], lgw, NF, tw);
  if constexpr (NF >= 3) {
    if (a.mode == COL_GAMMA) {
      const ItemDev* item = a.items + item_i;
      const GreenK<Real> gk = green_consts<Real>(item, a.mat);
      for (int idx = tid; idx < L * w; idx += nthr) {
        const int col = idx & (w - 1), g = idx >> lgw;
        int kk[LAT_MAX_AX] = {0};
        kk[x] = g;
        int64_t i = i0 + col;
        for (int y = dv.nax - 1; y > x; --y) {
          kk[y] = (int)(i % dv.ax_len[y]);
          i /= dv.ax_len[y];
        }
        C val[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) val[f] = cur[(size_t)f * L * w + idx];
        green_at<Real, NF>(dv, a.mat, item, gk, kk, val);
#pragma unroll
        for (int f = 0; f < NF; ++f) cur[(size_t)f * L * w + idx] = val[f];
      }
      __syncthreads();
    }
  }
  if (a.mode != COL_FWD) {
    C* other = (cur == s0) ? s1 : s0;
    cur = fft_mixed<C, true>(cur, other, L, dv.ax_rad[x], dv.ax_nrad[x], lgw, NF, tw);
    if (a.has_twiddle) {
      for (int idx = tid; idx < L * w; idx += nthr) {
        const int col = idx & (w - 1), g = idx >> lgw;
        const C W = gen_split_tw<C>(dv, (int64_t)g * ((i0 + col) % dv.Rlen));
#pragma unroll
        for (int f = 0; f < NF; ++f) cur[(size_t)f * L * w + idx] = cmulc(cur[(size_t)f * L * w + idx], W);
      }
      __syncthreads();
    }
  }
  const bool do_scale = a.do_scale != 0;
  const Real sc = do_scale ? (Real)a.scale : Real(1);
  for (int idx = tid; idx < NF * L * w; idx += nthr) {
    const int col = idx & (w - 1);
    if (col >= wv) continue;
    const int g = (idx >> lgw) % L, f = (idx >> lgw) / L;
    C v = cur[idx];
    if (do_scale) v = cscale(v, sc);
    dst[f * plane + base + (int64_t)g * ic + col] = v;
  }
}

// ------------------------------------------------------------------ complex row transform (lattice_fft)
__global__ void __launch_bounds__(256) gen_row_complex_kernel(LatDev dv, const double2* in, double2* out,
                                                              int inverse, double scale, int rpc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = dv.Rlen, ra = dv.nax - 1;
  double2* b0 = (double2*)smem_raw;
  double2* b1 = b0 + (size_t)rpc * R;
  const int64_t off = (int64_t)blockIdx.x * rpc * R;
  for (int idx = threadIdx.x; idx < rpc * R; idx += blockDim.x) b0[idx] = in[off + idx];
  __syncthreads();
  const double2* tw = (const double2*)dv.tw + dv.ax_twoff[ra];
  double2* r = inverse ? fft_mixed<double2, true>(b0, b1, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, rpc, tw)
                       : fft_mixed<double2, false>(b0, b1, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, rpc, tw);
  for (int idx = threadIdx.x; idx < rpc * R; idx += blockDim.x) {
    double2 v = r[idx];
    if (scale != 1.0) v = cscale(v, scale);
    out[off + idx] = v;
  }
}

// ------------------------------------------------------------------ conjugate gradients
// The stages of cg_row_kernel (kernels.cu: Chronopoulos-Gear conjugate gradients on the discrete
// Lippmann-Schwinger equation, its transform v -> -Gamma0 : (C : v) with k = 0 -> 0, tables holding C) on a
// general plan's rows: mixed-radix row transforms, one point per thread step.  The vectors x (the strain),
// r, p, q = A p and w = A r are held like the strain (binary64, or pairs in the pair kernels).
template <typename Real, int NC>
__global__ void __launch_bounds__(256) gen_cg_row_kernel(LatDev dv, RowArgs a, CgArgs cg) {
  typedef typename cplx_of<Real>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n_c = NC;
  const int R = dv.Rlen, rpc = a.rpc, nlines = n_c * rpc;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const int stage = cg.stage;
  if (stage != CG_FWD_X && *(volatile const int*)&isc->done != ITEM_ACTIVE) return;
  C* buf0 = (C*)smem_raw;
  C* buf1 = buf0 + (size_t)nlines * R;
  double* red = (double*)(buf1 + (size_t)nlines * R);
  __shared__ int s_last;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t m = dv.m, r0 = (int64_t)blockIdx.x * rpc;
  C* T = (C*)a.T + item_i * a.t_stride;
  const int ra = dv.nax - 1;
  const C* tw = (const C*)dv.tw + dv.ax_twoff[ra];
  const size_t voff = (size_t)item_i * cg.vstride;
  double* x = item->eps;
  double* r = cg.r + voff;
  double* p = cg.p + voff;
  double* q = cg.q + voff;
  double* w = cg.w + voff;
  const bool from_spectrum = (stage == CG_FULL0 || stage == CG_A);
  C* cur = buf0;
  if (from_spectrum) {
    for (int idx = tid; idx < nlines * R; idx += nthr) {
      const int line = idx / R, n = idx - line * R;
      const int c = line / rpc, row = line - c * rpc;
      cp_async_elem(buf0 + idx, T + (c * m + (r0 + row) * R + n));
    }
    cp_async_wait_all();
    __syncthreads();
    cur = fft_mixed<C, true>(buf0, buf1, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, nlines, tw);
  }
  C* other = (cur == buf0) ? buf1 : buf0;
  Real alpha = Real(0), beta = Real(0), lam0, two_mu0;
  if constexpr (is_df<Real>) {
    if (stage == CG_B) {
      alpha = isc->cg_alpha_df;
      beta = isc->cg_beta_df;
    }
    lam0 = item->lam0_df;
    two_mu0 = item->mu0_df + item->mu0_df;
  } else {
    if (stage == CG_B) {
      alpha = Real(isc->cg_alpha);
      beta = Real(isc->cg_beta);
    }
    lam0 = Real(item->lam0);
    two_mu0 = Real(2.0 * item->mu0);
  }
  const Real* Ct = tab_of<Real>(item->Dtab, item->Dtab_f, item->Dtab_df);
  Real acc0 = Real(0), acc1 = Real(0);   // <r, r>_C0 (or <w, r>_C0) and ||r||^2
  for (int idx = tid; idx < rpc * R; idx += nthr) {
    const int row = idx / R, n = idx - row * R;
    const int64_t g = (r0 + row) * R + n;
    Real v[NC];
    if (from_spectrum) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) v[c] = cur[((size_t)c * rpc + row) * R + n].x;
    }
    if (stage == CG_FWD_X) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) v[c] = eps_ld1<Real>(x + c * m + g);
    } else if (stage == CG_FULL0) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) eps_st1<Real>(r + c * m + g, v[c]);
      acc0 += c0_dot<Real, NC>(v, v, lam0, two_mu0);
      acc1 += frob2<Real, NC>(v);
    } else if (stage == CG_A) {
      Real s[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        v[c] = -v[c];
        eps_st1<Real>(w + c * m + g, v[c]);
        s[c] = eps_ld1<Real>(r + c * m + g);
      }
      acc0 += c0_dot<Real, NC>(v, s, lam0, two_mu0);
      continue;   // no polarization: the next stage starts from the updated vectors
    } else {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const int64_t o = c * m + g;
        Real rv = eps_ld1<Real>(r + o), pv = eps_ld1<Real>(p + o), qv = eps_ld1<Real>(q + o);
        const Real wv = eps_ld1<Real>(w + o);
        Real xv = eps_ld1<Real>(x + o);
        pv = rv + beta * pv;
        qv = wv + beta * qv;
        xv = xv + alpha * pv;
        rv = rv - alpha * qv;
        eps_st1<Real>(p + o, pv);
        eps_st1<Real>(q + o, qv);
        eps_st1<Real>(x + o, xv);
        eps_st1<Real>(r + o, rv);
        v[c] = rv;
      }
      acc0 += c0_dot<Real, NC>(v, v, lam0, two_mu0);
      acc1 += frob2<Real, NC>(v);
    }
    // tau = C : v for the next transform
    const Real* Cp = Ct + (int)item->phase[g] * n_c * n_c;
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      Real t = Real(0);
#pragma unroll
      for (int k = 0; k < n_c; ++k) t += ldg_r(Cp + c * n_c + k) * v[k];
      cur[((size_t)c * rpc + row) * R + n] = cpair<C>(t, Real(0));
    }
  }
  __syncthreads();
  if (stage != CG_A) {
    C* out = fft_mixed<C, false>(cur, other, R, dv.ax_rad[ra], dv.ax_nrad[ra], 0, nlines, tw);
    if (a.flags & ROW_GAMMA) {   // the row is the only logical axis
      const GreenK<Real> gk = green_consts<Real>(item, a.mat);
      for (int idx = tid; idx < rpc * R; idx += nthr) {
        const int row = idx / R, k = idx - row * R;
        C val[NC];
#pragma unroll
        for (int c = 0; c < n_c; ++c) val[c] = out[((size_t)c * rpc + row) * R + k];
        int kk[LAT_MAX_AX] = {0};
        kk[ra] = k;
        green_at<Real, NC>(dv, a.mat, item, gk, kk, val);
#pragma unroll
        for (int c = 0; c < n_c; ++c) out[((size_t)c * rpc + row) * R + k] = val[c];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < nlines * R; idx += nthr) {
      const int line = idx / R, n = idx - line * R;
      const int c = line / rpc, row = line - c * rpc;
      T[c * m + (r0 + row) * R + n] = out[idx];
    }
  }
  if (stage == CG_FWD_X) return;
  double* partials = a.it.partials + item_i * a.it.pstride;
  const Real vv[2] = {acc0, acc1};
  double tot[2];
  if (stage == CG_A) {
    if (!item_reduce<1>(vv, partials, isc, red, &s_last, tot)) return;
    if (tid == 0) {
      const double gam = isc->cg_gamma, delta = tot[0];
      const bool first = (isc->iter == 1) || isc->cg_alpha_prev == 0.0 || isc->cg_gamma_prev == 0.0;
      const double bet = first ? 0.0 : gam / isc->cg_gamma_prev;
      const double den = first ? delta : delta - bet * gam / isc->cg_alpha_prev;
      const double alp = (gam != 0.0 && den != 0.0) ? gam / den : 0.0;
      isc->cg_alpha = alp;
      isc->cg_beta = bet;
      isc->cg_alpha_df = dfloat(alp);
      isc->cg_beta_df = dfloat(bet);
      isc->cg_gamma_prev = gam;
      isc->cg_alpha_prev = alp;
      isc->counter = 0u;
    }
  } else {
    if (!item_reduce<2>(vv, partials, isc, red, &s_last, tot)) return;
    if (tid == 0) {
      const double rr = sqrt(tot[1]) / item->norm0;
      const double floor_rel = is_df<Real> ? 0x1p-38 : 0x1p-43;   // 1024 u
      if (stage == CG_FULL0) isc->cg_r0 = rr;
      isc->cg_gamma = tot[0];
      item_report(rr, isc, item_i, a.it, rr <= floor_rel * isc->cg_r0);
    }
  }
}

template <typename Real>
void launch_gen_cg_row(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items, int nthreads,
                       size_t smem, cudaStream_t st) {
  if constexpr (is_f32<Real>) {
    return;   // conjugate gradients run in binary64 or on pairs (checked on entry)
  } else {
    const dim3 grid(nblocks, n_items);
    if (dv.n_c == 6) gen_cg_row_kernel<Real, 6><<<grid, nthreads, smem, st>>>(dv, a, cg);
    else gen_cg_row_kernel<Real, 3><<<grid, nthreads, smem, st>>>(dv, a, cg);
  }
}
template void launch_gen_cg_row<double>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t,
                                        cudaStream_t);
template void launch_gen_cg_row<float>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t,
                                       cudaStream_t);
template void launch_gen_cg_row<dfloat>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t,
                                        cudaStream_t);

// ------------------------------------------------------------------ chirp-z rows (Bluestein)
// A largest divisor p with no split into two lines that fit in shared memory is transformed as
// X_k = w_k sum_n (x_n w_n) conj(w_{k-n}), w_n = exp(-i pi n^2 / p): the sum is a cyclic convolution of
// power-of-two length L >= 2p - 1, taken by the transforms of the plan diag(1, L) between pre and post.
// Y is in the storage order of the power-of-two sub-plan: slot s = n1 B + n2 holds sample n = n1 + A n2
__global__ void __launch_bounds__(256) blue_pre_kernel(const double2* __restrict__ src, int64_t src_stride,
                                                       int lines_per_item, int64_t p, int64_t L, int lgA, int lgB,
                                                       const double2* __restrict__ chirp, double2* __restrict__ Y,
                                                       int inverse, int64_t l0) {
  const int64_t l = l0 + blockIdx.y;
  const int64_t i = l / lines_per_item, j = l - i * lines_per_item;
  const double2* x = src + i * src_stride + j * p;
  double2* y = Y + (int64_t)blockIdx.y * L;
  const int64_t Bm = (int64_t(1) << lgB) - 1;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < L; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = (s >> lgB) + ((s & Bm) << lgA);
    double2 v = make_double2(0.0, 0.0);
    if (n < p) {
      v = x[n];
      if (inverse) v.y = -v.y;   // inverse DFT = conj(DFT(conj x))
      v = cmul(v, __ldg(chirp + n));
    }
    y[s] = v;
  }
}

__global__ void __launch_bounds__(256) blue_mul_kernel(double2* __restrict__ Y, const double2* __restrict__ bh,
                                                       int64_t L, double scale) {
  double2* y = Y + (int64_t)blockIdx.y * L;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = cscale(cmul(y[k], __ldg(bh + k)), scale);
}

__global__ void __launch_bounds__(256) blue_post_kernel(const double2* __restrict__ Y, double2* __restrict__ dst,
                                                        int64_t dst_stride, int lines_per_item, int64_t p, int64_t L,
                                                        int lgA, int lgB, const double2* __restrict__ chirp,
                                                        int inverse, double scale, int64_t l0) {
  const int64_t l = l0 + blockIdx.y;
  const int64_t i = l / lines_per_item, j = l - i * lines_per_item;
  double2* out = dst + i * dst_stride + j * p;
  const double2* y = Y + (int64_t)blockIdx.y * L;
  const int64_t Am = (int64_t(1) << lgA) - 1;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = cmul(y[((k & Am) << lgB) + (k >> lgA)], __ldg(chirp + k));
    if (inverse) v.y = -v.y;
    out[k] = cscale(v, scale);
  }
}

// the pointwise step of Algorithm 1 on a chirp-z plan (the row pass of gen_row_kernel without its row
// transforms, which run as the launches above): eps^(n+1) = Re of the inverse transform held in T, the
// Cauchy residual against eps^(n), tau = (C_y - C0) : eps^(n+1) back into T as a real signal
template <int NC>
__global__ void __launch_bounds__(256) blue_point_kernel(LatDev dv, RowArgs a) {
  constexpr int n_c = NC, D = (NC == 6) ? 3 : 2;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const bool update = (a.flags & ROW_UPDATE) != 0;
  if (update && *(volatile const int*)&isc->done != ITEM_ACTIVE) return;   // finished earlier
  __shared__ double red[32];
  __shared__ int s_last;
  const int64_t m = dv.m;
  double2* T = (double2*)a.T + item_i * a.t_stride;
  double* eps = item->eps;
  const uint8_t* phase = item->phase;
  const bool load = (a.flags & ROW_LOAD_EPS) != 0, field = (a.flags & ROW_FIELD) != 0;
  double dsum = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m; g += (int64_t)gridDim.x * blockDim.x) {
    double e[NC];
#pragma unroll
    for (int c = 0; c < n_c; ++c) e[c] = load ? eps[c * m + g] : T[c * m + g].x;
    const int ph = field ? 0 : phase[g];
    if (!field && update && a.mat.scheme == LAT_SCHEME_EYRE_MILTON) {
      // the transform returned u = (C + C0) eps: eps = (C_p + C0)^{-1} u
      const double* W = item->Wtab + ph * n_c * n_c;
      double u[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) u[c] = e[c];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < n_c; ++q) t += ldg_r(W + c * n_c + q) * u[q];
        e[c] = t;
      }
    }
    if (update) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        double* pe = eps + (c * m + g);
        const double d = e[c] - *pe;
        dsum += (c >= D ? 2.0 : 1.0) * (d * d);
        *pe = e[c];
      }
    }
    double t[NC];
    if (field) {   // per-point stiffness field: tau = C_y : eps - C0 : eps
      const GreenK<double> gk = green_consts<double>(item, a.mat);
      field_polarize<double, NC>(item->fld, m, g, gk.lam0, gk.mu0 + gk.mu0, e, t);
    } else {
      const double* Dt = item->Dtab + ph * n_c * n_c;
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < n_c; ++q) s += ldg_r(Dt + c * n_c + q) * e[q];
        t[c] = s;
      }
    }
#pragma unroll
    for (int c = 0; c < n_c; ++c) T[c * m + g] = make_double2(t[c], 0.0);
  }
  if (!update) return;
  double* partials = a.it.partials + item_i * a.it.pstride;
  double tot;
  if (!item_reduce<1>(&dsum, partials, isc, red, &s_last, &tot)) return;
  if (threadIdx.x == 0) item_report(sqrt(tot) / item->norm0, isc, item_i, a.it);
}

// the Green operator on the spectrum of a chirp-z plan whose row is its only logical axis (d_M = 1)
template <int NC>
__global__ void __launch_bounds__(256) blue_green_kernel(LatDev dv, RowArgs a) {
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  if (a.flags & ROW_UPDATE) {   // items that stopped in this iteration or earlier keep their spectrum
    const ItemScal* isc = (const ItemScal*)((const char*)a.it.scal + (size_t)item_i * 256);
    if (*(volatile const int*)&isc->done != ITEM_ACTIVE) return;
  }
  const GreenK<double> gk = green_consts<double>(item, a.mat);
  const int64_t m = dv.m;
  double2* T = (double2*)a.T + item_i * a.t_stride;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    double2 val[NC];
#pragma unroll
    for (int f = 0; f < NC; ++f) val[f] = T[f * m + k];
    int kk[LAT_MAX_AX] = {0};
    kk[0] = (int)k;
    green_at<double, NC>(dv, a.mat, item, gk, kk, val);
#pragma unroll
    for (int f = 0; f < NC; ++f) T[f * m + k] = val[f];
  }
}

static unsigned blue_grid_x(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 1024)); }

void launch_blue_pre(const double2* src, int64_t src_stride, int lines_per_item, int64_t p, int64_t L, int lgA,
                     int lgB, const double2* chirp, double2* Y, int inverse, int64_t l0, int nl, cudaStream_t st) {
  blue_pre_kernel<<<dim3(blue_grid_x(L), nl), 256, 0, st>>>(src, src_stride, lines_per_item, p, L, lgA, lgB, chirp, Y,
                                                            inverse, l0);
}
void launch_blue_mul(double2* Y, const double2* bh, int64_t L, int nl, double scale, cudaStream_t st) {
  blue_mul_kernel<<<dim3(blue_grid_x(L), nl), 256, 0, st>>>(Y, bh, L, scale);
}
void launch_blue_post(const double2* Y, double2* dst, int64_t dst_stride, int lines_per_item, int64_t p, int64_t L,
                      int lgA, int lgB, const double2* chirp, int inverse, double scale, int64_t l0, int nl,
                      cudaStream_t st) {
  blue_post_kernel<<<dim3(blue_grid_x(p), nl), 256, 0, st>>>(Y, dst, dst_stride, lines_per_item, p, L, lgA, lgB, chirp,
                                                             inverse, scale, l0);
}
void launch_blue_point(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, cudaStream_t st) {
  const dim3 grid(nblocks, n_items);
  if (dv.n_c == 6) blue_point_kernel<6><<<grid, 256, 0, st>>>(dv, a);
  else blue_point_kernel<3><<<grid, 256, 0, st>>>(dv, a);
}
void launch_blue_green(const LatDev& dv, const RowArgs& a, int n_items, cudaStream_t st) {
  const dim3 grid(blue_grid_x(dv.m), n_items);
  if (dv.n_c == 6) blue_green_kernel<6><<<grid, 256, 0, st>>>(dv, a);
  else blue_green_kernel<3><<<grid, 256, 0, st>>>(dv, a);
}

// ------------------------------------------------------------------ launchers
template <typename Real>
void launch_gen_row(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, int nthreads, size_t smem,
                    cudaStream_t st) {
  const dim3 grid(nblocks, n_items);
  if (dv.n_c == 6) gen_row_kernel<Real, 6><<<grid, nthreads, smem, st>>>(dv, a);
  else gen_row_kernel<Real, 3><<<grid, nthreads, smem, st>>>(dv, a);
}
template <typename Real>
void launch_gen_col(const LatDev& dv, const ColArgs& a, int n_items, int nthreads, size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned)(a.outer * a.tiles_main), n_items);
  if (a.n_f == 6) gen_col_kernel<Real, 6><<<grid, nthreads, smem, st>>>(dv, a);
  else if (a.n_f == 3) gen_col_kernel<Real, 3><<<grid, nthreads, smem, st>>>(dv, a);
  else if constexpr (std::is_same<Real, double>::value) gen_col_kernel<Real, 1><<<grid, nthreads, smem, st>>>(dv, a);
}
void launch_gen_row_complex(const LatDev& dv, const void* in, void* out, int inverse, double scale, int rpc,
                            int nthreads, size_t smem, cudaStream_t st) {
  const int64_t nb = dv.nrows / rpc;
  gen_row_complex_kernel<<<(unsigned)nb, nthreads, smem, st>>>(dv, (const double2*)in, (double2*)out, inverse, scale,
                                                              rpc);
}

template void launch_gen_row<double>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_gen_row<float>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_gen_row<dfloat>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_gen_col<double>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);
template void launch_gen_col<float>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);
template void launch_gen_col<dfloat>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);

template <typename K>
static cudaError_t gen_set_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

int lat_gen_kernel_attrs(int optin) {
  cudaError_t e = gen_set_smem(gen_row_kernel<double, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_kernel<double, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_kernel<dfloat, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_kernel<dfloat, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_cg_row_kernel<double, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_cg_row_kernel<double, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_cg_row_kernel<dfloat, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_cg_row_kernel<dfloat, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_kernel<float, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_kernel<float, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<float, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<float, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<double, 1>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<double, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<double, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<dfloat, 3>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_col_kernel<dfloat, 6>, optin);
  if (e == cudaSuccess) e = gen_set_smem(gen_row_complex_kernel, optin);
  return e == cudaSuccess ? 0 : (int)e;
}
