// kernels.cu -- the Basic Scheme iteration on sm_103a: row pass, column pass, update, averages.
//
// One iteration of Algorithm 1 (Sec. 3.2, arXiv 1605.05712) is two or three
// passes over HBM:
//   row pass    : inverse R2C FFT of the previous spectrum along the contiguous
//                 axis -> eps^(n+1) (Re of F^{-1}), Cauchy residual against eps^(n)
//                 in binary64, eps written, polarization tau = (C_y - C0) : eps,
//                 forward R2C FFT along the row;                 (fused)
//   column pass : four-step twiddle, forward FFT over the remaining divisor
//                 axes, eps_hat = -Gamma0(h) : tau_hat / m (h != 0), eps_hat_0 = E,
//                 inverse FFT, inverse twiddle;                 (fused)
//   (mid pass   : FFT over one more axis group when a tile would not fit)
// The residual reduction ends in the last block of the row pass, which also
// decides convergence and sets the CUDA-graph WHILE condition.
#include <math.h>
#include <math_constants.h>

#include <type_traits>

#include "fft_smem.cuh"
#include "kernels.cuh"
#include "kernels_dev.cuh"

// ------------------------------------------------------------------ row pass
// grid: (row blocks, items); one block = rpc rows x n_c components of one item
// index -> (line, slot) for the R2C pre/post-processing without a division.  The pairs (k, Rh - k) are
// walked in slot order: the spectrum is bit-reversed, so k < Rh/2 exactly when its slot bitrev(k) is
// even; first the even slots 2i (i < Rh/2) of every line, then slot 1 (k = Rh/2, its own partner) of each
// line.  Neighbouring threads then touch slots 2 apart, not the bit-reversed slots of neighbouring k
// (which share one shared-memory bank: a 32-way conflict on 1024-point half rows).
__device__ __forceinline__ void kslot_index(int idx, int nlines, int lgRh, int& line, int& slot) {
  const int lgq = lgRh > 0 ? lgRh - 1 : 0;
  const int n_lo = nlines << lgq;
  if (idx < n_lo) {
    line = idx >> lgq;
    slot = (idx & ((1 << lgq) - 1)) << 1;
  } else {
    line = idx - n_lo;
    slot = 1;
  }
}

// One row-pass block: rpc rows x n_c components of one item in shared memory, as complex slots (two
// neighbouring real points per slot, bit-reversed after the forward FFT) plus the Nyquist value of
// each line; T / TN are the item's spectrum planes.
template <typename Real>
struct RowTile {
  typedef typename cplx_of<Real>::type C;
  C* buf;
  C* nyq;
  C* T;
  C* TN;
  const C* tw;
  const double* lf;
  const double* rc;
  int Rh, lgRh, lgR, rpc, lgrpc, nlines, npl_total, tw_log2;
  int64_t r0, nrows;
  uint32_t hm32;
};

template <typename Real>
__device__ __forceinline__ RowTile<Real> make_row_tile(const LatDev& dv, const RowArgs& a, unsigned char* smem,
                                                       int item_i, int n_c) {
  typedef typename cplx_of<Real>::type C;
  RowTile<Real> t;
  t.Rh = dv.Rh;
  t.lgRh = dv.log2Rh;
  t.lgR = t.lgRh + 1;
  t.rpc = a.rpc;
  t.lgrpc = __ffs(a.rpc) - 1;
  t.nlines = n_c * t.rpc;
  // (line, k) pairs of the R2C pre/post-processing, k in [0, Rh/2]
  t.npl_total = (t.nlines << (t.lgRh > 0 ? t.lgRh - 1 : 0)) + (t.Rh >= 2 ? t.nlines : 0);
  t.tw_log2 = dv.tw_log2;
  t.r0 = (int64_t)blockIdx.x * t.rpc;
  t.nrows = dv.nrows;
  t.hm32 = (uint32_t)(dv.m / 2);
  t.buf = (C*)smem;
  t.nyq = t.buf + tile_span((int64_t)t.nlines * t.Rh, sizeof(C));
  t.T = (C*)a.T + item_i * a.t_stride;
  t.TN = (C*)a.TN + item_i * a.tn_stride;
  t.tw = (const C*)dv.tw;
  t.lf = dv.lf;
  t.rc = dv.rc;
  return t;
}

// the block's rows of the half spectrum -> real rows: tile loads, inverse of the R2C post-processing
// (X[0..Rh] -> Z = E + i O), inverse FFT
// fused radix-4 stage pairs (16 complex values per thread): binary32 only.  The double-float pair kernels
// ran 12-23 % slower fused; the binary64 fused multiply-add stages ran ~1 % slower fused at 2^21 (six
// components), with three times the register spills
template <typename Real, int NC>
constexpr bool fuse16() {
  return is_f32<Real>;
}

template <typename Real, int NC>
__device__ __forceinline__ void row_tile_inverse(const RowTile<Real>& t) {
  typedef typename cplx_of<Real>::type C;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Rh = t.Rh, lgRh = t.lgRh, rpc = t.rpc, lgrpc = t.lgrpc, nlines = t.nlines;
  C* buf = t.buf;
  C* nyq = t.nyq;
  for (int idx = tid; idx < nlines * Rh; idx += nthr) {
    const int line = idx >> lgRh, pos = idx & (Rh - 1);
    const int c = line >> lgrpc, row = line & (rpc - 1);
    cp_async_elem(buf + tpos<C>(idx), t.T + ((uint32_t)c * t.hm32 + (uint32_t)(t.r0 + row) * (uint32_t)Rh + (uint32_t)pos));
  }
  for (int idx = tid; idx < nlines; idx += nthr) {
    const int c = idx >> lgrpc, row = idx & (rpc - 1);
    cp_async_elem(nyq + idx, t.TN + (c * t.nrows + t.r0 + row));
  }
  cp_async_wait_all();
  __syncthreads();
  // k = 0 (with the Nyquist value) in a loop of its own, so that its arithmetic never rides predicated
  // along in the pairs' loop (it touches slot 0 and the Nyquist value only)
  for (int line = tid; line < nlines; line += nthr) {
    C& L0 = buf[tpos<C>(line * Rh)];
    const Real X0 = L0.x, XN = nyq[line].x;
    L0.x = X0 + XN;
    L0.y = X0 - XN;
  }
  for (int idx = tid; idx < t.npl_total; idx += nthr) {
    int line, slot;
    kslot_index(idx, nlines, lgRh, line, slot);
    const int k = (int)bitrev((uint32_t)slot, lgRh);
    const int lb = line * Rh;
    if (k != 0) {
      // Z_k = A + i B conj(W^k), A = X_k + conj X_{Rh-k}, B = X_k - conj X_{Rh-k}; the partner reuses
      // both: W_R^{Rh-k} = -conj(W_R^k), so Z_{Rh-k} = conj(A) + i conj(B conj(W^k))
      const int kp = Rh - k;
      const uint32_t pk = (uint32_t)slot, pkp = bitrev(kp, lgRh);
      const int ik = tpos<C>(lb + (int)pk), ikp = tpos<C>(lb + (int)pkp);
      const C Xk = buf[ik], Xkp = buf[ikp];
      if constexpr (std::is_same<C, double2>::value) {
        // conj(W^k) B = s (c B.x + B.y, c B.y - B.x), W^k = W_R^k, s = Im W^k, c = Re W^k / Im W^k: the
        // products fold into fused multiply-adds (10 operations for the pair instead of 12)
        const double2 e = __ldg((const double2*)t.rc + 2 * (k << (t.tw_log2 - t.lgR)));
        const double Ax = Xk.x + Xkp.x, Ay = Xk.y - Xkp.y, Bx = Xk.x - Xkp.x, By = Xk.y + Xkp.y;
        const double P = fma(e.x, Bx, By), Q = fma(e.x, By, -Bx);
        buf[ik] = make_double2(fma(-e.y, Q, Ax), fma(e.y, P, Ay));
        if (kp != k) buf[ikp] = make_double2(fma(e.y, Q, Ax), fma(e.y, P, -Ay));
      } else {
        const C wk = twid(t.tw, t.tw_log2, t.lgR, k);
        const C A = cadd(Xk, cconj(Xkp)), Pw = cmulc(csub(Xk, cconj(Xkp)), wk);
        buf[ik] = cadd(A, cmuli(Pw));
        if (kp != k) buf[ikp] = cadd(cconj(A), cmuli(cconj(Pw)));
      }
    }
  }
  __syncthreads();
  fft_dit_inv<C, fuse16<Real, NC>()>(buf, lgRh, 0, nlines, t.tw, t.tw_log2, t.lf, NC);
}

// real rows (written by every thread before the call) -> forward FFT, R2C post-processing
// X[k] = 1/2 (A - i W_R^k B), A = Z_k + conj Z_{Rh-k}, B = Z_k - conj Z_{Rh-k}, Gamma0 when the row is
// the only logical axis (ROW_GAMMA), stores of the half spectrum and the Nyquist column
template <typename Real, int NC>
__device__ __forceinline__ void row_tile_forward(const RowTile<Real>& t, const LatDev& dv, const RowArgs& a,
                                                 const ItemDev* item) {
  typedef typename cplx_of<Real>::type C;
  constexpr int n_c = NC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Rh = t.Rh, lgRh = t.lgRh, rpc = t.rpc, lgrpc = t.lgrpc, nlines = t.nlines;
  C* buf = t.buf;
  C* nyq = t.nyq;
  __syncthreads();
  fft_dif<C, fuse16<Real, NC>()>(buf, lgRh, 0, nlines, t.tw, t.tw_log2, t.lf, NC);
  for (int line = tid; line < nlines; line += nthr) {   // k = 0 and the Nyquist value, as in the inverse
    const C Z0 = buf[tpos<C>(line * Rh)];
    buf[tpos<C>(line * Rh)] = cpair<C>(Z0.x + Z0.y, Real(0));
    nyq[line] = cpair<C>(Z0.x - Z0.y, Real(0));
  }
  for (int idx = tid; idx < t.npl_total; idx += nthr) {
    int line, slot;
    kslot_index(idx, nlines, lgRh, line, slot);
    const int k = (int)bitrev((uint32_t)slot, lgRh);
    const int lb = line * Rh;
    if (k != 0) {
      // the partner reuses A and W^k B: X_{Rh-k} = 1/2 (conj(A) - i conj(W^k B)), since
      // W_R^{Rh-k} = -conj(W_R^k) and Z_{Rh-k} - conj Z_k = -conj(B)
      const int kp = Rh - k;
      const uint32_t pk = (uint32_t)slot, pkp = bitrev(kp, lgRh);
      const int ik = tpos<C>(lb + (int)pk), ikp = tpos<C>(lb + (int)pkp);
      const C Zk = buf[ik], Zkp = buf[ikp];
      if constexpr (std::is_same<C, double2>::value) {
        // W^k B = s (c B.x - B.y, c B.y + B.x) with the table's c and h = s / 2 (12 operations for the pair
        // instead of 16)
        const double2* e = (const double2*)t.rc + 2 * (k << (t.tw_log2 - t.lgR));
        const double c = __ldg(&e->x), h = __ldg(&e[1].x);
        const double Bx = Zk.x - Zkp.x, By = Zk.y + Zkp.y;
        const double P = fma(c, Bx, -By), Q = fma(c, By, Bx);
        const double Hx = 0.5 * (Zk.x + Zkp.x), Hy = 0.5 * (Zk.y - Zkp.y);
        buf[ik] = make_double2(fma(h, Q, Hx), fma(-h, P, Hy));
        if (kp != k) buf[ikp] = make_double2(fma(-h, Q, Hx), fma(-h, P, -Hy));
      } else {
        const C wk = twid(t.tw, t.tw_log2, t.lgR, k);
        const C A1 = cadd(Zk, cconj(Zkp)), Q = cmul(csub(Zk, cconj(Zkp)), wk);
        buf[ik] = cscale(csub(A1, cmuli(Q)), Real(0.5));
        if (kp != k) buf[ikp] = cscale(csub(cconj(A1), cmuli(cconj(Q))), Real(0.5));
      }
    }
  }
  __syncthreads();
  if (a.flags & ROW_GAMMA) {  // single logical axis: the row spectrum is the whole spectrum
    const GreenK<Real> gk = green_consts<Real>(item, a.mat);
    for (int idx = tid; idx < rpc * (Rh + 1); idx += nthr) {
      // k in [0, Rh) of every row first (shifts), then the Nyquist frequency k = Rh of each row
      const int n_lo = rpc << lgRh;
      const int row = idx < n_lo ? idx >> lgRh : idx - n_lo;
      const int k = idx < n_lo ? (idx & (Rh - 1)) : Rh;
      C val[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const int line = c * rpc + row;
        val[c] = (k == Rh) ? nyq[line] : buf[tpos<C>(line * Rh + (int)bitrev(k, lgRh))];
      }
      int kk[LAT_MAX_AX] = {0};
      kk[dv.nax - 1] = k;
      green_at<Real, NC>(dv, a.mat, item, gk, kk, val);
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const int line = c * rpc + row;
        if (k == Rh) nyq[line] = val[c];
        else buf[tpos<C>(line * Rh + (int)bitrev(k, lgRh))] = val[c];
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nlines * Rh; idx += nthr) {
    const int line = idx >> lgRh, pos = idx & (Rh - 1);
    const int c = line >> lgrpc, row = line & (rpc - 1);
    t.T[(uint32_t)c * t.hm32 + (uint32_t)(t.r0 + row) * (uint32_t)Rh + (uint32_t)pos] = buf[tpos<C>(idx)];
  }
  for (int idx = tid; idx < nlines; idx += nthr) {
    const int c = idx >> lgrpc, row = idx & (rpc - 1);
    t.TN[c * t.nrows + t.r0 + row] = nyq[idx];
  }
}

// resident blocks of 256 threads per SM the register budget is cut for: binary32 4 (64 registers;
// the pass is latency-bound and ran 18 % faster at 128^3 than with 80 registers and 3 blocks); the
// others keep the budgets the compiler picks on its own (binary64 2-D 64, pairs 2-D 80, 3-D 128)
template <typename Real, int NC>
constexpr int row_min_blocks() {
  return is_f32<Real> ? 4 : (NC == 6 ? 2 : (is_df<Real> ? 3 : 4));
}
// MAT, the form of the material: MAT_TABLE phase ids and per-phase n_c x n_c tables; MAT_ORTHO the same
// tables when they couple no normal and shear components and have a diagonal shear block (ROW_ORTHO: 12
// instead of 36 products per point in 3-D); MAT_FIELD a per-point stiffness field (basic_scheme_solve_field,
// Algorithm 1 only).  Separate instantiations, so that the general kernel keeps its own register allocation
#define MAT_TABLE 0
#define MAT_ORTHO 1
#define MAT_FIELD 2
template <typename Real, int NC, int MAT>
__global__ void __launch_bounds__(256, (row_min_blocks<Real, NC>())) row_pass_kernel(LatDev dv, RowArgs a) {
  typedef typename cplx_of<Real>::type C;
  constexpr bool FIELD = (MAT == MAT_FIELD);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n_c = NC, D = (NC == 6) ? 3 : 2;
  const int Rh = dv.Rh, lgRh = dv.log2Rh, rpc = a.rpc, lgrpc = __ffs(a.rpc) - 1;
  const int nlines = n_c * rpc;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const bool update = (a.flags & ROW_UPDATE) != 0;
  if (a.flags & ROW_ONLY_PAUSED) {
    if (*(volatile const int*)&isc->done != ITEM_PAUSED) return;
  } else if (update && *(volatile const int*)&isc->done != ITEM_ACTIVE) {
    return;  // this item finished (or paused) earlier
  }
  const RowTile<Real> tile = make_row_tile<Real>(dv, a, smem_raw, item_i, n_c);
  C* buf = tile.buf;
  double* red = (double*)(tile.nyq + nlines);
  __shared__ int s_last;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t m = dv.m, R = dv.Rlen;
  const int64_t r0 = tile.r0;
  const uint32_t m32 = (uint32_t)m;
  double* eps = item->eps;
  const uint8_t* phase = item->phase;
  const double* Dtab = item->Dtab;
  const float* Dtab_f = item->Dtab_f;

  if (update && !(a.flags & ROW_LOAD_EPS) && R >= 16) {
    // the block's strain rows (and phase ids) are read only after the inverse transform: send them towards
    // L2 now, so that the pointwise step finds them there instead of waiting on HBM
    const int lg_lpr = lgRh - 3;   // 128-byte lines per row of one component: R * 8 / 128
    const int n_pf = nlines << lg_lpr;
    for (int i = tid; i < n_pf; i += nthr) {
      const int line = i >> lg_lpr, k = i & ((1 << lg_lpr) - 1);
      const int c = line >> lgrpc, row = line & (rpc - 1);
      prefetch_l2(eps + ((uint32_t)c * m32 + (uint32_t)(r0 + row) * (uint32_t)R + 16u * (uint32_t)k));
    }
    if (!FIELD && R >= 128)
      for (int i = tid; i < (rpc << (lgRh - 6)); i += nthr)
        prefetch_l2(phase + ((uint32_t)(r0 + (i >> (lgRh - 6))) * (uint32_t)R + 128u * (uint32_t)(i & ((1 << (lgRh - 6)) - 1))));
  }

  if (a.flags & ROW_LOAD_EPS) {
    const bool eps_df = is_f32<Real> || is_df<Real>;   // binary64 kernels: binary64 strain
    for (int idx = tid; idx < nlines * Rh; idx += nthr) {
      const int line = idx >> lgRh, n = idx & (Rh - 1);
      const int c = line >> lgrpc, row = line & (rpc - 1);
      const double* pe = eps + ((uint32_t)c * m32 + (uint32_t)(r0 + row) * (uint32_t)R + 2u * n);
      if (eps_df) {
        const float4 v = *(const float4*)pe;
        if constexpr (is_df<Real>) buf[tpos<C>(idx)] = cpair<C>(dfloat(v.x, v.y), dfloat(v.z, v.w));
        else if constexpr (is_f32<Real>) buf[tpos<C>(idx)] = cpair<C>(v.x + v.y, v.z + v.w);
        else buf[tpos<C>(idx)] = cmake<C>((double)v.x + (double)v.y, (double)v.z + (double)v.w);
      } else {
        const double2 v = *(const double2*)pe;
        buf[tpos<C>(idx)] = cmake<C>(v.x, v.y);
      }
    }
    __syncthreads();
  } else {
    row_tile_inverse<Real, NC>(tile);
  }

  // pointwise: update, residual, polarization
  double dsum = 0.0, dsum_sh = 0.0;   // binary64 residual: normal and shear components (the latter counted twice)
  // increment form: T carries delta^(n-1) once the first update is done (iteration counter > 0), or
  // from the start after a cold-start prologue; the polarization is always taken of the increment
  // (binary64 kernels never carry the increment: ROW_INCREMENT comes with the binary32 kernels only,
  // ROW_TAU_DELTA and ROW_EPS_DF with the double-float restart; constant false there, so that no binary64
  // instruction of those paths is issued predicated off)
  constexpr bool DBL = std::is_same<Real, double>::value;
  const bool tau_of_delta = !DBL && update && (a.flags & (ROW_INCREMENT | ROW_TAU_DELTA)) != 0;
  const bool incr = !DBL && update && (a.flags & ROW_INCREMENT) != 0 &&
                    ((a.flags & ROW_INCR_FIRST) != 0 || *(volatile const int*)&isc->iter > 0);
  DF dfs = {0.f, 0.f}, dfs_shear = {0.f, 0.f};  // m <= 2^28: in-item offsets stay below 2^31
  dfloat dd_acc(0.f, 0.f), dd_shear(0.f, 0.f);    // residual of the double-float kernels
  for (int idx = tid; idx < rpc * Rh; idx += nthr) {
    const int row = idx >> lgRh, n = idx & (Rh - 1);
    const uint32_t g = (uint32_t)(r0 + row) * (uint32_t)R + 2u * n;
    Real e0[NC], e1[NC];
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      const C z = buf[tpos<C>((c * rpc + row) * Rh + n)];
      e0[c] = z.x;
      e1[c] = z.y;
    }
    uchar2 ph = make_uchar2(0, 0);
    if constexpr (!FIELD) ph = *(const uchar2*)(phase + g);  // g even
    if (!FIELD && update && a.mat.scheme == LAT_SCHEME_EYRE_MILTON) {
      // the transform returned u = (C + C0) eps (or its increment): eps = (C_p + C0)^{-1} u per point
      const Real* Wt;
      if constexpr (is_f32<Real>) Wt = (const Real*)item->Wtab_f;
      else if constexpr (is_df<Real>) Wt = (const Real*)item->Wtab_df;
      else Wt = (const Real*)item->Wtab;
      const Real* W0 = Wt + (int)ph.x * n_c * n_c;
      const Real* W1 = Wt + (int)ph.y * n_c * n_c;
      // u is still in shared memory: read it from there (no register copies on the common path)
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        Real t0 = Real(0), t1 = Real(0);
#pragma unroll
        for (int q = 0; q < n_c; ++q) {
          const C z = buf[tpos<C>((q * rpc + row) * Rh + n)];
          t0 += ldg_r(W0 + c * n_c + q) * z.x;
          t1 += ldg_r(W1 + c * n_c + q) * z.y;
        }
        e0[c] = t0;
        e1[c] = t1;
      }
    }
    if (update) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        double* pe = eps + (uint32_t)(c * m32) + (uint32_t)g;
        if constexpr (is_df<Real>) {
          // double-float pairs: the strain buffer holds pairs during the solve, binary32 pipes only
          const float4 o = *(const float4*)pe;
          const dfloat o0(o.x, o.y), o1(o.z, o.w);
          dfloat n0 = e0[c], n1 = e1[c], d0, d1;
          if (incr) {
            d0 = n0;
            d1 = n1;
            n0 = n0 + o0;
            n1 = n1 + o1;
          } else {
            d0 = n0 - o0;
            d1 = n1 - o1;
          }
          if (c >= D) {
            df_acc_sq(dd_shear, d0);
            df_acc_sq(dd_shear, d1);
          } else {
            df_acc_sq(dd_acc, d0);
            df_acc_sq(dd_acc, d1);
          }
          *(float4*)pe = make_float4(n0.hi, n0.lo, n1.hi, n1.lo);
          if (tau_of_delta) {
            e0[c] = d0;
            e1[c] = d1;
          }
        } else if constexpr (is_f32<Real>) {
          // binary32 kernels: the strain is a double-float pair; no binary64 arithmetic
          float4 o = *(float4*)pe;
          float d0, d1;
          if (incr) {  // T carried the increment itself
            d0 = e0[c];
            d1 = e1[c];
            df_acc(o.x, o.y, d0);
            df_acc(o.z, o.w, d1);
          } else {     // T carried the new strain
            d0 = df_diff(e0[c], o.x, o.y);
            d1 = df_diff(e1[c], o.z, o.w);
            o = make_float4(e0[c], 0.f, e1[c], 0.f);
          }
          *(float4*)pe = o;
          if (c >= D) {
            df_add_sq(dfs_shear, d0);
            df_add_sq(dfs_shear, d1);
          } else {
            df_add_sq(dfs, d0);
            df_add_sq(dfs, d1);
          }
          if (tau_of_delta) {
            e0[c] = d0;
            e1[c] = d1;
          }
        } else {
          // binary64: T carried the new strain; the Cauchy increment is the difference to the stored one
          const double2 old = *(const double2*)pe;
          const double n0 = (double)e0[c], n1 = (double)e1[c];
          const double d0 = n0 - old.x, d1 = n1 - old.y;
          double& acc = (c >= D) ? dsum_sh : dsum;   // c is unrolled: a register, no select
          acc = fma(d0, d0, acc);
          acc = fma(d1, d1, acc);
          *(double2*)pe = make_double2(n0, n1);
        }
      }
    }
    if constexpr (FIELD) {
      const Real* F;
      if constexpr (is_f32<Real>) F = (const Real*)item->fld_f;
      else if constexpr (is_df<Real>) F = (const Real*)item->fld_df;
      else F = (const Real*)item->fld;
      const GreenK<Real> gk = green_consts<Real>(item, a.mat);
      const Real two_mu0 = gk.mu0 + gk.mu0;
      Real t0[NC], t1[NC];
      field_polarize<Real, NC>(F, m, g, gk.lam0, two_mu0, e0, t0);
      field_polarize<Real, NC>(F, m, g + 1, gk.lam0, two_mu0, e1, t1);
#pragma unroll
      for (int c = 0; c < n_c; ++c) buf[tpos<C>((c * rpc + row) * Rh + n)] = cpair<C>(t0[c], t1[c]);
    } else {
      const Real* Dt;
      if constexpr (is_f32<Real>) Dt = (const Real*)Dtab_f;
      else if constexpr (is_df<Real>) Dt = (const Real*)item->Dtab_df;
      else Dt = (const Real*)Dtab;
      const Real* D0 = Dt + (int)ph.x * n_c * n_c;
      const Real* D1 = Dt + (int)ph.y * n_c * n_c;
      if constexpr (MAT == MAT_ORTHO) {   // normal block D x D, shear diagonal
#pragma unroll
        for (int c = 0; c < D; ++c) {
          Real a0, b0, a1, b1;
          ldg_r2(D0 + c * n_c, a0, b0);   // NC == 6: rows 16-byte aligned
          ldg_r2(D1 + c * n_c, a1, b1);
          Real t0 = a0 * e0[0], t1 = a1 * e1[0];
          t0 += b0 * e0[1];
          t1 += b1 * e1[1];
          t0 += ldg_r(D0 + c * n_c + 2) * e0[2];
          t1 += ldg_r(D1 + c * n_c + 2) * e1[2];
          buf[tpos<C>((c * rpc + row) * Rh + n)] = cpair<C>(t0, t1);
        }
#pragma unroll
        for (int c = D; c < n_c; ++c)
          buf[tpos<C>((c * rpc + row) * Rh + n)] =
              cpair<C>(ldg_r(D0 + c * (n_c + 1)) * e0[c], ldg_r(D1 + c * (n_c + 1)) * e1[c]);
      } else {
#pragma unroll
        for (int c = 0; c < n_c; ++c) {
          Real t0 = 0, t1 = 0;
          if constexpr (NC == 6) {   // rows of 6 entries: pairs of entries in one load (rows 16-byte aligned)
#pragma unroll
            for (int q = 0; q < n_c; q += 2) {
              Real a0, b0, a1, b1;
              ldg_r2(D0 + c * n_c + q, a0, b0);
              ldg_r2(D1 + c * n_c + q, a1, b1);
              t0 += a0 * e0[q];
              t0 += b0 * e0[q + 1];
              t1 += a1 * e1[q];
              t1 += b1 * e1[q + 1];
            }
          } else {
#pragma unroll
            for (int q = 0; q < n_c; ++q) {
              t0 += ldg_r(D0 + c * n_c + q) * e0[q];
              t1 += ldg_r(D1 + c * n_c + q) * e1[q];
            }
          }
          buf[tpos<C>((c * rpc + row) * Rh + n)] = cpair<C>(t0, t1);
        }
      }
    }
  }
  row_tile_forward<Real, NC>(tile, dv, a, item);
  if (!update) return;
  // residual: block partial -> the item's last block sums in block order and decides its
  // convergence; the last item to arrive in this iteration sets the WHILE condition
  double* partials = a.it.partials + item_i * a.it.pstride;
  double tot;
  if constexpr (is_f32<Real> || is_df<Real>) {
    // the pair kernels keep the partial a pair (shear terms counted twice, exactly) down to the warp sums
    dfloat pr;
    if constexpr (is_f32<Real>) pr = dfloat(dfs.hi, dfs.lo) + dfloat(2.f * dfs_shear.hi, 2.f * dfs_shear.lo);
    else pr = dd_acc + (dd_shear + dd_shear);
    if (!item_reduce<1>(&pr, partials, isc, red, &s_last, &tot)) return;
  } else {
    dsum = fma(2.0, dsum_sh, dsum);
    if (!item_reduce<1>(&dsum, partials, isc, red, &s_last, &tot)) return;
  }
  if (tid == 0) item_report(sqrt(tot) / item->norm0, isc, item_i, a.it);
}

// ------------------------------------------------------------------ conjugate gradients
// Conjugate gradients on the discrete Lippmann-Schwinger equation A e = -Gamma0 C E, A = Gamma0 C, for
// the compatible zero-mean part e of the strain (one of the accelerated schemes Sec. 6 says carry over to
// patterns).  On those fields Gamma0 C0 is the identity, so A is self-adjoint and positive in the inner
// product <a, c>_C0 = sum_y a_y : C0 : c_y; the recurrences are the Chronopoulos-Gear form of CG, whose
// two inner products come from one pass, so an iteration needs one reduction instead of two:
//   p = r + beta p,  q = w + beta q,  x += alpha p,  r -= alpha q,  w = A r,
//   gamma = <r, r>_C0, delta = <w, r>_C0, beta = gamma / gamma_prev,
//   alpha = gamma / (delta - beta gamma / alpha_prev)        (first step: beta = 0, alpha = gamma / delta)
// with q = A p carried by recurrence.  Rounding leaves each update a residual part outside the compatible
// fields of relative size ~u (unit roundoff); A annihilates it, so once ||r|| falls to the rounding
// level of ||r_0|| the step lengths are meaningless and the iteration stops: at ||r|| <= 1024 u ||r_0||
// (u = 2^-53 in binary64, 2^-48 for the pairs), or at once when r_0 = 0 (E is the exact solution).
// The transform maps a field v to -Gamma0 : (C : v) (the Green step
// of Algorithm 1 with k = 0 mapped to 0), so r = -Gamma0 : sigma(x) is Algorithm 1's increment at x and
// the stopping test takes its measure ||r|| / ||eps^(0)||.  The material tables hold C (not C - C0).
// The vectors are held like the strain: binary64, or double-float pairs in the pair kernels.
template <typename Real>
__device__ __forceinline__ void fld_ld2(const double* p, Real& v0, Real& v1) {
  if constexpr (is_df<Real>) {
    const float4 o = *(const float4*)p;
    v0 = dfloat(o.x, o.y);
    v1 = dfloat(o.z, o.w);
  } else {
    const double2 o = *(const double2*)p;
    v0 = (Real)o.x;
    v1 = (Real)o.y;
  }
}
template <typename Real>
__device__ __forceinline__ void fld_st2(double* p, Real v0, Real v1) {
  if constexpr (is_df<Real>) *(float4*)p = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
  else *(double2*)p = make_double2((double)v0, (double)v1);
}
// the update stage keeps five vectors of a point pair live: 3 blocks of 256 threads per SM (85 registers)
// for 2-D, the row pass's budget for 3-D
template <typename Real, int NC>
constexpr int cg_min_blocks() {
  return NC == 6 ? 2 : 3;
}
template <typename Real, int NC>
__global__ void __launch_bounds__(256, (cg_min_blocks<Real, NC>())) cg_row_kernel(LatDev dv, RowArgs a, CgArgs cg) {
  typedef typename cplx_of<Real>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n_c = NC;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const int stage = cg.stage;
  if (stage != CG_FWD_X && *(volatile const int*)&isc->done != ITEM_ACTIVE) return;
  const RowTile<Real> tile = make_row_tile<Real>(dv, a, smem_raw, item_i, n_c);
  const int Rh = tile.Rh, lgRh = tile.lgRh, rpc = tile.rpc;
  C* buf = tile.buf;
  double* red = (double*)(tile.nyq + tile.nlines);
  __shared__ int s_last;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t m32 = (uint32_t)dv.m, R = (uint32_t)dv.Rlen;
  const size_t voff = (size_t)item_i * cg.vstride;
  double* x = item->eps;
  double* r = cg.r + voff;
  double* p = cg.p + voff;
  double* q = cg.q + voff;
  double* w = cg.w + voff;
  const bool from_spectrum = (stage == CG_FULL0 || stage == CG_A);
  if (from_spectrum) row_tile_inverse<Real, NC>(tile);
  Real alpha = Real(0), beta = Real(0), lam0, two_mu0;
  if constexpr (is_df<Real>) {  // host- or last-block-made pairs: no binary64 conversions per thread
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
  const Real* Ct;
  if constexpr (is_df<Real>) Ct = (const Real*)item->Dtab_df;
  else Ct = (const Real*)item->Dtab;
  Real acc0 = Real(0), acc1 = Real(0);  // <r, r>_C0 (or <w, r>_C0) and ||r||^2
  for (int idx = tid; idx < rpc * Rh; idx += nthr) {
    const int row = idx >> lgRh, n = idx & (Rh - 1);
    const uint32_t g = (uint32_t)(tile.r0 + row) * R + 2u * n;
    Real v0[NC], v1[NC];
    if (from_spectrum) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const C z = buf[tpos<C>((c * rpc + row) * Rh + n)];
        v0[c] = z.x;
        v1[c] = z.y;
      }
    }
    if (stage == CG_FWD_X) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) fld_ld2<Real>(x + (uint32_t)(c * m32) + g, v0[c], v1[c]);
    } else if (stage == CG_FULL0) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) fld_st2<Real>(r + (uint32_t)(c * m32) + g, v0[c], v1[c]);
      acc0 += c0_dot<Real, NC>(v0, v0, lam0, two_mu0) + c0_dot<Real, NC>(v1, v1, lam0, two_mu0);
      acc1 += frob2<Real, NC>(v0) + frob2<Real, NC>(v1);
    } else if (stage == CG_A) {
      Real s0[NC], s1[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        v0[c] = -v0[c];
        v1[c] = -v1[c];
        fld_st2<Real>(w + (uint32_t)(c * m32) + g, v0[c], v1[c]);
        fld_ld2<Real>(r + (uint32_t)(c * m32) + g, s0[c], s1[c]);
      }
      acc0 += c0_dot<Real, NC>(v0, s0, lam0, two_mu0) + c0_dot<Real, NC>(v1, s1, lam0, two_mu0);
      continue;  // no polarization: the next stage starts from the updated vectors
    } else {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const uint32_t o = (uint32_t)(c * m32) + g;
        Real r0, r1, p0, p1, q0, q1, w0, w1, x0, x1;
        fld_ld2<Real>(r + o, r0, r1);
        fld_ld2<Real>(p + o, p0, p1);
        fld_ld2<Real>(q + o, q0, q1);
        fld_ld2<Real>(w + o, w0, w1);
        fld_ld2<Real>(x + o, x0, x1);
        p0 = r0 + beta * p0;
        p1 = r1 + beta * p1;
        q0 = w0 + beta * q0;
        q1 = w1 + beta * q1;
        x0 = x0 + alpha * p0;
        x1 = x1 + alpha * p1;
        r0 = r0 - alpha * q0;
        r1 = r1 - alpha * q1;
        fld_st2<Real>(p + o, p0, p1);
        fld_st2<Real>(q + o, q0, q1);
        fld_st2<Real>(x + o, x0, x1);
        fld_st2<Real>(r + o, r0, r1);
        v0[c] = r0;
        v1[c] = r1;
      }
      acc0 += c0_dot<Real, NC>(v0, v0, lam0, two_mu0) + c0_dot<Real, NC>(v1, v1, lam0, two_mu0);
      acc1 += frob2<Real, NC>(v0) + frob2<Real, NC>(v1);
    }
    // tau = C : v for the next transform
    const uchar2 ph = *(const uchar2*)(item->phase + g);  // g even
    const Real* C0p = Ct + (int)ph.x * n_c * n_c;
    const Real* C1p = Ct + (int)ph.y * n_c * n_c;
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      Real t0 = Real(0), t1 = Real(0);
#pragma unroll
      for (int k = 0; k < n_c; ++k) {
        t0 += ldg_r(C0p + c * n_c + k) * v0[k];
        t1 += ldg_r(C1p + c * n_c + k) * v1[k];
      }
      buf[tpos<C>((c * rpc + row) * Rh + n)] = cpair<C>(t0, t1);
    }
  }
  if (stage != CG_A) row_tile_forward<Real, NC>(tile, dv, a, item);
  if (stage == CG_FWD_X) return;
  double* partials = a.it.partials + item_i * a.it.pstride;
  const Real v[2] = {acc0, acc1};
  double tot[2];
  if (stage == CG_A) {
    if (!item_reduce<1>(v, partials, isc, red, &s_last, tot)) return;
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
    if (!item_reduce<2>(v, partials, isc, red, &s_last, tot)) return;
    if (tid == 0) {
      const double rr = sqrt(tot[1]) / item->norm0;
      const double floor_rel = is_df<Real> ? 0x1p-38 : 0x1p-43;  // 1024 u
      if (stage == CG_FULL0) isc->cg_r0 = rr;
      isc->cg_gamma = tot[0];
      item_report(rr, isc, item_i, a.it, rr <= floor_rel * isc->cg_r0);
    }
  }
}

// ------------------------------------------------------------------ column pass
// resident blocks of 256 threads per SM the column pass's register budget is cut for (the compiler's own
// choice spilled the binary32 3-D pass): 85 registers for 2-D, 128 for the 3-D binary64 and pair passes
template <typename Real, int NC>
constexpr int col_min_blocks() {
  return NC == 6 ? (is_f32<Real> ? 3 : 2) : (NC == 3 ? 3 : 4);
}
template <typename Real, int NC>
__global__ void __launch_bounds__(256, (col_min_blocks<Real, NC>())) col_pass_kernel(LatDev dv, ColArgs a) {
  typedef typename cplx_of<Real>::type C;
  const int item_i = blockIdx.y;
  if (a.scal) {
    const int st = *(volatile const int*)&((const ItemScal*)((const char*)a.scal + (size_t)item_i * 256))->done;
    if (a.only_paused ? st != ITEM_PAUSED : st != ITEM_ACTIVE) return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = (C*)smem_raw;
  const int tid = threadIdx.x, nthr = blockDim.x;
  constexpr int n_f = NC, D = (NC == 6) ? 3 : 2;
  const int G = a.G;
  // block -> (outer index, tile) in 32-bit arithmetic: a 64-bit division runs on the binary64 pipe
  uint32_t b = blockIdx.x;
  const uint32_t main_blocks = (uint32_t)(a.outer * a.tiles_main);   // < gridDim.x
  const bool nyqt = b >= main_blocks;
  int64_t o, t, inner_count;
  int w;
  if (!nyqt) {
    const uint32_t tm = (uint32_t)a.tiles_main, oo = b / tm;
    o = oo;
    t = b - oo * tm;
    w = a.w;
    inner_count = a.inner * a.row_slots;
  } else {
    b -= main_blocks;
    const uint32_t tn = (uint32_t)a.tiles_nyq, oo = b / tn;
    o = oo;
    t = b - oo * tn;
    w = a.wN;
    inner_count = a.inner;
  }
  const int64_t i0 = t * w;
  const int wv = (int)min((int64_t)w, inner_count - i0);
  const int lgw = __ffs(w) - 1, lgG = __ffs(G) - 1;
  const int64_t plane = a.outer * (int64_t)G * inner_count;
  C* dst = nyqt ? (C*)a.TN + item_i * a.tn_stride : (C*)a.T + item_i * a.t_stride;
  const C* src = (a.Tin && !nyqt) ? (const C*)a.Tin : dst;
  const C* tw = (const C*)dv.tw;
  const int lg_slots = __ffs(a.row_slots) - 1;

  // in-item offsets: plane * n_f <= 6 * 2^27 < 2^31
  const uint32_t plane32 = (uint32_t)plane, ic32 = (uint32_t)inner_count;
  const uint32_t base32 = (uint32_t)(o * G) * ic32 + (uint32_t)i0;
  for (int idx = tid; idx < n_f * G * w; idx += nthr) {
    const int col = idx & (w - 1);
    const int g = (idx >> lgw) & (G - 1);
    const int f = idx >> (lgw + lgG);
    if (col < wv) cp_async_elem(s + tpos<C>(idx), src + ((uint32_t)f * plane32 + base32 + (uint32_t)g * ic32 + (uint32_t)col));
    else s[tpos<C>(idx)] = cmake<C>(0.0, 0.0);
  }
  cp_async_wait_all();
  __syncthreads();

  // four-step twiddle W_e^{n1 k2} (k2 = row frequency of this column)
  int lg_after_n1 = 0;
  int len_n1 = 1;
  if (a.has_twiddle) {
    for (int x = dv.split_n1 + 1; x < a.a1; ++x) lg_after_n1 += dv.ax_log2[x];
    len_n1 = dv.ax_len[dv.split_n1];
  }
  auto col_krow = [&](int col) -> int64_t {
    const int64_t ii = i0 + col;
    if (nyqt) return (int64_t)dv.Rh;
    return (int64_t)bitrev((uint32_t)(ii & (a.row_slots - 1)), lg_slots);   // row_slots is a power of two
  };
  auto split_tw = [&](int64_t j) -> C {
    const C* st = (const C*)dv.stw;
    const int sh = dv.split_lo_log2;
    const C hi = ldg_c(st + (j >> sh));
    const C lo = ldg_c(st + dv.stw_hi_n + (j & ((int64_t(1) << sh) - 1)));
    return cmul(hi, lo);
  };
  if (a.has_twiddle && a.mode != COL_INV) {
    for (int idx = tid; idx < G * w; idx += nthr) {
      const int col = idx & (w - 1), g = idx >> lgw;
      const int64_t n1 = (g >> lg_after_n1) & (len_n1 - 1);
      const C W = split_tw(n1 * col_krow(col));
#pragma unroll
      for (int f = 0; f < n_f; ++f) s[tpos<C>(f * G * w + idx)] = cmul(s[tpos<C>(f * G * w + idx)], W);
    }
    __syncthreads();
  }
  if (a.mode != COL_INV) {
    int64_t after = 1;
    for (int x = a.a1 - 1; x >= a.a0; --x) {
      int64_t before = 1;
      for (int y = a.a0; y < x; ++y) before *= dv.ax_len[y];
      fft_dif<C, fuse16<Real, NC>()>(s, dv.ax_log2[x], lgw + (__ffsll(after) - 1), (int)(n_f * before), tw,
                                     dv.tw_log2, dv.lf, n_f);
      after *= dv.ax_len[x];
    }
  }
  if (NC >= 3 && a.mode == COL_GAMMA) {
    const ItemDev* item = a.items + item_i;
    const GreenK<Real> gk = green_consts<Real>(item, a.mat);
    // the frequency's coordinates v = sum_x k_x cv[x] split into the column's share (the axes between the
    // group and the row, transformed by the mid passes, and the row; a thread keeps its column, since the
    // block size is a multiple of w) and the group's share, which varies with g
    uint32_t vc32[3] = {0u, 0u, 0u};
    int64_t vc64[3] = {0, 0, 0};
    {
      const int col = tid & (w - 1);
      const int64_t ii = i0 + col;
      int64_t mid = nyqt ? ii : (ii >> lg_slots);
      for (int x = dv.nax - 2; x >= a.a1; --x) {
        const int pos = (int)(mid & (dv.ax_len[x] - 1));
        mid >>= dv.ax_log2[x];
        v_add<D>(dv, x, (int)bitrev(pos, dv.ax_log2[x]), vc32, vc64);
      }
      v_add<D>(dv, dv.nax - 1, (int)col_krow(col), vc32, vc64);
    }
    for (int idx = tid; idx < G * w; idx += nthr) {
      const int g = idx >> lgw;
      uint32_t v32[3] = {vc32[0], vc32[1], vc32[2]};
      int64_t v64[3] = {vc64[0], vc64[1], vc64[2]};
      // group axes (bit-reversed after the DIF)
      int rem = g;
      for (int x = a.a1 - 1; x >= a.a0; --x) {
        const int pos = rem & (dv.ax_len[x] - 1);
        rem >>= dv.ax_log2[x];
        v_add<D>(dv, x, (int)bitrev(pos, dv.ax_log2[x]), v32, v64);
      }
      C val[NC];
#pragma unroll
      for (int f = 0; f < n_f; ++f) val[f] = s[tpos<C>(f * G * w + idx)];
      if constexpr (NC >= 3) green_from_v<Real, NC>(dv, a.mat, item, gk, v32, v64, val);
#pragma unroll
      for (int f = 0; f < n_f; ++f) s[tpos<C>(f * G * w + idx)] = val[f];
    }
    __syncthreads();
  }
  if (a.mode != COL_FWD) {
    int64_t before = 1;
    for (int x = a.a0; x < a.a1; ++x) {
      int64_t after = 1;
      for (int y = x + 1; y < a.a1; ++y) after *= dv.ax_len[y];
      fft_dit_inv<C, fuse16<Real, NC>()>(s, dv.ax_log2[x], lgw + (__ffsll(after) - 1), (int)(n_f * before), tw,
                                         dv.tw_log2, dv.lf, n_f);
      before *= dv.ax_len[x];
    }
    if (a.has_twiddle) {
      for (int idx = tid; idx < G * w; idx += nthr) {
        const int col = idx & (w - 1), g = idx >> lgw;
        const int64_t n1 = (g >> lg_after_n1) & (len_n1 - 1);
        const C W = split_tw(n1 * col_krow(col));
#pragma unroll
        for (int f = 0; f < n_f; ++f) s[tpos<C>(f * G * w + idx)] = cmulc(s[tpos<C>(f * G * w + idx)], W);
      }
      __syncthreads();
    }
  }
  const bool do_scale = a.do_scale != 0;
  Real sc = Real(1);
  if (do_scale) sc = (Real)a.scale;
  for (int idx = tid; idx < n_f * G * w; idx += nthr) {
    const int col = idx & (w - 1);
    if (col >= wv) continue;
    const int g = (idx >> lgw) & (G - 1);
    const int f = idx >> (lgw + lgG);
    C val = s[tpos<C>(idx)];
    if (do_scale) val = cscale(val, sc);
    dst[(uint32_t)f * plane32 + base32 + (uint32_t)g * ic32 + (uint32_t)col] = val;
  }
}

// ------------------------------------------------------------------ complex row transform (lattice_fft)
template <typename Real>
__global__ void __launch_bounds__(256) row_complex_kernel(LatDev dv, const void* in, void* out, int n_f,
                                                          int inverse, double scale, int rpc) {
  typedef typename cplx_of<Real>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = (C*)smem_raw;
  const int R = dv.Rlen, lgR = dv.log2Rh + 1, nlines = n_f * rpc;
  const int64_t m = dv.m, r0 = (int64_t)blockIdx.x * rpc;
  const C* src = (const C*)in + (int64_t)blockIdx.y * n_f * m;   // grid.y: groups of n_f fields
  C* dst = (C*)out + (int64_t)blockIdx.y * n_f * m;
  for (int idx = threadIdx.x; idx < nlines * R; idx += blockDim.x) {
    const int line = idx / R, pos = idx - line * R;
    const int f = line / rpc, row = line - f * rpc;
    buf[tpos<C>(idx)] = src[f * m + (r0 + row) * R + pos];
  }
  __syncthreads();
  if (inverse) fft_dit_inv(buf, lgR, 0, nlines, (const C*)dv.tw, dv.tw_log2, dv.lf);
  else fft_dif(buf, lgR, 0, nlines, (const C*)dv.tw, dv.tw_log2, dv.lf);
  const Real sc = (Real)scale;
  for (int idx = threadIdx.x; idx < nlines * R; idx += blockDim.x) {
    const int line = idx / R, pos = idx - line * R;
    const int f = line / rpc, row = line - f * rpc;
    C v = buf[tpos<C>(idx)];
    if (scale != 1.0) v = cscale(v, sc);
    dst[f * m + (r0 + row) * R + pos] = v;
  }
}

// ------------------------------------------------------------------ fill, effective stress
__global__ void fill_kernel(const ItemDev* items, int n_c, int64_t m) {
  const ItemDev* it = items + blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    for (int c = 0; c < n_c; ++c) it->eps[c * m + i] = it->E[c];
}

// sigma_y = C_y : eps_y and sigma_bar = (1/m) sum_y sigma_y  (Sec. 3.1, effective matrix); grid.y = item
__global__ void __launch_bounds__(256) eff_kernel(LatDev dv, EffArgs a) {
  __shared__ double red[32];
  __shared__ int s_last;
  const int n_c = dv.n_c;
  const ItemDev* it = a.items + blockIdx.y;
  ItemScal* isc = (ItemScal*)((char*)a.scal + (size_t)blockIdx.y * 256);
  double* partials = a.partials + blockIdx.y * a.pstride;
  const int64_t m = dv.m, stride = (int64_t)gridDim.x * blockDim.x;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    double e[6];
    for (int c = 0; c < n_c; ++c) e[c] = it->eps[c * m + i];
    if (it->fld) {   // per-point stiffness field: sigma = C_y : eps (tau + C0 : eps with C0 = 0)
      double sg[6];
      if (n_c == 6) field_polarize<double, 6>(it->fld, m, i, 0.0, 0.0, e, sg);
      else field_polarize<double, 3>(it->fld, m, i, 0.0, 0.0, e, sg);
      for (int c = 0; c < n_c; ++c) {
        if (it->sigma) it->sigma[c * m + i] = sg[c];
        acc[c] += sg[c];
      }
      continue;
    }
    const double* Cp = it->Ctab + (int)it->phase[i] * n_c * n_c;
    for (int c = 0; c < n_c; ++c) {
      double sgm = 0;
      for (int q = 0; q < n_c; ++q) sgm += __ldg(Cp + c * n_c + q) * e[q];
      if (it->sigma) it->sigma[c * m + i] = sgm;
      acc[c] += sgm;
    }
  }
  for (int c = 0; c < n_c; ++c) {
    const double bs = block_sum(acc[c], red);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * n_c + c] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&isc->eff_counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    for (int c = 0; c < n_c; ++c) {
      double t = 0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t += __ldcg(partials + (int64_t)b * n_c + c);
      t = warp_sum(t);
      if (threadIdx.x == 0) isc->sigma_bar[c] = t / (double)m;
    }
    if (threadIdx.x == 0) isc->eff_counter = 0u;
  }
}

// ------------------------------------------------------------------ launchers
template <typename Real>
void launch_row_pass(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, int nthreads, size_t smem,
                     cudaStream_t st) {
  const dim3 grid(nblocks, n_items);
  if (a.flags & ROW_FIELD) {
    if (dv.n_c == 6) row_pass_kernel<Real, 6, MAT_FIELD><<<grid, nthreads, smem, st>>>(dv, a);
    else row_pass_kernel<Real, 3, MAT_FIELD><<<grid, nthreads, smem, st>>>(dv, a);
  } else if (dv.n_c == 6) {
    if (a.flags & ROW_ORTHO) row_pass_kernel<Real, 6, MAT_ORTHO><<<grid, nthreads, smem, st>>>(dv, a);
    else row_pass_kernel<Real, 6, MAT_TABLE><<<grid, nthreads, smem, st>>>(dv, a);
  } else {
    row_pass_kernel<Real, 3, MAT_TABLE><<<grid, nthreads, smem, st>>>(dv, a);
  }
}
template <typename Real>
void launch_cg_row(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items, int nthreads,
                   size_t smem, cudaStream_t st) {
  if constexpr (is_f32<Real>) {
    return;  // the conjugate-gradient scheme runs in binary64 or on double-float pairs (checked on entry)
  } else {
    if (dv.general) return launch_gen_cg_row<Real>(dv, a, cg, nblocks, n_items, nthreads, smem, st);
    const dim3 grid(nblocks, n_items);
    if (dv.n_c == 6) cg_row_kernel<Real, 6><<<grid, nthreads, smem, st>>>(dv, a, cg);
    else cg_row_kernel<Real, 3><<<grid, nthreads, smem, st>>>(dv, a, cg);
  }
}
template <typename Real>
void launch_col_pass(const LatDev& dv, const ColArgs& a, int n_items, int nthreads, size_t smem, cudaStream_t st) {
  const dim3 grid((unsigned)(a.outer * (a.tiles_main + a.tiles_nyq)), n_items);
  if (a.n_f == 6) col_pass_kernel<Real, 6><<<grid, nthreads, smem, st>>>(dv, a);
  else if (a.n_f == 3) col_pass_kernel<Real, 3><<<grid, nthreads, smem, st>>>(dv, a);
  else if constexpr (!is_df<Real>) col_pass_kernel<Real, 1><<<grid, nthreads, smem, st>>>(dv, a);
}
template <typename Real>
void launch_row_complex(const LatDev& dv, const void* in, void* out, int n_f, int inverse, double scale, int rpc,
                        int nthreads, size_t smem, cudaStream_t st, int n_groups) {
  const int64_t nb = dv.nrows / rpc;
  row_complex_kernel<Real><<<dim3((unsigned)nb, (unsigned)n_groups), nthreads, smem, st>>>(dv, in, out, n_f, inverse,
                                                                                          scale, rpc);
}
// in place: binary64 strain <-> double-float pairs (to_df = 1: before a mixed solve's prologue)
__global__ void eps_df_kernel(const ItemDev* items, int n_c, int64_t m, int to_df) {
  double* eps = items[blockIdx.y].eps;
  const int64_t n = (int64_t)n_c * m;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (to_df) {
      const double v = eps[i];
      *(float2*)(eps + i) = df_of(v);
    } else {
      const float2 p = *(const float2*)(eps + i);
      eps[i] = (double)p.x + (double)p.y;
    }
  }
}

__global__ void prep_restart_kernel(ItemScal* scal, GlobScal* glob, int n_items) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = 0;
  for (int i = 0; i < n_items; ++i)
    n += ((const ItemScal*)((const char*)scal + (size_t)i * 256))->done == ITEM_PAUSED;
  glob->active = n;
  glob->arrivals = 0u;
}

__global__ void set_cond_kernel(const GlobScal* glob, unsigned long long cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, glob->active > 0 ? 1u : 0u);
}

// grid (blocks, items); t_elems / tn_elems complex values per item in T / TN
__global__ void spectrum_to_f32_kernel(const double2* T64, const double2* TN64, float2* T32, float2* TN32,
                                       int64_t t_elems, int64_t tn_elems, int64_t t_stride, int64_t tn_stride,
                                       const ItemScal* scal) {
  const int item_i = blockIdx.y;
  if (((const ItemScal*)((const char*)scal + (size_t)item_i * 256))->done != ITEM_ACTIVE) return;
  // the restart spectrum holds double-float pairs (re hi, re lo, im hi, im lo)
  const float4* a = (const float4*)T64 + item_i * t_stride;
  float2* b = T32 + item_i * t_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < t_elems; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = a[i];
    b[i] = make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
  }
  const float4* an = (const float4*)TN64 + item_i * tn_stride;
  float2* bn = TN32 + item_i * tn_stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tn_elems; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = an[i];
    bn[i] = make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
  }
}

void launch_eps_df(const ItemDev* items, int n_items, int n_c, int64_t m, int to_df, cudaStream_t st) {
  int64_t nb = ((int64_t)n_c * m + 255) / 256;
  if (nb > 2432) nb = 2432;
  eps_df_kernel<<<dim3((unsigned)nb, n_items), 256, 0, st>>>(items, n_c, m, to_df);
}
void launch_prep_restart(ItemScal* scal, GlobScal* glob, int n_items, cudaStream_t st) {
  prep_restart_kernel<<<1, 32, 0, st>>>(scal, glob, n_items);
}
void launch_set_cond(const GlobScal* glob, unsigned long long cond, cudaStream_t st) {
  set_cond_kernel<<<1, 32, 0, st>>>(glob, cond);
}
void launch_spectrum_to_f32(const void* T64, const void* TN64, void* T32, void* TN32, int64_t t_elems,
                            int64_t tn_elems, int64_t t_stride, int64_t tn_stride, const ItemScal* scal,
                            int n_items, cudaStream_t st) {
  int64_t nb = (t_elems + 255) / 256;
  if (nb > 1216) nb = 1216;
  spectrum_to_f32_kernel<<<dim3((unsigned)nb, n_items), 256, 0, st>>>(
      (const double2*)T64, (const double2*)TN64, (float2*)T32, (float2*)TN32, t_elems, tn_elems, t_stride, tn_stride,
      scal);
}

// the host decode of a finished solve, on the device: m = 1 (trivial) iterates to E at once (r = 0 after one
// iteration when tol > 0); maxit = 0 reports no residual; non-finite or diverging residuals are LAT_DIVERGED
__global__ void scalars_out_kernel(const ItemScal* scal, int n_items, int n_c, double tol, int maxit, int trivial,
                                   double* sigma_bar, int* iters, double* resid, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const ItemScal* sc = (const ItemScal*)((const char*)scal + (size_t)i * 256);
  int it = sc->iter;
  double r = sc->last_r;
  if (trivial) {
    it = (maxit > 0 && tol > 0) ? 1 : maxit;
    r = maxit > 0 ? 0.0 : CUDART_NAN;
  } else if (maxit == 0) {
    r = CUDART_NAN;
  }
  if (iters) iters[i] = it;
  if (resid) resid[i] = r;
  if (sigma_bar)
    for (int c = 0; c < n_c; ++c) sigma_bar[i * n_c + c] = sc->sigma_bar[c];
  if (status) {
    int s = LAT_OK;
    if ((!isfinite(r) || sc->diverged) && maxit > 0) s = LAT_DIVERGED;
    else if (!(r < tol)) s = LAT_NOT_CONVERGED;
    status[i] = s;
  }
}

void launch_scalars_out(const ItemScal* scal, int n_items, int n_c, double tol, int maxit, bool trivial,
                        double* sigma_bar, int* iters, double* resid, int* status, cudaStream_t st) {
  scalars_out_kernel<<<(n_items + 127) / 128, 128, 0, st>>>(scal, n_items, n_c, tol, maxit, trivial ? 1 : 0,
                                                            sigma_bar, iters, resid, status);
}

__global__ void field_copies_kernel(const double* fld, float* fld_f, dfloat* fld_df, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = fld[i];
    if (fld_f) fld_f[i] = (float)v;
    if (fld_df) {
      const float2 p = df_of(v);
      fld_df[i] = dfloat(p.x, p.y);
    }
  }
}

void launch_field_copies(const double* fld, float* fld_f, dfloat* fld_df, int64_t n, cudaStream_t st) {
  int64_t nb = (n + 255) / 256;
  if (nb > 4864) nb = 4864;
  field_copies_kernel<<<(unsigned)nb, 256, 0, st>>>(fld, fld_f, fld_df, n);
}

void launch_fill(const ItemDev* items, int n_items, int n_c, int64_t m, cudaStream_t st) {
  int64_t nb = (m + 255) / 256;
  if (nb > 2048) nb = 2048;
  fill_kernel<<<dim3((unsigned)nb, n_items), 256, 0, st>>>(items, n_c, m);
}
void launch_eff(const LatDev& dv, const EffArgs& a, int nblocks, int n_items, cudaStream_t st) {
  eff_kernel<<<dim3(nblocks, n_items), 256, 0, st>>>(dv, a);
}

template void launch_row_pass<double>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_row_pass<float>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_row_pass<dfloat>(const LatDev&, const RowArgs&, int, int, int, size_t, cudaStream_t);
template void launch_cg_row<double>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t, cudaStream_t);
template void launch_cg_row<float>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t, cudaStream_t);
template void launch_cg_row<dfloat>(const LatDev&, const RowArgs&, const CgArgs&, int, int, int, size_t, cudaStream_t);
template void launch_col_pass<double>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);
template void launch_col_pass<float>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);
template void launch_col_pass<dfloat>(const LatDev&, const ColArgs&, int, int, size_t, cudaStream_t);
template void launch_row_complex<double>(const LatDev&, const void*, void*, int, int, double, int, int, size_t,
                                         cudaStream_t, int);

template <typename K>
static cudaError_t set_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

int lat_kernel_attrs(size_t max_smem) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
    optin = (int)max_smem;
  cudaError_t e = set_smem(row_pass_kernel<double, 3, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<double, 6, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<float, 3, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<float, 6, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<double, 3, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<double, 6, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<float, 3, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<float, 6, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<dfloat, 3, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<dfloat, 6, MAT_FIELD>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<double, 1>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<double, 3>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<double, 6>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<float, 3>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<float, 6>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<dfloat, 3, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<dfloat, 6, MAT_TABLE>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<double, 6, MAT_ORTHO>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<float, 6, MAT_ORTHO>, optin);
  if (e == cudaSuccess) e = set_smem(row_pass_kernel<dfloat, 6, MAT_ORTHO>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<dfloat, 3>, optin);
  if (e == cudaSuccess) e = set_smem(col_pass_kernel<dfloat, 6>, optin);
  if (e == cudaSuccess) e = set_smem(row_complex_kernel<double>, optin);
  if (e == cudaSuccess) e = set_smem(cg_row_kernel<double, 3>, optin);
  if (e == cudaSuccess) e = set_smem(cg_row_kernel<double, 6>, optin);
  if (e == cudaSuccess) e = set_smem(cg_row_kernel<dfloat, 3>, optin);
  if (e == cudaSuccess) e = set_smem(cg_row_kernel<dfloat, 6>, optin);
  if (e == cudaSuccess) e = (cudaError_t)lat_gen_kernel_attrs(optin);
  return e == cudaSuccess ? 0 : (int)e;
}
