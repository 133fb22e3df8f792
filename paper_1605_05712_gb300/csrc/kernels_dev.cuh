// kernels_dev.cuh -- device helpers shared by the solver kernels (kernels.cu) and the mixed-radix
// kernels (kernels_gen.cu): the Green operator of Sec. 3.1 at a decoded frequency, double-float
// accumulation, cp.async tile loads, block reductions and the per-item convergence report of
// Algorithm 1 (Sec. 3.2, with the Cauchy criterion of Sec. 5.2).
#pragma once
#include <math.h>

#include <type_traits>

#include "fft_smem.cuh"
#include "kernels.cuh"

// kernel precisions: binary64, binary32 (mixed), double-float pairs on the binary32 pipes
template <typename R> constexpr bool is_f32 = std::is_same<R, float>::value;
template <typename R> constexpr bool is_df = std::is_same<R, dfloat>::value;

template <typename R> __device__ __forceinline__ R ldg_r(const R* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfloat ldg_r<dfloat>(const dfloat* p) { return ldg_df(p); }
// start the 128-byte line holding p towards L2 (no value comes back)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// two consecutive table entries in one read-only load (p aligned to twice the entry size)
__device__ __forceinline__ void ldg_r2(const double* p, double& a, double& b) {
  const double2 v = __ldg((const double2*)p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ldg_r2(const float* p, float& a, float& b) {
  const float2 v = __ldg((const float2*)p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ldg_r2(const dfloat* p, dfloat& a, dfloat& b) {
  const float4 v = __ldg((const float4*)p);
  a = dfloat(v.x, v.y);
  b = dfloat(v.z, v.w);
}

// ------------------------------------------------------------------ Green operator (Sec. 3.1)
// sc Gamma0(h) : tau for isotropic C0 (closed form of grad (grad^H C0 grad)^{-1} grad^H), applied to the
// real and imaginary parts of tau_hat at once so that the products of h and the constants are shared:
//   (Gamma0 : tau)_ij = [c1 (h_i w_j + h_j w_i) - q h_i h_j] / |h|^2,  q = c2 (h . w) / |h|^2,
//   w = tau h, c1 = 1/(2 mu0), c2 = (lam0 + mu0) / (mu0 (lam0 + 2 mu0)).
// Written as a symmetrized outer product, sc Gamma0 : tau = k (x) z + z (x) k with k = sc h / |h|^2 and
//   z = c1 w - (q / 2) h = w' - (c2 mu0 / |h|^2)(h . w') h,   w' = tau (c1 h),
// every product folds into a fused multiply-add: 25 operations per part after the shared setup (the
// grouped form took ~43).  No intermediate leaves the binary32 range for |h| < 2^31.
template <typename Real, int D>
__device__ __forceinline__ void gamma_apply2(const Real* h, Real c1, Real c2mu0, Real sc, const Real* tr,
                                             const Real* ti, Real* gr, Real* gi) {
  Real n2 = h[0] * h[0] + h[1] * h[1];
  if constexpr (D == 3) n2 = n2 + h[2] * h[2];
  const Real a = Real(1) / n2;
  const Real ka = sc * a, qf = c2mu0 * a;
  Real hc[3], hk[3], hk2[3];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    hc[i] = c1 * h[i];
    hk[i] = ka * h[i];
    hk2[i] = hk[i] + hk[i];
  }
  auto one = [&](const Real* t, Real* out) {
    Real A[3][3];
    if constexpr (D == 2) {
      A[0][0] = t[0]; A[1][1] = t[1]; A[0][1] = A[1][0] = t[2];
    } else {
      A[0][0] = t[0]; A[1][1] = t[1]; A[2][2] = t[2];
      A[1][2] = A[2][1] = t[3]; A[0][2] = A[2][0] = t[4]; A[0][1] = A[1][0] = t[5];
    }
    Real w[3], s = Real(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      Real acc = A[i][0] * hc[0];
#pragma unroll
      for (int j = 1; j < D; ++j) acc += A[i][j] * hc[j];
      w[i] = acc;
      s += h[i] * acc;
    }
    const Real qs = qf * s;
    Real z[3];
#pragma unroll
    for (int i = 0; i < D; ++i) z[i] = w[i] - qs * h[i];
#define GAMO(i, j) (hk[i] * z[j] + hk[j] * z[i])
    if constexpr (D == 2) {
      out[0] = hk2[0] * z[0]; out[1] = hk2[1] * z[1]; out[2] = GAMO(0, 1);
    } else {
      out[0] = hk2[0] * z[0]; out[1] = hk2[1] * z[1]; out[2] = hk2[2] * z[2];
      out[3] = GAMO(1, 2); out[4] = GAMO(0, 2); out[5] = GAMO(0, 1);
    }
#undef GAMO
  };
  one(tr, gr);
  one(ti, gi);
}

__device__ __forceinline__ int64_t mod_ed(const LatDev& dv, int64_t v) {
  if (dv.ed_mask >= 0) return v & dv.ed_mask;
  int64_t r = v % dv.ed;
  return r < 0 ? r + dv.ed : r;
}

// h~ = M^T v' with v' the symmetric representative of v (mod e_d) in [-e_d/2, e_d/2)
template <int D>
__device__ __forceinline__ void v_to_h(const LatDev& dv, const int64_t* v, int64_t* h) {
  int64_t vp[D];
#pragma unroll
  for (int r = 0; r < D; ++r) vp[r] = (2 * v[r] >= dv.ed) ? v[r] - dv.ed : v[r];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) acc += dv.MT[i][j] * vp[j];
    h[i] = acc;
  }
}

// Green-operator constants of one item in the kernel's precision
template <typename Real>
struct GreenK {
  Real c1, c2mu0, sc;  // c2mu0 = c2 mu0 (gamma_apply2)
  Real lam0, mu0;      // Eyre-Milton: C0 applied after Gamma0
};
template <typename Real>
__device__ __forceinline__ GreenK<Real> green_consts(const ItemDev* item, const MatArgs& mt) {
  GreenK<Real> g;
  if constexpr (is_f32<Real>) {
    g.c1 = item->c1f;
    g.c2mu0 = item->c2f * item->mu0f;
    g.lam0 = item->lam0f;
    g.mu0 = item->mu0f;
    g.sc = mt.gscale_f;
  } else if constexpr (is_df<Real>) {  // host-made pairs: no binary64 conversions per thread
    g.c1 = item->c1_df;
    g.c2mu0 = item->c2_df * item->mu0_df;
    g.lam0 = item->lam0_df;
    g.mu0 = item->mu0_df;
    g.sc = mt.gscale_df;
  } else {
    g.c1 = item->c1;
    g.c2mu0 = item->c2 * item->mu0;
    g.lam0 = item->lam0;
    g.mu0 = item->mu0;
    g.sc = mt.gscale;
  }
  return g;
}

// symmetric representative and h~ = M^T v' in 32-bit arithmetic (plan guarantees the range)
template <int D>
__device__ __forceinline__ void v_to_h32(const LatDev& dv, const uint32_t* v, int32_t* h) {
  const int32_t ed = (int32_t)dv.ed;
  int32_t vp[D];
#pragma unroll
  for (int r = 0; r < D; ++r) vp[r] = (2u * v[r] >= (uint32_t)ed) ? (int32_t)v[r] - ed : (int32_t)v[r];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    int32_t acc = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) acc += (int32_t)dv.MT[i][j] * vp[j];
    h[i] = acc;
  }
}

// eps_hat = -Gammabar0(k) : tau_hat / m at the frequency with v = e_d Q^{-T} E^{-1} k (mod e_d);
// in/out are n_c complex values.  v == 0 (k = 0) -> E (or 0 for an increment).
// Real h~ components come from the 32-bit path when the plan allows it, else from int64.
template <typename Real, int NC>
__device__ __forceinline__ void green_point_h(const LatDev& dv, const MatArgs& mt, const ItemDev* item,
                                              const GreenK<Real>& gk, bool zero, bool boundary, const Real* h,
                                              const Real* h2, typename cplx_of<Real>::type* val) {
  typedef typename cplx_of<Real>::type C;
  constexpr int d = (NC == 6) ? 3 : 2, n_c = NC;
  if (zero) {
    if (mt.scheme == LAT_SCHEME_EYRE_MILTON) {
      // <u> = <v> + 2 C0 : E (the forward transform is unnormalized: -sc = 1/m); an increment keeps <v>
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        val[c].x = -gk.sc * val[c].x;
        val[c].y = -gk.sc * val[c].y;
        if (!mt.increment) val[c].x += Real(item->twoC0E[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < n_c; ++c) val[c] = mt.increment ? cmake<C>(0.0, 0.0) : cmake<C>(item->E[c], 0.0);
    }
    return;
  }
  if (boundary && mt.boundary_zero) {
#pragma unroll
    for (int c = 0; c < n_c; ++c) val[c] = cmake<C>(0.0, 0.0);
    return;
  }
  Real tr[NC], ti[NC], gr[NC], gi[NC];   // gr, gi = sc Gamma0 : tau_hat
#pragma unroll
  for (int c = 0; c < n_c; ++c) tr[c] = val[c].x, ti[c] = val[c].y;
  gamma_apply2<Real, d>(h, gk.c1, gk.c2mu0, gk.sc, tr, ti, gr, gi);
  if (boundary) {
    // average with -h(-k): Gamma0 is even in h, so evaluate at h(-k) directly
    Real gr2[NC], gi2[NC];
    gamma_apply2<Real, d>(h2, gk.c1, gk.c2mu0, gk.sc, tr, ti, gr2, gi2);
#pragma unroll
    for (int c = 0; c < n_c; ++c) gr[c] = Real(0.5) * (gr[c] + gr2[c]), gi[c] = Real(0.5) * (gi[c] + gi2[c]);
  }
  if (mt.scheme == LAT_SCHEME_EYRE_MILTON) {
    // u_hat = v_hat / m - 2 C0 : Gamma0 : v_hat / m = -sc v_hat + 2 C0 : (sc Gamma0 : v_hat)
    Real trr = Real(0), tri = Real(0);
#pragma unroll
    for (int c = 0; c < d; ++c) trr += gr[c], tri += gi[c];
    const Real two = Real(2);
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      Real cr = two * gk.mu0 * gr[c], ci = two * gk.mu0 * gi[c];
      if (c < d) cr += gk.lam0 * trr, ci += gk.lam0 * tri;
      val[c].x = two * cr - gk.sc * tr[c];
      val[c].y = two * ci - gk.sc * ti[c];
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < n_c; ++c) {
    val[c].x = gr[c];
    val[c].y = gi[c];
  }
}

// h <- L^{-T} h in the kernel's precision (the matrix comes in all three forms, no binary64 conversion)
template <typename Real>
__device__ __forceinline__ Real cell_entry(const LatDev& dv, int i, int j) {
  if constexpr (is_f32<Real>) return dv.cellT_f[i][j];
  else if constexpr (is_df<Real>) return dfloat(dv.cellT_f[i][j], dv.cellT_lo[i][j]);
  else return dv.cellT[i][j];
}
template <typename Real, int D>
__device__ __forceinline__ void cell_map(const LatDev& dv, Real* h) {
  Real t[3];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Real acc = Real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) acc += cell_entry<Real>(dv, i, j) * h[j];
    t[i] = acc;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) h[i] = t[i];
}

// frequency from the per-axis spectral indices: kk[x] for the logical axes (row last)
// the Green step at the frequency whose fractional coordinates are v / e_d: v32 are the per-component
// sums of kk[x] cv[x] in wrapping 32-bit arithmetic (used when dv.h32), v64 the same sums in int64
template <typename Real, int NC>
__device__ __forceinline__ void green_from_v(const LatDev& dv, const MatArgs& mt, const ItemDev* item,
                                             const GreenK<Real>& gk, const uint32_t* v32, const int64_t* v64,
                                             typename cplx_of<Real>::type* val) {
  constexpr int d = (NC == 6) ? 3 : 2;
  Real h[3] = {0, 0, 0}, h2[3] = {0, 0, 0};
  bool zero = true, boundary = false;
  if (dv.h32) {
    uint32_t v[3], vn[3];
    const uint32_t mask = (uint32_t)dv.ed_mask;
#pragma unroll
    for (int r = 0; r < d; ++r) {
      v[r] = v32[r] & mask;   // exact mod 2^32, hence mod e_d
      zero = zero && (v[r] == 0u);
      boundary = boundary || (2u * v[r] == (uint32_t)dv.ed);  // v' = -e_d/2: -v has the same representative
      vn[r] = (0u - v[r]) & mask;
    }
    if (!zero) {
      int32_t hi[3] = {0, 0, 0};
      v_to_h32<d>(dv, v, hi);
#pragma unroll
      for (int i = 0; i < d; ++i) h[i] = (Real)hi[i];
      if (boundary) {
        v_to_h32<d>(dv, vn, hi);
#pragma unroll
        for (int i = 0; i < d; ++i) h2[i] = (Real)hi[i];
      }
    }
  } else {
    int64_t v[3] = {0, 0, 0}, vn[3] = {0, 0, 0};
#pragma unroll
    for (int r = 0; r < d; ++r) {
      v[r] = mod_ed(dv, v64[r]);
      zero = zero && (v[r] == 0);
      boundary = boundary || (2 * v[r] == dv.ed);
      vn[r] = mod_ed(dv, dv.ed - v[r]);
    }
    if (!zero) {
      int64_t hi[3] = {0, 0, 0};
      v_to_h<d>(dv, v, hi);
#pragma unroll
      for (int i = 0; i < d; ++i) h[i] = (Real)hi[i];
      if (boundary) {
        v_to_h<d>(dv, vn, hi);
#pragma unroll
        for (int i = 0; i < d; ++i) h2[i] = (Real)hi[i];
      }
    }
  }
  if (dv.cell && !zero) {
    // transformed pattern P_L(M) (Sec. 3.3, Def. 3.3): the index h is the frequency L^{-T} h
    cell_map<Real, d>(dv, h);
    if (boundary) cell_map<Real, d>(dv, h2);
  }
  green_point_h<Real, NC>(dv, mt, item, gk, zero, boundary, h, h2, val);
}

// adds the contribution k cv[x] of spectral index k on logical axis x to the sums of green_from_v
template <int D>
__device__ __forceinline__ void v_add(const LatDev& dv, int x, int k, uint32_t* v32, int64_t* v64) {
#pragma unroll
  for (int r = 0; r < D; ++r) {
    v32[r] += (uint32_t)k * (uint32_t)dv.ax_cv[x][r];
    v64[r] += (int64_t)k * dv.ax_cv[x][r];
  }
}

// frequency from the per-axis spectral indices: kk[x] for the logical axes (row last)
template <typename Real, int NC>
__device__ __forceinline__ void green_at(const LatDev& dv, const MatArgs& mt, const ItemDev* item,
                                         const GreenK<Real>& gk, const int* kk,
                                         typename cplx_of<Real>::type* val) {
  constexpr int d = (NC == 6) ? 3 : 2;
  uint32_t v32[3] = {0u, 0u, 0u};
  int64_t v64[3] = {0, 0, 0};
  for (int x = 0; x < dv.nax; ++x) v_add<d>(dv, x, kk[x], v32, v64);
  green_from_v<Real, NC>(dv, mt, item, gk, v32, v64, val);
}

// ------------------------------------------------------------------ per-point stiffness field
// Voigt index (11, 22, 33, 23, 13, 12 -> 0..5) of tensor component c; 2-D (plane strain) takes 11, 22, 12
template <int NC>
__device__ __forceinline__ constexpr int fld_vidx(int c) { return NC == 6 ? c : (c == 2 ? 5 : c); }
// position of entry (i, j), i <= j, of a symmetric 6x6 matrix in its row-major upper triangle
__device__ __forceinline__ constexpr int fld_tri(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }

// tau = C_y : e - C0 : e at one point, from the 21 upper-triangle Voigt entries of C_y (6x6 on engineering
// strain; plane p of fld at stride fs holds entry p); e and tau tensor components.  C_y : e is the
// symmetric product on the engineering strain, each stored entry read once.
template <typename Real, int NC>
__device__ __forceinline__ void field_polarize(const Real* fld, int64_t fs, int64_t g, Real lam0, Real two_mu0,
                                               const Real* e, Real* tau) {
  constexpr int D = (NC == 6) ? 3 : 2;
  Real ev[NC], s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    ev[c] = c < D ? e[c] : e[c] + e[c];
    s[c] = Real(0);
  }
#pragma unroll
  for (int a = 0; a < NC; ++a)
#pragma unroll
    for (int b = a; b < NC; ++b) {
      const int va = fld_vidx<NC>(a), vb = fld_vidx<NC>(b);
      const Real cab = ldg_r(fld + fld_tri(va < vb ? va : vb, va < vb ? vb : va) * fs + g);
      s[a] += cab * ev[b];
      if (b != a) s[b] += cab * ev[a];
    }
  Real tr = e[0];
#pragma unroll
  for (int c = 1; c < D; ++c) tr += e[c];
#pragma unroll
  for (int c = 0; c < NC; ++c) tau[c] = c < D ? s[c] - (lam0 * tr + two_mu0 * e[c]) : s[c] - two_mu0 * e[c];
}

// ------------------------------------------------------------------ double-float accumulation
// Sum of squares carried as an unevaluated pair of binary32 values (hi + lo), with Knuth's TwoSum
// for the addition and the FMA-based exact product (Dekker) for the square: about 2^-48 relative,
// the accuracy of a binary64 accumulator, computed on the binary32 pipes.
struct DF {
  float hi, lo;
};
// strain held as a double-float pair (hi, lo) in the 8 bytes of its binary64 slot during a mixed solve
// (binary32 arithmetic only: GB300 issues binary64 at 1/58 of the binary32 rate)
__device__ __forceinline__ void df_acc(float& hi, float& lo, float x) {  // (hi, lo) += x
  float s, e, h, l;
  two_sum(hi, x, s, e);
  fast_two_sum(s, __fadd_rn(lo, e), h, l);
  hi = h;
  lo = l;
}
__device__ __forceinline__ float df_diff(float x, float hi, float lo) {  // x - (hi + lo), rounded once
  float s, e;
  two_sum(x, -hi, s, e);
  return __fadd_rn(s, __fsub_rn(e, lo));
}
__device__ __forceinline__ float2 df_of(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ void df_add_sq(DF& acc, float x) {
  const float p = __fmul_rn(x, x);
  const float pe = __fmaf_rn(x, x, -p);      // x*x = p + pe exactly
  float s, e;
  two_sum(acc.hi, p, s, e);
  fast_two_sum(s, __fadd_rn(__fadd_rn(acc.lo, pe), e), acc.hi, acc.lo);
}

// ------------------------------------------------------------------ asynchronous tile loads
// global -> shared copies that bypass registers (cp.async, sm_80 and later), so that a thread has all
// its tile elements in flight at once; cp.async.wait_all then waits for this thread's copies, and a
// __syncthreads() after it publishes the tile.  Both addresses are aligned to the element size.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* dst, const C* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
  } else {
    static_assert(sizeof(C) == 8, "complex element of 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// block sum of x into out (valid on thread 0); red has >= 32 doubles
static __device__ double block_sum(double x, double* red) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double t = 0;
  if (wid == 0) {
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// block sum of a double-float pair into a binary64 value (valid on thread 0): the warps add pairs (binary32
// pipes) and convert once per warp, so the pair kernels issue no binary64 arithmetic per thread
static __device__ double block_sum(dfloat x, double* red) {
  for (int o = 16; o > 0; o >>= 1)
    x = x + dfloat(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = (double)x;
  __syncthreads();
  double t = 0;
  if (wid == 0) {
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// ordered sum of n values written by other blocks (bypasses L1), result on every lane of warp 0
static __device__ double ordered_sum(const double* p, int n) {
  double t = 0;
  for (int i = threadIdx.x; i < n; i += 32) t += __ldcg(p + i);
  return warp_sum(t);
}

// per-item reduction of NV values (binary64, or pairs in the pair kernels) over the blocks of grid.x: block
// sums go to
// partials[v * gridDim.x + blockIdx.x]; the item's last block to arrive returns true on warp 0, with
// the totals (summed in block order) in tot on lane 0; every other thread returns false
template <int NV, typename V>
__device__ __forceinline__ bool item_reduce(const V* v, double* partials, ItemScal* isc, double* red,
                                            int* s_last, double* tot) {
  double bs[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) bs[k] = block_sum(v[k], red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = bs[k];
    __threadfence();
    const unsigned t = atomicAdd(&isc->counter, 1u);
    *s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!*s_last || threadIdx.x >= 32) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = ordered_sum(partials + k * gridDim.x, gridDim.x);
  return true;
}

// thread 0 of an item's last block: record residual r, decide the item's state (stop: end the
// iteration whatever r is); the last item to report in this iteration recounts the active items and
// sets the WHILE condition
__device__ __forceinline__ void item_report(double r, ItemScal* isc, int item_i, const IterArgs& it,
                                            bool stop = false) {
  const int n = isc->iter + 1;
  isc->iter = n;
  if (n - 1 < LAT_HIST_CAP) it.hist[(size_t)item_i * LAT_HIST_CAP + n - 1] = r;
  // divergence: a residual that grew for LAT_DIVERGE_STEPS iterations in a row to above 1 (an increment
  // larger than the start strain) belongs to an iteration that does not contract (e.g. C0 too soft)
  const int grow = (n > 1 && r > isc->last_r) ? isc->grow + 1 : 0;
  isc->grow = grow;
  const bool diverging = grow >= LAT_DIVERGE_STEPS && r > 1.0;
  if (diverging) isc->diverged = 1;
  isc->last_r = r;
  const bool cont = isfinite(r) && !(r < it.tol) && n < it.maxit && !stop && !diverging;
  isc->counter = 0u;
  if (!cont) isc->done = ITEM_DONE;
  else if (it.pause_tol > 0 && r < it.pause_tol) isc->done = ITEM_PAUSED;
  else isc->done = ITEM_ACTIVE;
  __threadfence();
  GlobScal* gs = it.glob;
  const unsigned arrived = atomicAdd(&gs->arrivals, 1u);
  if ((int)arrived == *(volatile int*)&gs->active - 1) {  // every active item has reported
    int active = 0;
    for (int i = 0; i < it.n_items; ++i)
      active += !*(volatile const int*)&((const ItemScal*)((const char*)it.scal + (size_t)i * 256))->done;
    gs->active = active;
    gs->arrivals = 0u;
    if (it.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)it.cond, active > 0 ? 1u : 0u);
  }
}

// ------------------------------------------------------------------ conjugate-gradient inner products
// a : C0 : c for isotropic C0 on tensor components (shear components stored once, counted twice)
template <typename Real, int NC>
__device__ __forceinline__ Real c0_dot(const Real* a, const Real* c, Real lam0, Real two_mu0) {
  constexpr int D = (NC == 6) ? 3 : 2;
  Real ta = Real(0), tc = Real(0), s = Real(0), sh = Real(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ta += a[k];
    tc += c[k];
    s += a[k] * c[k];
  }
#pragma unroll
  for (int k = D; k < NC; ++k) sh += a[k] * c[k];
  return lam0 * (ta * tc) + two_mu0 * (s + (sh + sh));
}
template <typename Real, int NC>
__device__ __forceinline__ Real frob2(const Real* a) {
  constexpr int D = (NC == 6) ? 3 : 2;
  Real s = Real(0), sh = Real(0);
#pragma unroll
  for (int k = 0; k < D; ++k) s += a[k] * a[k];
#pragma unroll
  for (int k = D; k < NC; ++k) sh += a[k] * a[k];
  return s + (sh + sh);
}
