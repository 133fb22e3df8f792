// kernels_blue_cg.cu -- conjugate gradients on lattices whose largest divisor is transformed by chirp-z
// rows (Bluestein; plans with lat_plan::blue, binary64 only).
//
// The scheme is the one of the row kernels (kernels.cu, kernels_gen.cu): conjugate gradients on the
// discrete Lippmann-Schwinger equation A e = -Gamma0 C E with A = Gamma0 C, self-adjoint in the inner
// product <a, c>_C0, in the Chronopoulos-Gear form (q = A p carried by recurrence, both inner products of
// an iteration from one pass).  On a chirp-z plan the row transforms are separate launches (solve.cu,
// blue_rows), so a stage here is the stage arithmetic alone, grid-stride over the points:
//   CG_FWD_X  tau = C : x                                    (prologue; then forward transform)
//   CG_FULL0  r = -A x from the inverse transform, <r, r>_C0, ||r||^2; tau = C : r
//   CG_A      w = A r from the inverse transform, <w, r>_C0; the item's last block forms alpha, beta
//   CG_B      p = r + beta p, q = w + beta q, x += alpha p, r -= alpha q, <r, r>_C0, ||r||^2, the
//             residual report (Algorithm 1's measure ||r|| / ||eps^(0)||, Sec. 5.2); tau = C : r
#include <math.h>

#include <algorithm>

#include "kernels_dev.cuh"
#include "solve_detail.h"

namespace {

// the end of a stage in each block of an item: stage A sums <w, r>_C0 and the item's last block forms the
// step lengths; FULL0 and B sum <r, r>_C0 and ||r||^2 and the last block reports the residual, stopping at
// the rounding floor 1024 u ||r_0|| (u = 2^-53); the same recurrences as the row kernels' stage end
__device__ __forceinline__ void blue_cg_stage_end(int stage, double acc0, double acc1, const ItemDev* item,
                                                  ItemScal* isc, int item_i, const IterArgs& it, double* red,
                                                  int* s_last) {
  double* partials = it.partials + item_i * it.pstride;
  const double vv[2] = {acc0, acc1};
  double tot[2];
  if (stage == CG_A) {
    if (!item_reduce<1>(vv, partials, isc, red, s_last, tot)) return;
    if (threadIdx.x == 0) {
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
    if (!item_reduce<2>(vv, partials, isc, red, s_last, tot)) return;
    if (threadIdx.x == 0) {
      const double rr = sqrt(tot[1]) / item->norm0;
      if (stage == CG_FULL0) isc->cg_r0 = rr;
      isc->cg_gamma = tot[0];
      item_report(rr, isc, item_i, it, rr <= 0x1p-43 * isc->cg_r0);
    }
  }
}

// the pointwise part of a conjugate-gradient stage: the vector updates and inner products of the stage
// and, except in stage A, tau = C : v back into T as a real signal; grid-stride over the points
template <int NC>
__global__ void __launch_bounds__(256) blue_cg_point_kernel(LatDev dv, RowArgs a, CgArgs cg) {
  constexpr int n_c = NC;
  const int item_i = blockIdx.y;
  const ItemDev* item = a.items + item_i;
  ItemScal* isc = (ItemScal*)((char*)a.it.scal + (size_t)item_i * 256);
  const int stage = cg.stage;
  if (stage != CG_FWD_X && *(volatile const int*)&isc->done != ITEM_ACTIVE) return;
  __shared__ double red[32];
  __shared__ int s_last;
  const int64_t m = dv.m;
  double2* T = (double2*)a.T + item_i * a.t_stride;
  const size_t voff = (size_t)item_i * cg.vstride;
  double* x = item->eps;
  double* r = cg.r + voff;
  double* p = cg.p + voff;
  double* q = cg.q + voff;
  double* w = cg.w + voff;
  const bool from_spectrum = (stage == CG_FULL0 || stage == CG_A);
  const double alpha = (stage == CG_B) ? isc->cg_alpha : 0.0, beta = (stage == CG_B) ? isc->cg_beta : 0.0;
  const double lam0 = item->lam0, two_mu0 = 2.0 * item->mu0;
  double acc0 = 0.0, acc1 = 0.0;   // <r, r>_C0 (or <w, r>_C0) and ||r||^2
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m; g += (int64_t)gridDim.x * blockDim.x) {
    double v[NC];
    if (from_spectrum) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) v[c] = T[c * m + g].x;
    }
    if (stage == CG_FWD_X) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) v[c] = x[c * m + g];
    } else if (stage == CG_FULL0) {
#pragma unroll
      for (int c = 0; c < n_c; ++c) r[c * m + g] = v[c];
      acc0 += c0_dot<double, NC>(v, v, lam0, two_mu0);
      acc1 += frob2<double, NC>(v);
    } else if (stage == CG_A) {
      double s[NC];
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        v[c] = -v[c];
        w[c * m + g] = v[c];
        s[c] = r[c * m + g];
      }
      acc0 += c0_dot<double, NC>(v, s, lam0, two_mu0);
      continue;   // no polarization: the next stage starts from the updated vectors
    } else {
#pragma unroll
      for (int c = 0; c < n_c; ++c) {
        const int64_t o = c * m + g;
        double rv = r[o], pv = p[o], qv = q[o];
        pv = rv + beta * pv;
        qv = w[o] + beta * qv;
        const double xv = x[o] + alpha * pv;
        rv = rv - alpha * qv;
        p[o] = pv;
        q[o] = qv;
        x[o] = xv;
        r[o] = rv;
        v[c] = rv;
      }
      acc0 += c0_dot<double, NC>(v, v, lam0, two_mu0);
      acc1 += frob2<double, NC>(v);
    }
    // tau = C : v for the next transform
    const double* Cp = item->Dtab + (int)item->phase[g] * n_c * n_c;
#pragma unroll
    for (int c = 0; c < n_c; ++c) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < n_c; ++k) t += ldg_r(Cp + c * n_c + k) * v[k];
      T[c * m + g] = make_double2(t, 0.0);
    }
  }
  if (stage == CG_FWD_X) return;
  blue_cg_stage_end(stage, acc0, acc1, item, isc, item_i, a.it, red, &s_last);
}

}  // namespace

namespace latms_detail {

void launch_blue_cg_point(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items,
                          cudaStream_t st) {
  const dim3 grid(nblocks, n_items);
  if (dv.n_c == 6) blue_cg_point_kernel<6><<<grid, 256, 0, st>>>(dv, a, cg);
  else blue_cg_point_kernel<3><<<grid, 256, 0, st>>>(dv, a, cg);
}

}  // namespace latms_detail
