// solve.cu -- the solve drivers: workspace layout, launch geometry, batching of independent
// problems and the CUDA-graph WHILE loop that runs Algorithm 1 (Sec. 3.2, arXiv 1605.05712)
// without a host round trip per iteration.
//
// Every solve is a batch of "items" (load cases of one microstructure, or independent
// microstructures on one lattice): each kernel launch covers all items (grid.y), each item keeps
// its own strain, spectrum, material tables, reference medium and convergence state, and blocks of
// finished items return at once.  The loop runs until every item has stopped.
//
// The same drivers run the accelerated schemes of lat_solve_opts.scheme: the Eyre-Milton iteration
// (the same passes with another Green step and per-phase (C + C0)^{-1} tables) and conjugate
// gradients (the two cg_row_kernel stages around the column passes, with its own prologue and a loop
// condition that starts from the active count).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "solve_detail.h"

namespace latms_detail {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  return n;
}

int ensure_attrs() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (done[dev]) return 0;
  int rc = lat_kernel_attrs(kMaxSmem);
  if (rc == 0) done[dev] = true;
  return rc;
}

LatDev make_dev(const lat_plan* P, int kind) {
  LatDev dv;
  memset(&dv, 0, sizeof(dv));
  dv.d = P->d;
  dv.n_c = P->d * (P->d + 1) / 2;
  dv.nax = P->nax;
  dv.Rlen = P->Rlen;
  dv.Rh = P->Rh;
  dv.log2Rh = P->log2Rh;
  dv.m = P->m;
  dv.nrows = P->nrows;
  dv.ed = P->ed;
  dv.ed_mask = ((P->ed & (P->ed - 1)) == 0) ? P->ed - 1 : -1;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dv.MT[i][j] = P->M[j][i];
  {  // |h~_i| = |sum_j M_ji v'_j| <= (e_d / 2) sum_j |M_ji|
    double hb = 0;
    for (int i = 0; i < P->d; ++i) {
      double r = 0;
      for (int j = 0; j < P->d; ++j) r += fabs((double)P->M[j][i]);
      hb = std::max(hb, r * (double)P->ed / 2);
    }
    dv.h32 = (dv.ed_mask >= 0 && P->ed <= (int64_t(1) << 31) && hb < 2147483647.0) ? 1 : 0;
  }
  for (int a = 0; a < P->nax; ++a) {
    dv.ax_len[a] = P->ax[a].len;
    dv.ax_log2[a] = P->ax[a].log2len;
    for (int r = 0; r < 3; ++r) dv.ax_cv[a][r] = P->ax[a].cv[r];
  }
  dv.general = P->general;
  for (int a = 0; a < LAT_MAX_AX; ++a) {
    dv.ax_nrad[a] = P->ax_nrad[a];
    dv.ax_twoff[a] = P->ax_twoff[a];
    for (int r = 0; r < LAT_MAX_RADIX; ++r) dv.ax_rad[a][r] = P->ax_rad[a][r];
  }
  dv.blue = P->blue;
  dv.blue_L = P->blue_L;
  dv.blue_lgA = P->blue_lgA;
  dv.blue_lgB = P->blue_lgB;
  dv.blue_chirp = P->d_chirp;
  dv.blue_bh = P->d_bh;
  dv.blue_plan = P;
  dv.split = P->split;
  dv.split_n1 = P->split_n1;
  dv.split_lo_log2 = P->split_lo_log2;
  dv.split_e = P->split_e;
  dv.stw_hi_n = P->stw_hi_n;
  dv.tw_log2 = P->tw_log2;
  dv.cell = P->has_cell;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double v = P->has_cell ? P->cell_LinvT[i][j] : (i == j ? 1.0 : 0.0);
      dv.cellT[i][j] = v;
      dv.cellT_f[i][j] = (float)v;
      dv.cellT_lo[i][j] = (float)(v - (double)(float)v);
    }
  dv.tw = kind == LAT_MIXED ? (const void*)P->d_twf : kind == LAT_DF64 ? (const void*)P->d_twdf : (const void*)P->d_tw;
  dv.stw = kind == LAT_MIXED ? (const void*)P->d_stwf : kind == LAT_DF64 ? (const void*)P->d_stwdf : (const void*)P->d_stw;
  dv.lf = P->d_lf;
  dv.rc = P->d_rc;
  return dv;
}

int tune_bucket(int n_items) {
  int b = 0;
  while (b < 7 && (2 << b) <= n_items) ++b;
  return b;
}

size_t row_smem_bytes(const lat_plan* P, int n_f, size_t cs, bool nyq, int rpc) {
  const int row_len = nyq ? P->Rh : P->Rlen;
  // the padded tile of the rows, the Nyquist values of each line, 32 doubles for block reductions
  return ((size_t)tile_span((int64_t)n_f * rpc * row_len, cs) + (nyq ? (size_t)n_f * rpc : 0)) * cs +
         32 * sizeof(double);
}
size_t col_smem_bytes(const lat_plan* P, int n_f, size_t cs, int k, int64_t w) {
  return (size_t)tile_span((int64_t)n_f * P->grp[k].G * w, cs) * cs;
}

int geometry_set_rpc(const lat_plan* P, int n_f, size_t cs, bool nyq, int rpc, Geometry& g) {
  if (rpc < 1 || P->nrows % rpc != 0) return lat_fail(LAT_ERR_ARG, "rows per block must divide the row count");
  const size_t sm = row_smem_bytes(P, n_f, cs, nyq, rpc);
  if (sm > kMaxSmem) return lat_fail(LAT_ERR_UNSUPPORTED, "row does not fit in shared memory");
  g.rpc = rpc;
  g.row_blocks = (int)(P->nrows / rpc);
  g.row_smem = sm;
  return LAT_OK;
}
int geometry_set_w(const lat_plan* P, int n_f, size_t cs, int row_slots, bool nyq, int k, int64_t w, Geometry& g) {
  const LatGroup& G = P->grp[k];
  const int64_t ic = G.inner * row_slots;
  if (w < 1 || (w & (w - 1)) != 0 || w > ic) return lat_fail(LAT_ERR_ARG, "tile width must be a power of two <= the columns");
  if (col_smem_bytes(P, n_f, cs, k, w) > kMaxSmem) return lat_fail(LAT_ERR_UNSUPPORTED, "column group does not fit in shared memory");
  const int64_t wN = std::min<int64_t>(w, G.inner);
  g.w[k] = (int)w;
  g.wN[k] = (int)wN;
  g.tiles_main[k] = ic / w;
  g.tiles_nyq[k] = nyq ? G.inner / wN : 0;
  g.col_smem[k] = col_smem_bytes(P, n_f, cs, k, w);
  return LAT_OK;
}

// row_slots = Rh (solver) or Rlen (complex transform); n_f planes per tile; n_items blocks in grid.y;
// kind >= 0: a solve of that precision, which takes the plan's autotuned shapes when it has them
// launch shapes of a general plan's mixed-radix kernels: two tile buffers (ping-pong) of n_f planes; rows
// per block a power of two dividing the row count, column tiles of a power-of-two width (the last tile
// of an axis may be ragged)
static int geometry_general(const lat_plan* P, int n_f, size_t cs, Geometry& g, int n_items) {
  const int nsm = num_sms();
  const int64_t nrows = P->nrows, R = P->Rlen;
  auto row_smem = [&](int rpc) { return 2 * (size_t)n_f * rpc * R * cs + 32 * sizeof(double); };
  if (P->blue) {   // chirp-z rows: the pointwise step runs on its own, grid-stride over the points
    g.rpc = 1;
    g.row_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P->m + 1023) / 1024, 1024));
    g.row_smem = 0;
  } else {
    if (row_smem(1) > kMaxSmem) return lat_fail(LAT_ERR_UNSUPPORTED, "row does not fit in shared memory");
    int rpc = 1;
    while (nrows % (2 * rpc) == 0 && row_smem(2 * rpc) <= kRowSmemTarget && n_items * (nrows / (2 * rpc)) >= 2 * nsm)
      rpc *= 2;
    g.rpc = rpc;
    g.row_blocks = (int)(nrows / rpc);
    g.row_smem = row_smem(rpc);
  }
  for (int k = 0; k < P->ngroups; ++k) {
    const LatGroup& G = P->grp[k];
    const int64_t ic = G.inner * R;
    auto smem = [&](int64_t w) { return 2 * (size_t)n_f * G.G * w * cs; };
    if (smem(1) > kMaxSmem) return lat_fail(LAT_ERR_UNSUPPORTED, "column does not fit in shared memory");
    int64_t w = 32;
    while (w > 1 && (w / 2 >= ic || smem(w) > kColSmemMax || n_items * G.outer * ((ic + w - 1) / w) < 2 * nsm)) w /= 2;
    g.w[k] = (int)w;
    g.wN[k] = 0;
    g.tiles_main[k] = (ic + w - 1) / w;
    g.tiles_nyq[k] = 0;
    g.col_smem[k] = smem(w);
  }
  return LAT_OK;
}

int geometry(const lat_plan* P, int n_f, size_t cs, int row_slots, bool nyq, Geometry& g, int n_items, int kind) {
  if (P->general) return geometry_general(P, n_f, cs, g, n_items);
  const int nsm = num_sms();
  const int64_t nrows = P->nrows;
  int rpc = 1;
  while (nrows % (2 * rpc) == 0 && row_smem_bytes(P, n_f, cs, nyq, 2 * rpc) <= kRowSmemTarget &&
         n_items * (nrows / (2 * rpc)) >= 2 * nsm)
    rpc *= 2;
  if (int rc = geometry_set_rpc(P, n_f, cs, nyq, rpc, g)) return rc;
  for (int k = 0; k < P->ngroups; ++k) {
    const LatGroup& G = P->grp[k];
    const int64_t ic = G.inner * row_slots;
    int64_t w = std::min<int64_t>(32, ic);
    while (w > 1 && (col_smem_bytes(P, n_f, cs, k, w) > kColSmemMax || n_items * G.outer * (ic / w) < 2 * nsm)) w /= 2;
    if (int rc = geometry_set_w(P, n_f, cs, row_slots, nyq, k, w, g)) return rc;
  }
  if (kind >= 0 && kind < 3 && nyq) {
    const lat_plan::Tune& t = P->tune[kind][tune_bucket(n_items)];
    if (t.valid) {
      Geometry tg = g;
      bool ok = geometry_set_rpc(P, n_f, cs, nyq, t.rpc, tg) == LAT_OK;
      for (int k = 0; ok && k < P->ngroups; ++k) ok = geometry_set_w(P, n_f, cs, row_slots, nyq, k, t.w[k], tg) == LAT_OK;
      if (ok) g = tg;
    }
  }
  return LAT_OK;
}

Work layout(const lat_plan* P, int n_items, int precision, int phases_per_table, int n_tables, int scheme,
            bool field) {
  const int n_c = P->d * (P->d + 1) / 2;
  const size_t cs = (precision == LAT_MIXED) ? 8 : 16;
  Work w;
  // half spectrum + Nyquist plane (power-of-two plans), or the full complex spectrum (general plans)
  w.t_per_lc = P->general ? (size_t)n_c * P->m * cs : (size_t)n_c * (P->m / 2) * cs;
  // general plans: no Nyquist plane; a chirp-z row takes the convolution lines there (blue_L per row)
  w.tn_per_lc = P->general ? (P->blue ? (size_t)n_c * P->nrows * P->blue_L * 16 : 0) : (size_t)n_c * P->nrows * cs;
  // two values per row block (conjugate gradients), n_c per block of the effective stress
  w.pstride = std::max<int64_t>(2 * P->nrows, (int64_t)kEffBlocksMax * 6);
  if (P->blue) w.pstride = std::max<int64_t>(w.pstride, 2 * 1024);   // chirp-z: up to 1024 point blocks
  w.table_bytes = (size_t)phases_per_table * n_c * n_c * sizeof(double);
  size_t off = 0;
  w.T = off;
  off = align256(off + n_items * w.t_per_lc);
  w.TN = off;
  off = align256(off + n_items * w.tn_per_lc);
  w.items = off;
  off = align256(off + (size_t)n_items * sizeof(ItemDev));
  w.tables = off;
  off = align256(off + (size_t)n_tables * 2 * w.table_bytes);
  w.tables_f = off;
  off = align256(off + (size_t)n_tables * w.table_bytes / 2);
  w.tables_df = off;   // (C - C0) as double-float pairs: 8 bytes per entry like binary64
  off = align256(off + (precision != LAT_FP64 ? (size_t)n_tables * w.table_bytes : 0));  // mixed: its restart
  // (C + C0)^{-1} of the Eyre-Milton iteration: binary64, binary32, pairs
  w.tables_w = off;
  off = align256(off + (size_t)n_tables * w.table_bytes);
  w.tables_wf = off;
  off = align256(off + (size_t)n_tables * w.table_bytes / 2);
  w.tables_wdf = off;
  off = align256(off + (size_t)n_tables * w.table_bytes);
  w.partials = off;
  off = align256(off + (size_t)n_items * w.pstride * sizeof(double));
  w.scal = off;
  off = align256(off + (size_t)n_items * kScalBytes + kScalBytes);
  w.hist = off;
  off = align256(off + (size_t)n_items * LAT_HIST_CAP * sizeof(double));
  w.T64 = w.TN64 = off;
  if (precision == LAT_MIXED) {   // the restart's pair spectrum: as T (and TN) with 16-byte values
    w.T64 = off;
    off = align256(off + (size_t)n_items * n_c * (P->general ? P->m : P->m / 2) * 16);
    w.TN64 = off;
    off = align256(off + (P->general ? 0 : (size_t)n_items * n_c * P->nrows * 16));
  }
  w.cgv = off;
  w.cg_stride = (int64_t)n_c * P->m;
  if (scheme == LAT_SCHEME_CG) off = align256(off + (size_t)n_items * 4 * w.cg_stride * sizeof(double));
  // the stiffness field in the kernels' types: binary32 (mixed) and pairs (df64, and the mixed restart)
  w.fld_f = off;
  if (field && precision == LAT_MIXED) off = align256(off + (size_t)21 * P->m * sizeof(float));
  w.fld_df = off;
  if (field && precision != LAT_FP64) off = align256(off + (size_t)21 * P->m * sizeof(dfloat));
  w.total = off;
  return w;
}

// inverse of an n x n matrix (n <= 6) by Gauss-Jordan with partial pivoting; false if singular
bool invert_small(const double* A, int n, double* out) {
  double M[6][12];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  double scale = 0;
  for (int i = 0; i < n * n; ++i) scale = std::max(scale, fabs(A[i]));
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (!(fabs(M[piv][c]) > 1e-14 * scale)) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(M[c][j], M[piv][j]);
    const double inv = 1.0 / M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] *= inv;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double f = M[r][c];
        for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = M[i][n + j];
  return true;
}

// tensor-component form of a 6x6 Voigt matrix: out[I][J] = V[vi][vj] * (J shear ? 2 : 1)
void voigt_to_tc(const double* V, int d, double* out) {
  static const int idx3[6] = {0, 1, 2, 3, 4, 5};
  static const int idx2[3] = {0, 1, 5};
  const int n_c = d * (d + 1) / 2;
  const int* vi = d == 3 ? idx3 : idx2;
  for (int I = 0; I < n_c; ++I)
    for (int J = 0; J < n_c; ++J) out[I * n_c + J] = V[vi[I] * 6 + vi[J]] * (J >= d ? 2.0 : 1.0);
}

// true when the tensor-component matrix T (n_c x n_c) couples no normal and shear components and has a
// diagonal shear block (exact zeros): the polarization needs the normal block and the shear diagonal only
bool tc_ortho(const double* T, int n_c, int d) {
  for (int I = 0; I < n_c; ++I)
    for (int J = 0; J < n_c; ++J)
      if (I != J && (I >= d || J >= d) && T[I * n_c + J] != 0.0) return false;
  return true;
}

#define CK(x)                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename Real>
void enqueue_col_group(const LatDev& dv, const lat_plan* P, const Geometry& g, ColArgs c, int k, int mode,
                       int n_items, cudaStream_t st) {
  const LatGroup& G = P->grp[k];
  c.mode = mode;
  c.gidx = k;
  c.a0 = G.a0;
  c.a1 = G.a1;
  c.G = G.G;
  c.outer = G.outer;
  c.inner = G.inner;
  c.has_twiddle = G.has_twiddle;
  c.w = g.w[k];
  c.wN = g.wN[k];
  c.tiles_main = g.tiles_main[k];
  c.tiles_nyq = g.tiles_nyq[k];
  if (dv.general) launch_gen_col<Real>(dv, c, n_items, kThreads, g.col_smem[k], st);
  else launch_col_pass<Real>(dv, c, n_items, kThreads, g.col_smem[k], st);
}

// the length-L transforms of a chirp-z row on nl lines of Y (L apart), in place: forward (unnormalized,
// the sub-plan's spectral order) or its inverse (unnormalized), the passes of lattice_fft on the
// power-of-two plan S = diag(1, L) with one line per item
static void blue_sub_fft(const lat_plan* S, const LatDev& sdv, const Geometry& geo, double2* Y, int nl, int inverse,
                         cudaStream_t st) {
  ColArgs base;
  memset(&base, 0, sizeof(base));
  base.row_slots = S->Rlen;
  base.n_f = 1;
  base.T = Y;
  base.t_stride = S->m;
  base.scale = 1.0;
  auto col = [&](int k, int mode) {
    ColArgs c = base;
    const LatGroup& G = S->grp[k];
    c.mode = mode;
    c.gidx = k;
    c.a0 = G.a0;
    c.a1 = G.a1;
    c.G = G.G;
    c.outer = G.outer;
    c.inner = G.inner;
    c.has_twiddle = G.has_twiddle;
    c.w = geo.w[k];
    c.wN = geo.wN[k];
    c.tiles_main = geo.tiles_main[k];
    launch_col_pass<double>(sdv, c, nl, kThreads, geo.col_smem[k], st);
  };
  if (!inverse) {
    launch_row_complex<double>(sdv, Y, Y, 1, 0, 1.0, geo.rpc, kThreads, geo.row_smem, st, nl);
    for (int k = S->ngroups - 1; k >= 0; --k) col(k, COL_FWD);
  } else {
    for (int k = 0; k < S->ngroups; ++k) col(k, COL_INV);
    launch_row_complex<double>(sdv, Y, Y, 1, 1, 1.0, geo.rpc, kThreads, geo.row_smem, st, nl);
  }
}

// Bluestein's chirp-z form of the DFT along a row of length p (Sec. 2.2's DFT over the largest divisor):
// X_k = w_k sum_n (x_n w_n) conj(w_{k-n}), w_n = exp(-i pi n^2 / p), the sum a cyclic convolution of
// length L >= 2p - 1 taken by the sub-plan's transforms; the inverse is conj(DFT(conj x)).  Lines j <
// lines_per_item of item i start at src + i src_stride + j p (complex binary64) and go to dst likewise;
// Y holds y_lines lines of L; scale multiplies the result.
void blue_rows(const LatDev& dv, const double2* src, int64_t src_stride, double2* dst, int64_t dst_stride,
               int lines_per_item, int n_items, double2* Y, int64_t y_lines, int inverse, double scale,
               cudaStream_t st) {
  const lat_plan* P = (const lat_plan*)dv.blue_plan;
  const lat_plan* S = P->blue_sub;
  const int64_t p = dv.Rlen, L = dv.blue_L;
  const int64_t total = (int64_t)lines_per_item * n_items;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(total, 65535), y_lines));
  const LatDev sdv = make_dev(S, LAT_FP64);
  Geometry geo;
  memset(&geo, 0, sizeof(geo));
  geometry(S, 1, 16, S->Rlen, false, geo, (int)chunk);   // a power-of-two plan of one field always fits
  for (int64_t l0 = 0; l0 < total; l0 += chunk) {
    const int nl = (int)std::min<int64_t>(chunk, total - l0);
    launch_blue_pre(src, src_stride, lines_per_item, p, L, dv.blue_lgA, dv.blue_lgB, dv.blue_chirp, Y, inverse, l0,
                    nl, st);
    blue_sub_fft(S, sdv, geo, Y, nl, 0, st);
    launch_blue_mul(Y, dv.blue_bh, L, nl, 1.0 / (double)L, st);
    blue_sub_fft(S, sdv, geo, Y, nl, 1, st);
    launch_blue_post(Y, dst, dst_stride, lines_per_item, p, L, dv.blue_lgA, dv.blue_lgB, dv.blue_chirp, inverse, scale,
                     l0, nl, st);
  }
}

// the row pass of a chirp-z plan: inverse row transforms of the spectrum (except on a pass that starts
// from the strain), the pointwise step, forward row transforms, and the Green operator when the row is
// the only logical axis.  The convolution lines live in the Nyquist slot of the workspace (RowArgs::TN).
static void blue_row_pass(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, cudaStream_t st) {
  const int lines = (int)(dv.n_c * dv.nrows);
  double2* T = (double2*)a.T;
  double2* Y = (double2*)a.TN;
  const int64_t y_lines = (int64_t)lines * n_items;
  if (!(a.flags & ROW_LOAD_EPS)) blue_rows(dv, T, a.t_stride, T, a.t_stride, lines, n_items, Y, y_lines, 1, 1.0, st);
  launch_blue_point(dv, a, nblocks, n_items, st);
  blue_rows(dv, T, a.t_stride, T, a.t_stride, lines, n_items, Y, y_lines, 0, 1.0, st);
  if (a.flags & ROW_GAMMA) launch_blue_green(dv, a, n_items, st);
}

// a conjugate-gradient stage on a chirp-z plan: inverse row transforms of the spectrum (stages that start
// from it), the stage's pointwise part, and for every stage but A the forward row transforms and the Green
// operator when the row is the only logical axis (the order of gen_cg_row_kernel)
static void blue_cg_row_pass(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items,
                             cudaStream_t st) {
  const int lines = (int)(dv.n_c * dv.nrows);
  double2* T = (double2*)a.T;
  double2* Y = (double2*)a.TN;
  const int64_t y_lines = (int64_t)lines * n_items;
  if (cg.stage == CG_FULL0 || cg.stage == CG_A)
    blue_rows(dv, T, a.t_stride, T, a.t_stride, lines, n_items, Y, y_lines, 1, 1.0, st);
  launch_blue_cg_point(dv, a, cg, nblocks, n_items, st);
  if (cg.stage == CG_A) return;
  blue_rows(dv, T, a.t_stride, T, a.t_stride, lines, n_items, Y, y_lines, 0, 1.0, st);
  if (a.flags & ROW_GAMMA) launch_blue_green(dv, a, n_items, st);
}

// a conjugate-gradient stage of a plan's rows: the chirp-z stages (binary64 only: other precisions are
// refused on entry for these plans) or the row kernels
template <typename Real>
void cg_row(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items, size_t smem,
            cudaStream_t st) {
  if (dv.blue) {
    if constexpr (std::is_same<Real, double>::value) blue_cg_row_pass(dv, a, cg, nblocks, n_items, st);
    return;
  }
  launch_cg_row<Real>(dv, a, cg, nblocks, n_items, kThreads, smem, st);
}

int lat_blue_transform_bh_impl(lat_plan* P) {
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  const lat_plan* S = P->blue_sub;
  const LatDev sdv = make_dev(S, LAT_FP64);
  Geometry geo;
  memset(&geo, 0, sizeof(geo));
  if (int rc = geometry(S, 1, 16, S->Rlen, false, geo, 1)) return rc;
  blue_sub_fft(S, sdv, geo, P->d_bh, 1, 0, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(0));
  return LAT_OK;
}

// the row pass of a plan: power-of-two kernels or the mixed-radix kernels of a general plan
template <typename Real>
void launch_row(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, size_t smem, cudaStream_t st) {
  if (dv.blue) {   // binary64 only: other precisions are refused on entry for these plans
    if constexpr (std::is_same<Real, double>::value) blue_row_pass(dv, a, nblocks, n_items, st);
    return;
  }
  if (dv.general) launch_gen_row<Real>(dv, a, nblocks, n_items, kThreads, smem, st);
  else launch_row_pass<Real>(dv, a, nblocks, n_items, kThreads, smem, st);
}

template <typename Real>
void enqueue_columns(const LatDev& dv, const lat_plan* P, const Geometry& g, ColArgs base, int n_items,
                     cudaStream_t st) {
  // forward over mid groups (innermost first), Gamma group, inverse mid groups
  for (int k = P->ngroups - 1; k >= 0; --k) enqueue_col_group<Real>(dv, P, g, base, k, k == 0 ? COL_GAMMA : COL_FWD, n_items, st);
  for (int k = 1; k < P->ngroups; ++k) enqueue_col_group<Real>(dv, P, g, base, k, COL_INV, n_items, st);
}
template void enqueue_columns<double>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, cudaStream_t);
template void enqueue_columns<float>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, cudaStream_t);
template void enqueue_columns<dfloat>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, cudaStream_t);
template void enqueue_col_group<double>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, int, int, cudaStream_t);
template void enqueue_col_group<float>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, int, int, cudaStream_t);
template void enqueue_col_group<dfloat>(const LatDev&, const lat_plan*, const Geometry&, ColArgs, int, int, int, cudaStream_t);

namespace {

// one iteration of a group: row pass (update, residual, convergence) + column passes; conjugate
// gradients: update stage, column passes, the stage that forms w = A r and the step lengths
template <typename Real>
void enqueue_body(const GroupRun& g, const RowArgs& full, cudaStream_t st) {
  if (g.cg) {
    CgArgs cb = g.cga;
    cb.stage = CG_B;
    cg_row<Real>(g.dv, full, cb, g.geo.row_blocks, g.n_items, g.geo.row_smem, st);
    enqueue_columns<Real>(g.dv, g.P, g.geo, g.cl, g.n_items, st);
    cb.stage = CG_A;
    cg_row<Real>(g.dv, full, cb, g.geo.row_blocks, g.n_items, g.geo.row_smem, st);
    return;
  }
  launch_row<Real>(g.dv, full, g.geo.row_blocks, g.n_items, g.geo.row_smem, st);
  enqueue_columns<Real>(g.dv, g.P, g.geo, g.cl, g.n_items, st);
}

// adds a WHILE node to `top` after `dep` (or as a root): body = one iteration (enqueue_body); the
// last block of the convergence test sets the node's condition
template <typename Real>
int add_loop_node(const GroupRun& g, const RowArgs& body_row, cudaGraph_t top, const cudaGraphNode_t* dep,
                  cudaGraphConditionalHandle handle, cudaGraphNode_t* node_out) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  CK(cudaGraphAddNode(node_out, top, dep, nullptr, dep ? 1 : 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (ce == cudaSuccess) {
    RowArgs full = body_row;
    full.it.cond = (unsigned long long)handle;
    enqueue_body<Real>(g, full, cap);
    cudaGraph_t captured = nullptr;
    ce = cudaStreamEndCapture(cap, &captured);
  }
  cudaStreamDestroy(cap);
  if (ce != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  return LAT_OK;
}

// one iteration of one group with plain launches (no graph condition)
template <typename Real>
int plain_iteration(const GroupRun& g, const RowArgs& body_row, cudaStream_t st) {
  RowArgs full = body_row;
  full.it.cond = 0;
  enqueue_body<Real>(g, full, st);
  CK(cudaGetLastError());
  return LAT_OK;
}

// the binary64-accurate restart of the paused items (mixed precision only, double-float kernels);
// cond2 != 0 sets the condition of
// the loop that follows from the number of resumed items
int enqueue_restart(const GroupRun& g, unsigned long long cond2, cudaStream_t st) {
  const Work& wl = g.wl;
  ItemScal* scal = (ItemScal*)(g.ws + wl.scal);
  launch_prep_restart(scal, g.full.it.glob, g.n_items, st);
  launch_row<dfloat>(g.dv64, g.r_pro, g.geo64.row_blocks, g.n_items, g.geo64.row_smem, st);
  enqueue_columns<dfloat>(g.dv64, g.P, g.geo64, g.c64, g.n_items, st);
  launch_row<dfloat>(g.dv64, g.r_upd, g.geo64.row_blocks, g.n_items, g.geo64.row_smem, st);
  // general plans: the full complex spectrum, no Nyquist plane
  const int64_t te = (int64_t)g.n_c * (g.P->general ? g.P->m : g.P->m / 2);
  const int64_t tne = g.P->general ? 0 : (int64_t)g.n_c * g.P->nrows;
  launch_spectrum_to_f32(g.ws + wl.T64, g.ws + wl.TN64, g.ws + wl.T, g.ws + wl.TN, te, tne, g.full.t_stride,
                         g.full.tn_stride, scal, g.n_items, st);
  if (g.P->nax > 1) enqueue_columns<float>(g.dv, g.P, g.geo, g.cl, g.n_items, st);
  if (cond2) launch_set_cond(g.full.it.glob, cond2, st);
  CK(cudaGetLastError());
  return LAT_OK;
}

// the loops of one group in `top`: WHILE (with pause) [-> restart chain -> WHILE]
int add_group_loops(const GroupRun& g, cudaGraph_t top) {
  cudaGraphConditionalHandle h1;
  cudaGraphNode_t n1;
  int rc = LAT_OK;
  if (g.cg) {
    // the conjugate-gradient prologue may already have stopped every item (a homogeneous medium, or
    // maxit = 1): the loop's condition starts from the active count, set by a node before the loop
    CK(cudaGraphConditionalHandleCreate(&h1, top, 0, cudaGraphCondAssignDefault));
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraphNode_t leaf = nullptr;
    cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
      launch_set_cond(g.full.it.glob, (unsigned long long)h1, cap);
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaError_t ie = cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &deps, nullptr, &nd);
      if (ie == cudaSuccess && nd == 1) leaf = deps[0];
      cudaGraph_t captured = nullptr;
      ce = cudaStreamEndCapture(cap, &captured);
      if (ce == cudaSuccess && ie != cudaSuccess) ce = ie;
    }
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("loop condition capture: ") + cudaGetErrorString(ce));
    if (!leaf) return lat_fail(LAT_ERR_CUDA, "loop condition capture: no single leaf node");
    return by_kind(g.kind, [&](auto tag) { return add_loop_node<decltype(tag)>(g, g.full, top, &leaf, h1, &n1); });
  }
  CK(cudaGraphConditionalHandleCreate(&h1, top, 1, cudaGraphCondAssignDefault));
  rc = by_kind(g.kind, [&](auto tag) {
    return add_loop_node<decltype(tag)>(g, g.full, top, nullptr, h1, &n1);
  });
  if (rc != LAT_OK || !g.restart) return rc;
  cudaGraphConditionalHandle h2;
  CK(cudaGraphConditionalHandleCreate(&h2, top, 0, cudaGraphCondAssignDefault));
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraphNode_t leaf = nullptr;
  cudaError_t ce = cudaStreamBeginCaptureToGraph(cap, top, &n1, nullptr, 1, cudaStreamCaptureModeRelaxed);
  if (ce == cudaSuccess) {
    rc = enqueue_restart(g, (unsigned long long)h2, cap);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t ie = cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    if (ie == cudaSuccess && nd == 1) leaf = deps[0];
    cudaGraph_t captured = nullptr;
    ce = cudaStreamEndCapture(cap, &captured);
    if (ce == cudaSuccess && ie != cudaSuccess) ce = ie;
  }
  cudaStreamDestroy(cap);
  if (ce != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("restart capture: ") + cudaGetErrorString(ce));
  if (rc != LAT_OK) return rc;
  if (!leaf) return lat_fail(LAT_ERR_CUDA, "restart capture: no single leaf node");
  cudaGraphNode_t n2;
  return add_loop_node<float>(g, g.full2, top, &leaf, h2, &n2);
}

}  // namespace

int group_prepare(const lat_plan* P, const std::vector<ItemHost>& items, const std::vector<const double*>& stiff,
                  const std::vector<int>& nph, double tol, int maxit, const lat_solve_opts& o, char* ws,
                  const Work& wl, const LatDev& dv, GroupRun& g, cudaStream_t st) {
  const int n_items = (int)items.size();
  const int d = P->d, n_c = d * (d + 1) / 2;
  const int64_t m = P->m;
  const bool fp32 = (o.precision == LAT_MIXED);
  g.kind = o.precision;
  g.P = P;
  g.n_items = n_items;
  g.n_c = n_c;
  g.tol = tol;
  g.maxit = maxit;
  g.fp32 = fp32;
  g.dv = dv;
  g.ws = ws;
  g.wl = wl;
  g.loop = false;
  g.restart = false;
  g.want_hist = o.resid_history != nullptr && maxit > 0;
  g.cg = (o.scheme == LAT_SCHEME_CG);
  // material tables: per table, D = C - C0 (binary64 and binary32) and C, in tensor-component form;
  // the reference medium is the table's (items sharing a table share C0)
  const int n_tables = (int)stiff.size();
  const size_t tstride = wl.table_bytes / sizeof(double);
  std::vector<double> tabs((size_t)n_tables * 2 * tstride, 0.0);
  std::vector<double> tabs_w((size_t)n_tables * tstride, 0.0);
  for (int t = 0; t < n_tables; ++t) {
    int owner = -1;
    for (int i = 0; i < n_items && owner < 0; ++i)
      if (items[i].table == t) owner = i;
    double c0tc[36];
    memset(c0tc, 0, sizeof(c0tc));
    if (owner >= 0) {
      double C0v[36];
      memset(C0v, 0, sizeof(C0v));
      const double lam0 = items[owner].C0[0], mu0 = items[owner].C0[1];
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) C0v[i * 6 + j] = lam0;
        C0v[i * 6 + i] = lam0 + 2 * mu0;
        C0v[(i + 3) * 6 + (i + 3)] = mu0;
      }
      voigt_to_tc(C0v, d, c0tc);
    }
    for (int p = 0; p < nph[t]; ++p) {
      double* Dp = &tabs[(size_t)(2 * t) * tstride + (size_t)p * n_c * n_c];
      double* Cp = &tabs[(size_t)(2 * t + 1) * tstride + (size_t)p * n_c * n_c];
      voigt_to_tc(stiff[t] + 36 * p, d, Cp);
      // conjugate gradients transform C : v, not the polarization (C - C0) : eps
      for (int k = 0; k < n_c * n_c; ++k) Dp[k] = o.scheme == LAT_SCHEME_CG ? Cp[k] : Cp[k] - c0tc[k];
      if (o.scheme == LAT_SCHEME_EYRE_MILTON) {
        double S[36];
        for (int k = 0; k < n_c * n_c; ++k) S[k] = Cp[k] + c0tc[k];
        if (!invert_small(S, n_c, &tabs_w[(size_t)t * tstride + (size_t)p * n_c * n_c]))
          return lat_fail(LAT_ERR_ARG, "Eyre-Milton: C_p + C0 is singular");
      }
    }
  }
  // the isotropic reference medium has the structure, so D = C - C0 has it exactly when C has
  bool ortho = true;
  for (int t = 0; t < n_tables; ++t)
    for (int p = 0; p < nph[t]; ++p)
      ortho = ortho && tc_ortho(&tabs[(size_t)(2 * t + 1) * tstride + (size_t)p * n_c * n_c], n_c, d);
  std::vector<ItemDev> hdev(n_items);
  for (int i = 0; i < n_items; ++i) {
    const ItemHost& it = items[i];
    ItemDev& v = hdev[i];
    memset(&v, 0, sizeof(v));
    v.eps = it.eps;
    v.sigma = it.sigma;
    v.phase = it.phase;
    if (it.field) {
      v.fld = it.field;
      v.fld_f = o.precision == LAT_MIXED ? (const float*)(ws + wl.fld_f) : nullptr;
      v.fld_df = o.precision != LAT_FP64 ? (const dfloat*)(ws + wl.fld_df) : nullptr;
    }
    v.Ctab = (const double*)(ws + wl.tables + (size_t)(2 * it.table + 1) * wl.table_bytes);
    v.Dtab = (const double*)(ws + wl.tables + (size_t)(2 * it.table) * wl.table_bytes);
    v.Dtab_f = (const float*)(ws + wl.tables_f + (size_t)it.table * wl.table_bytes / 2);
    v.Dtab_df = (const dfloat*)(ws + wl.tables_df + (size_t)it.table * wl.table_bytes);
    v.Wtab = (const double*)(ws + wl.tables_w + (size_t)it.table * wl.table_bytes);
    v.Wtab_f = (const float*)(ws + wl.tables_wf + (size_t)it.table * wl.table_bytes / 2);
    v.Wtab_df = (const dfloat*)(ws + wl.tables_wdf + (size_t)it.table * wl.table_bytes);
    const double lam0 = it.C0[0], mu0 = it.C0[1];
    v.lam0 = lam0;
    v.mu0 = mu0;
    v.lam0f = (float)lam0;
    v.mu0f = (float)mu0;
    {  // 2 C0 : E on tensor components
      double C0v[36], c0e[36];
      memset(C0v, 0, sizeof(C0v));
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) C0v[a * 6 + b] = lam0;
        C0v[a * 6 + a] = lam0 + 2 * mu0;
        C0v[(a + 3) * 6 + (a + 3)] = mu0;
      }
      voigt_to_tc(C0v, d, c0e);
      for (int c = 0; c < 6; ++c) {
        double acc = 0;
        for (int q = 0; c < n_c && q < n_c; ++q) acc += c0e[c * n_c + q] * it.E[q];
        v.twoC0E[c] = 2.0 * acc;
      }
    }
    v.c1 = 0.5 / mu0;
    v.c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
    v.c1f = (float)v.c1;
    v.c2f = (float)v.c2;
    v.c1_df = dfloat(v.c1);
    v.c2_df = dfloat(v.c2);
    v.lam0_df = dfloat(lam0);
    v.mu0_df = dfloat(mu0);
    double nE2 = 0;
    for (int c = 0; c < 6; ++c) v.E[c] = c < n_c ? it.E[c] : 0.0;
    for (int c = 0; c < n_c; ++c) nE2 += (c >= d ? 2.0 : 1.0) * it.E[c] * it.E[c];
    v.norm0 = nE2 > 0 ? sqrt((double)m * nE2) : 1.0;
  }
  g.tabs.swap(tabs);
  g.tabs_f.assign((size_t)n_tables * tstride, 0.0f);
  for (int t = 0; t < n_tables; ++t)
    for (size_t k = 0; k < tstride; ++k) g.tabs_f[(size_t)t * tstride + k] = (float)g.tabs[(size_t)(2 * t) * tstride + k];
  if (g.kind != LAT_FP64) {
    g.tabs_df.assign((size_t)n_tables * tstride, make_float2(0.f, 0.f));
    for (int t = 0; t < n_tables; ++t)
      for (size_t k = 0; k < tstride; ++k) {
        const double v = g.tabs[(size_t)(2 * t) * tstride + k];
        const float hi = (float)v;
        g.tabs_df[(size_t)t * tstride + k] = make_float2(hi, (float)(v - (double)hi));
      }
  }
  g.tabs_w.swap(tabs_w);
  g.tabs_wf.assign(g.tabs_w.size(), 0.f);
  g.tabs_wdf.assign(g.tabs_w.size(), make_float2(0.f, 0.f));
  for (size_t k = 0; k < g.tabs_w.size(); ++k) {
    const double v = g.tabs_w[k];
    g.tabs_wf[k] = (float)v;
    g.tabs_wdf[k] = make_float2((float)v, (float)(v - (double)(float)v));
  }
  g.hdev.swap(hdev);
  g.glob0.arrivals = 0;
  g.glob0.active = n_items;
  // host buffers stay alive in g until the caller synchronizes
  CK(cudaMemcpyAsync(ws + wl.tables, g.tabs.data(), g.tabs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ws + wl.tables_f, g.tabs_f.data(), g.tabs_f.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  if (g.kind != LAT_FP64)
    CK(cudaMemcpyAsync(ws + wl.tables_df, g.tabs_df.data(), g.tabs_df.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
  if (o.scheme == LAT_SCHEME_EYRE_MILTON) {
    CK(cudaMemcpyAsync(ws + wl.tables_w, g.tabs_w.data(), g.tabs_w.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws + wl.tables_wf, g.tabs_wf.data(), g.tabs_wf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws + wl.tables_wdf, g.tabs_wdf.data(), g.tabs_wdf.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(ws + wl.items, g.hdev.data(), g.hdev.size() * sizeof(ItemDev), cudaMemcpyHostToDevice, st));
  // device scalars start from zero; the batch starts with every item active
  CK(cudaMemsetAsync(ws + wl.scal, 0, (size_t)n_items * kScalBytes + kScalBytes, st));
  GlobScal* glob = (GlobScal*)(ws + wl.scal + (size_t)n_items * kScalBytes);
  CK(cudaMemcpyAsync(glob, &g.glob0, sizeof(GlobScal), cudaMemcpyHostToDevice, st));
  const ItemDev* ditems = (const ItemDev*)(ws + wl.items);
  const bool field = n_items > 0 && items[0].field != nullptr;   // a field solve: all items share the field
  const int matflag = field ? ROW_FIELD : (ortho ? ROW_ORTHO : 0);   // the material's form
  if (field && o.precision != LAT_FP64)
    launch_field_copies(items[0].field, o.precision == LAT_MIXED ? (float*)(ws + wl.fld_f) : nullptr,
                        (dfloat*)(ws + wl.fld_df), (int64_t)21 * m, st);
  if (!o.warm_start) launch_fill(ditems, n_items, n_c, m, st);
  // mixed precision: the strain is held as double-float pairs in its own buffer during the solve
  if (g.kind != LAT_FP64) launch_eps_df(ditems, n_items, n_c, m, 1, st);
  CK(cudaGetLastError());
  if (P->nax > 0 && maxit > 0) {
    Geometry& geo = g.geo;
    memset(&geo, 0, sizeof(geo));
    int rc = geometry(P, n_c, fp32 ? 8 : 16, P->Rh, true, geo, n_items, g.kind);
    if (rc != LAT_OK) return rc;
    RowArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.rpc = geo.rpc;
    ra.items = ditems;
    ra.T = ws + wl.T;
    ra.TN = ws + wl.TN;
    ra.t_stride = (int64_t)(wl.t_per_lc / (fp32 ? 8 : 16));
    ra.tn_stride = (int64_t)(wl.tn_per_lc / (fp32 ? 8 : 16));
    mat_set_gscale(ra.mat, -1.0 / (double)m);
    ra.mat.boundary_zero = o.boundary == LAT_BOUNDARY_ZERO;
    ra.mat.scheme = o.scheme == LAT_SCHEME_EYRE_MILTON ? LAT_SCHEME_EYRE_MILTON : LAT_SCHEME_BASIC;
    ra.it.partials = (double*)(ws + wl.partials);
    ra.it.pstride = wl.pstride;
    ra.it.scal = (ItemScal*)(ws + wl.scal);
    ra.it.glob = glob;
    ra.it.hist = (double*)(ws + wl.hist);
    ra.it.tol = tol;
    ra.it.maxit = maxit;
    ra.it.n_items = n_items;
    ColArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.row_slots = P->general ? P->Rlen : P->Rh;
    ca.has_nyq = P->general ? 0 : 1;
    ca.n_f = n_c;
    ca.T = ra.T;
    ca.TN = ra.TN;
    ca.t_stride = ra.t_stride;
    ca.tn_stride = ra.tn_stride;
    ca.scale = 1.0;
    ca.items = ditems;
    ca.mat = ra.mat;
    const bool gamma_in_row = (P->nax == 1);
    if (g.cg) {
      // conjugate gradients (binary64 or double-float pairs): every transform maps v to
      // -Gamma0 : (C : v) with k = 0 -> 0.  Prologue: r = -A x (x = E), then w = A r and the first
      // step lengths; p and q start at 0 (the first update multiplies them by beta = 0)
      ra.flags = gamma_in_row ? ROW_GAMMA : 0;
      ra.mat.increment = 1;
      ca.mat = ra.mat;
      g.full = ra;
      g.cl = ca;
      g.cl.scal = ra.it.scal;
      CgArgs cg;
      memset(&cg, 0, sizeof(cg));
      cg.vstride = wl.cg_stride;
      cg.r = (double*)(ws + wl.cgv);
      cg.p = cg.r + (size_t)n_items * wl.cg_stride;
      cg.q = cg.p + (size_t)n_items * wl.cg_stride;
      cg.w = cg.q + (size_t)n_items * wl.cg_stride;
      g.cga = cg;
      CK(cudaMemsetAsync(cg.p, 0, (size_t)2 * n_items * wl.cg_stride * sizeof(double), st));
      ColArgs c0 = ca;
      c0.scal = nullptr;
      by_kind(g.kind, [&](auto tag) {
        typedef decltype(tag) Real;
        CgArgs cs = cg;
        cs.stage = CG_FWD_X;
        cg_row<Real>(dv, ra, cs, geo.row_blocks, n_items, geo.row_smem, st);
        enqueue_columns<Real>(dv, P, geo, c0, n_items, st);
        cs.stage = CG_FULL0;
        cg_row<Real>(dv, ra, cs, geo.row_blocks, n_items, geo.row_smem, st);
        enqueue_columns<Real>(dv, P, geo, g.cl, n_items, st);
        cs.stage = CG_A;
        cg_row<Real>(dv, ra, cs, geo.row_blocks, n_items, geo.row_smem, st);
        return 0;
      });
      CK(cudaGetLastError());
      g.loop = true;
    } else {
      const bool incr = fp32 && o.mixed_increment;
      // prologue: tau^(0) from eps^(0), forward transform, Gamma (k = 0 -> E), inverse columns.  In the
      // increment form from a cold start (eps^(0) = E everywhere) k = 0 maps to 0 instead, so that T
      // holds the first increment G(E) - E and the binary32 rounding is relative to it, not to E
      // (the Eyre-Milton cold start u = (C + C0) E varies in space, so its first step is taken in full)
      const bool incr_first = incr && !o.warm_start && o.scheme == LAT_SCHEME_BASIC;
      RowArgs first = ra;
      first.flags = ROW_LOAD_EPS | (gamma_in_row ? ROW_GAMMA : 0) | matflag;
      first.mat.increment = incr_first ? 1 : 0;
      ColArgs c0 = ca;
      c0.scal = nullptr;
      c0.mat.increment = incr_first ? 1 : 0;
      g.full = ra;
      g.full.flags = ROW_UPDATE | (gamma_in_row ? ROW_GAMMA : 0) | (incr ? ROW_INCREMENT : 0) | matflag |
                     (incr_first ? ROW_INCR_FIRST : 0);
      g.full.mat.increment = incr ? 1 : 0;
      g.cl = ca;
      g.cl.scal = ra.it.scal;
      g.cl.mat.increment = incr ? 1 : 0;   // the loop's spectra carry increments: k = 0 gets 0
      by_kind(g.kind, [&](auto tag) {
        launch_row<decltype(tag)>(dv, first, geo.row_blocks, n_items, geo.row_smem, st);
        enqueue_columns<decltype(tag)>(dv, P, geo, c0, n_items, st);
        return 0;
      });
      CK(cudaGetLastError());
      g.loop = true;
      // one binary64-accurate restart (double-float kernels) when an item's residual first falls below
      // sqrt(tol): the increment recurrence accumulates binary32 rounding as a standing offset of the
      // fixed point (it never re-evaluates G(eps)); the restart recomputes the increment exactly, and
      // the iterations after it contract the offset
      const double pause = sqrt(tol);
      g.restart = incr && o.mixed_restart >= 0 && tol > 0 && pause > tol && maxit > 1;
      if (g.restart) {
        g.full.it.pause_tol = pause;
        g.dv64 = make_dev(P, LAT_DF64);   // the restart runs on double-float pairs
        memset(&g.geo64, 0, sizeof(g.geo64));
        if ((rc = geometry(P, n_c, 16, P->Rh, true, g.geo64, n_items, LAT_DF64)) != LAT_OK) return rc;
        RowArgs r64 = ra;
        r64.rpc = g.geo64.rpc;
        r64.T = ws + wl.T64;
        r64.TN = ws + wl.TN64;
        r64.it.pause_tol = 0.0;
        g.r_pro = r64;
        g.r_pro.flags = ROW_LOAD_EPS | ROW_ONLY_PAUSED | ROW_EPS_DF | (gamma_in_row ? ROW_GAMMA : 0) | matflag;
        g.r_pro.mat.increment = 0;
        g.r_upd = r64;
        g.r_upd.flags =
            ROW_UPDATE | ROW_TAU_DELTA | ROW_ONLY_PAUSED | ROW_EPS_DF | (gamma_in_row ? ROW_GAMMA : 0) | matflag;
        g.r_upd.mat.increment = 1;
        g.c64 = ca;
        g.c64.T = r64.T;
        g.c64.TN = r64.TN;
        g.c64.scal = ra.it.scal;
        g.c64.only_paused = 1;
        g.c64.mat.increment = 0;
        g.full2 = g.full;
        g.full2.it.pause_tol = 0.0;
      }
    }
  }
  g.ea.items = ditems;
  g.ea.partials = (double*)(ws + wl.partials);
  g.ea.pstride = wl.pstride;
  g.ea.scal = (ItemScal*)(ws + wl.scal);
  g.eff_blocks = (int)std::min<int64_t>(kEffBlocksMax, std::max<int64_t>(1, (m + 255) / 256));
  return LAT_OK;
}

int group_plain_iteration(const GroupRun& g, const RowArgs& body_row, cudaStream_t st) {
  if (!g.loop) return LAT_OK;
  return by_kind(g.kind, [&](auto tag) { return plain_iteration<decltype(tag)>(g, body_row, st); });
}

const int* group_active_flag(const GroupRun& g) { return &g.full.it.glob->active; }

int group_finish(GroupRun& g, cudaStream_t st, const AsyncOut* aout) {
  if (g.kind != LAT_FP64) launch_eps_df(g.ea.items, g.n_items, g.n_c, g.P->m, 0, st);
  launch_eff(g.dv, g.ea, g.eff_blocks, g.n_items, st);
  CK(cudaGetLastError());
  if (aout) {   // scalars to device memory, no host copy
    launch_scalars_out((const ItemScal*)(g.ws + g.wl.scal), g.n_items, g.n_c, g.tol, g.maxit, g.P->nax == 0,
                       aout->sigma_bar, aout->iters, aout->resid, aout->status, st);
    CK(cudaGetLastError());
    return LAT_OK;
  }
  g.scal.resize((size_t)g.n_items * kScalBytes);
  CK(cudaMemcpyAsync(g.scal.data(), g.ws + g.wl.scal, g.scal.size(), cudaMemcpyDeviceToHost, st));
  if (g.want_hist) {
    g.hist.resize((size_t)g.n_items * LAT_HIST_CAP);
    CK(cudaMemcpyAsync(g.hist.data(), g.ws + g.wl.hist, g.hist.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  return LAT_OK;
}

int group_decode(const GroupRun& g, const lat_solve_opts& o, double* sigma_bar, int* iters, double* resid) {
  const lat_plan* P = g.P;
  const int n_c = g.n_c, maxit = g.maxit;
  const double tol = g.tol;
  int status = LAT_OK;
  for (int i = 0; i < g.n_items; ++i) {
    const ItemScal* sc = (const ItemScal*)(g.scal.data() + (size_t)i * kScalBytes);
    int it = sc->iter;
    double r = sc->last_r;
    if (P->nax == 0) {  // m = 1: every iterate equals E, r_n = 0; stop at the first r_n < tol
      it = (maxit > 0 && tol > 0) ? 1 : maxit;
      r = maxit > 0 ? 0.0 : NAN;
    } else if (maxit == 0) {
      r = NAN;
    }
    if (iters) iters[i] = it;
    if (resid) resid[i] = r;
    if (sigma_bar)
      for (int c = 0; c < n_c; ++c) sigma_bar[i * n_c + c] = sc->sigma_bar[c];
    if (g.want_hist) {
      if (P->nax == 0)
        for (int k = 0; k < it; ++k) o.resid_history[(size_t)i * maxit + k] = 0.0;
      for (int k = 0; k < std::min(it, std::min(maxit, LAT_HIST_CAP)) && P->nax > 0; ++k)
        o.resid_history[(size_t)i * maxit + k] = g.hist[(size_t)i * LAT_HIST_CAP + k];
    }
    int s = LAT_OK;
    if ((!isfinite(r) || sc->diverged) && maxit > 0) s = LAT_DIVERGED;
    else if (!(r < tol)) s = LAT_NOT_CONVERGED;
    status = std::max(status, s);
  }
  return status;
}

namespace {

// plain launches: every group still active takes one iteration of its current loop, then the host
// reads the active counts; phase 0 = first loop, 1 = second loop after the restart
int plain_loops(std::vector<GroupRun>& groups, int phase, cudaStream_t st) {
  int maxit = 0;
  for (const GroupRun& g : groups) maxit = std::max(maxit, g.loop ? g.maxit : 0);
  std::vector<char> live(groups.size());
  for (size_t k = 0; k < groups.size(); ++k) live[k] = groups[k].loop && (phase == 0 || groups[k].restart);
  std::vector<int> active(groups.size(), 0);
  for (int n = 0; n < maxit; ++n) {
    bool any = false;
    for (size_t k = 0; k < groups.size(); ++k) {
      if (!live[k]) continue;
      int rc = group_plain_iteration(groups[k], phase == 0 ? groups[k].full : groups[k].full2, st);
      if (rc != LAT_OK) return rc;
      CK(cudaMemcpyAsync(&active[k], group_active_flag(groups[k]), sizeof(int), cudaMemcpyDeviceToHost, st));
      any = true;
    }
    if (!any) break;
    CK(cudaStreamSynchronize(st));
    for (size_t k = 0; k < groups.size(); ++k)
      if (live[k] && active[k] == 0) live[k] = 0;
  }
  return LAT_OK;
}

}  // namespace

int run_groups(std::vector<GroupRun>& groups, bool use_graph, cudaStream_t st, const AsyncOut* aout) {
  bool any_loop = false;
  for (const GroupRun& g : groups) any_loop |= g.loop;
  if (any_loop && use_graph) {
    // one graph: per group a WHILE node (plus its restart chain and second WHILE node); the groups
    // are parallel branches and iterate concurrently
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    for (const GroupRun& g : groups) {
      if (!g.loop) continue;
      int rc = add_group_loops(g, top);
      if (rc != LAT_OK) {
        cudaGraphDestroy(top);
        return rc;
      }
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ce = cudaGraphInstantiate(&exec, top, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, st);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(top);
    if (ce != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
  } else if (any_loop) {
    int rc = plain_loops(groups, 0, st);
    if (rc != LAT_OK) return rc;
    bool any_restart = false;
    for (const GroupRun& g : groups)
      if (g.loop && g.restart) {
        if ((rc = enqueue_restart(g, 0, st)) != LAT_OK) return rc;
        any_restart = true;
      }
    if (any_restart && (rc = plain_loops(groups, 1, st)) != LAT_OK) return rc;
  }
  for (GroupRun& g : groups) {
    int rc = group_finish(g, st, aout);
    if (rc != LAT_OK) return rc;
  }
  if (!aout) CK(cudaStreamSynchronize(st));
  return LAT_OK;
}

int run_batch(const lat_plan* P, const std::vector<ItemHost>& items, const std::vector<const double*>& stiff,
              const std::vector<int>& nph, double tol, int maxit, const lat_solve_opts& o, char* ws, const Work& wl,
              const LatDev& dv, bool use_graph, double* sigma_bar, int* iters, double* resid, cudaStream_t st) {
  std::vector<GroupRun> groups(1);
  int rc = group_prepare(P, items, stiff, nph, tol, maxit, o, ws, wl, dv, groups[0], st);
  if (rc != LAT_OK) return rc;
  if ((rc = run_groups(groups, use_graph, st)) != LAT_OK) return rc;
  return group_decode(groups[0], o, sigma_bar, iters, resid);
}

int check_common(const lat_plan* P, double tol, int maxit, const lat_solve_opts& o) {
  if (maxit < 0 || !(tol >= 0)) return lat_fail(LAT_ERR_ARG, "bad maxit/tol");
  if (o.precision != LAT_FP64 && o.precision != LAT_MIXED && o.precision != LAT_DF64)
    return lat_fail(LAT_ERR_ARG, "bad precision");
  if (o.boundary != LAT_BOUNDARY_AVERAGE && o.boundary != LAT_BOUNDARY_ZERO) return lat_fail(LAT_ERR_ARG, "bad boundary");
  if (o.scheme != LAT_SCHEME_BASIC && o.scheme != LAT_SCHEME_EYRE_MILTON && o.scheme != LAT_SCHEME_CG)
    return lat_fail(LAT_ERR_ARG, "bad scheme");
  if (P && P->blue && o.precision != LAT_FP64)
    return lat_fail(LAT_ERR_UNSUPPORTED, "lattices whose largest divisor takes the chirp-z transform run in LAT_FP64");
  if (o.scheme == LAT_SCHEME_EYRE_MILTON && o.boundary == LAT_BOUNDARY_ZERO)
    return lat_fail(LAT_ERR_ARG, "the Eyre-Milton scheme takes the averaged boundary treatment");
  if (o.scheme == LAT_SCHEME_CG) {
    if (o.precision == LAT_MIXED)
      return lat_fail(LAT_ERR_ARG, "the conjugate-gradient scheme runs in LAT_FP64 or LAT_DF64");
    if (o.warm_start) return lat_fail(LAT_ERR_ARG, "the conjugate-gradient scheme starts from eps = E");
    // an even largest divisor means boundary frequencies, where the averaged Green operator is not a
    // projector and the iteration operator is not self-adjoint
    if (o.boundary == LAT_BOUNDARY_AVERAGE && P && P->ed % 2 == 0)
      return lat_fail(LAT_ERR_ARG, "the conjugate-gradient scheme needs LAT_BOUNDARY_ZERO on lattices with an "
                                   "even largest divisor (boundary frequencies)");
  }
  return check_geometry(P, o.precision);
}

// the shared-memory limits bind at the smallest launch shape (one row per block, one column per
// tile), which does not depend on the number of items
int check_geometry(const lat_plan* P, int precision) {
  if (P->nax == 0) return LAT_OK;
  Geometry geo;
  memset(&geo, 0, sizeof(geo));
  // the mixed path also runs binary64 passes (its restart)
  return geometry(P, P->d * (P->d + 1) / 2, 16, P->Rh, true, geo, 1);
}

// the power-of-two kernels move the strain of two neighbouring points at once (16 bytes); the mixed-radix
// kernels of general plans one point (8 bytes), so odd m and per-load-case offsets of n_c m points are fine
size_t eps_align_mask(const lat_plan* P) { return P->general ? 7 : 15; }

int check_c0(const double* C0) {
  if (!(C0[1] > 0) || !(C0[0] + 2 * C0[1] > 0)) return lat_fail(LAT_ERR_ARG, "C0 must have mu0 > 0 and lam0 + 2 mu0 > 0");
  return LAT_OK;
}

// items of basic_scheme_solve: n_loads load cases of one microstructure
void load_case_items(const lat_plan* P, const uint8_t* phase, const double* C0, const double* E, int n_loads,
                     double* eps, double* sigma, std::vector<ItemHost>& items) {
  const int n_c = P->d * (P->d + 1) / 2;
  items.resize(n_loads);
  for (int lc = 0; lc < n_loads; ++lc) {
    ItemHost& it = items[lc];
    it.field = nullptr;
    it.phase = phase;
    it.table = 0;
    it.C0[0] = C0[0];
    it.C0[1] = C0[1];
    for (int c = 0; c < n_c; ++c) it.E[c] = E[(size_t)lc * n_c + c];
    it.eps = eps + (size_t)lc * n_c * P->m;
    it.sigma = sigma ? sigma + (size_t)lc * n_c * P->m : nullptr;
  }
}

}  // namespace latms_detail

using namespace latms_detail;

int lat_blue_transform_bh(lat_plan* P) { return lat_blue_transform_bh_impl(P); }

// the precision argument of the workspace queries: a precision, plus LAT_WS_CG for conjugate gradients
static int ws_scheme(int precision) { return (precision & LAT_WS_CG) ? LAT_SCHEME_CG : LAT_SCHEME_BASIC; }
static int ws_precision(int precision) { return precision & ~LAT_WS_CG; }

extern "C" size_t lattice_workspace_bytes(const lat_plan* P, int n_loads, int precision) {
  const int prec = ws_precision(precision);
  if (!P || n_loads <= 0 || check_geometry(P, prec) != LAT_OK) return 0;
  return layout(P, n_loads, prec, kMaxPhases, 1, ws_scheme(precision)).total;
}

extern "C" size_t lattice_batch_workspace_bytes(const lat_plan* P, int n_items, int precision) {
  const int prec = ws_precision(precision);
  if (!P || n_items <= 0 || check_geometry(P, prec) != LAT_OK) return 0;
  return layout(P, n_items, prec, LAT_BATCH_MAX_PHASES, n_items, ws_scheme(precision)).total;
}

extern "C" size_t lattice_fft_workspace_bytes(const lat_plan* P, int n_fields) {
  // the convolution lines of a chirp-z row (blue_L complex binary64 per row of every field); else none
  if (!P || n_fields < 1 || !P->blue) return 0;
  return (size_t)n_fields * P->nrows * P->blue_L * sizeof(double2);
}

extern "C" int basic_scheme_solve(const lat_plan* P, const uint8_t* phase, int n_phases, const double* stiffness,
                                  const double* C0, const double* E, int n_loads, double tol, int maxit,
                                  const lat_solve_opts* opts, double* eps, double* sigma, double* sigma_bar,
                                  int* iters, double* resid, void* workspace, size_t workspace_bytes,
                                  void* stream) {
  if (!P || !phase || !stiffness || !C0 || !E || !eps || !workspace)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve: NULL argument");
  if (n_phases < 1 || n_phases > kMaxPhases) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve: n_phases not in 1..256");
  if (n_loads < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve: n_loads < 1");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  if (int rc = check_c0(C0)) return rc;
  const Work wl = layout(P, n_loads, o.precision, kMaxPhases, 1, o.scheme);
  if (workspace_bytes < wl.total) return lat_fail(LAT_ERR_SIZE, "workspace too small");
  if (((uintptr_t)eps & eps_align_mask(P)) != 0) return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  std::vector<ItemHost> items;
  load_case_items(P, phase, C0, E, n_loads, eps, sigma, items);
  const LatDev dv = make_dev(P, o.precision);
  return run_batch(P, items, {stiffness}, {n_phases}, tol, maxit, o, (char*)workspace, wl, dv, o.plain_launches == 0, sigma_bar,
                   iters, resid, (cudaStream_t)stream);
}

extern "C" int basic_scheme_solve_async(const lat_plan* P, const uint8_t* phase, int n_phases,
                                        const double* stiffness, const double* C0, const double* E, int n_loads,
                                        double tol, int maxit, const lat_solve_opts* opts, double* eps, double* sigma,
                                        double* sigma_bar_d, int* iters_d, double* resid_d, int* status_d,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  if (!P || !phase || !stiffness || !C0 || !E || !eps || !workspace)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_async: NULL argument");
  if (n_phases < 1 || n_phases > kMaxPhases)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_async: n_phases not in 1..256");
  if (n_loads < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_async: n_loads < 1");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.resid_history || o.plain_launches)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_async: no residual history and no plain launches (both need "
                                 "the host during the solve)");
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  if (int rc = check_c0(C0)) return rc;
  const Work wl = layout(P, n_loads, o.precision, kMaxPhases, 1, o.scheme);
  if (workspace_bytes < wl.total) return lat_fail(LAT_ERR_SIZE, "workspace too small");
  if (((uintptr_t)eps & eps_align_mask(P)) != 0) return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  std::vector<ItemHost> items;
  load_case_items(P, phase, C0, E, n_loads, eps, sigma, items);
  const LatDev dv = make_dev(P, o.precision);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<GroupRun> groups(1);
  if (int rc = group_prepare(P, items, {stiffness}, {n_phases}, tol, maxit, o, (char*)workspace, wl, dv, groups[0], st))
    return rc;
  const AsyncOut aout = {sigma_bar_d, iters_d, resid_d, status_d};
  return run_groups(groups, true, st, &aout);
}

extern "C" size_t lattice_field_workspace_bytes(const lat_plan* P, int n_loads, int precision) {
  if (!P || n_loads <= 0 || check_geometry(P, precision) != LAT_OK) return 0;
  return layout(P, n_loads, precision, 1, 1, LAT_SCHEME_BASIC, true).total;
}

extern "C" int basic_scheme_solve_field(const lat_plan* P, const double* voigt, const double* C0, const double* E,
                                        int n_loads, double tol, int maxit, const lat_solve_opts* opts, double* eps,
                                        double* sigma, double* sigma_bar, int* iters, double* resid,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  if (!P || !voigt || !C0 || !E || !eps || !workspace)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_field: NULL argument");
  if (n_loads < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_field: n_loads < 1");
  if (((uintptr_t)voigt & 15) != 0) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_field: field not 16-byte aligned");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.scheme != LAT_SCHEME_BASIC)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_field: Algorithm 1 only (the accelerated schemes need "
                                 "per-phase tables)");
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  if (int rc = check_c0(C0)) return rc;
  const Work wl = layout(P, n_loads, o.precision, 1, 1, LAT_SCHEME_BASIC, true);
  if (workspace_bytes < wl.total) return lat_fail(LAT_ERR_SIZE, "workspace too small");
  if (((uintptr_t)eps & eps_align_mask(P)) != 0) return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  std::vector<ItemHost> items;
  load_case_items(P, nullptr, C0, E, n_loads, eps, sigma, items);
  for (ItemHost& it : items) it.field = voigt;
  // the per-phase tables are not read; one placeholder phase (the reference medium) keeps their layout
  double ref[36];
  memset(ref, 0, sizeof(ref));
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) ref[a * 6 + b] = C0[0];
    ref[a * 6 + a] = C0[0] + 2 * C0[1];
    ref[(a + 3) * 6 + (a + 3)] = C0[1];
  }
  const LatDev dv = make_dev(P, o.precision);
  return run_batch(P, items, {ref}, {1}, tol, maxit, o, (char*)workspace, wl, dv, o.plain_launches == 0, sigma_bar,
                   iters, resid, (cudaStream_t)stream);
}

extern "C" int basic_scheme_solve_batch(const lat_plan* P, const lat_batch_item* bitems, int n_items, double tol,
                                        int maxit, const lat_solve_opts* opts, double* sigma_bar, int* iters,
                                        double* resid, void* workspace, size_t workspace_bytes, void* stream) {
  if (!P || !bitems || !workspace || n_items < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_batch: bad argument");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  const int n_c = P->d * (P->d + 1) / 2;
  std::vector<ItemHost> items(n_items);
  std::vector<const double*> stiff(n_items);
  std::vector<int> nph(n_items);
  for (int i = 0; i < n_items; ++i) {
    const lat_batch_item& b = bitems[i];
    if (!b.phase || !b.stiffness || !b.E || !b.eps) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_batch: NULL item field");
    if (b.n_phases < 1 || b.n_phases > LAT_BATCH_MAX_PHASES)
      return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_batch: item n_phases not in 1..LAT_BATCH_MAX_PHASES");
    if (int rc = check_c0(b.C0)) return rc;
    if (((uintptr_t)b.eps & eps_align_mask(P)) != 0) return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
    ItemHost& it = items[i];
    it.phase = b.phase;
    it.table = i;
    it.C0[0] = b.C0[0];
    it.C0[1] = b.C0[1];
    for (int c = 0; c < n_c; ++c) it.E[c] = b.E[c];
    it.eps = b.eps;
    it.sigma = b.sigma;
    stiff[i] = b.stiffness;
    nph[i] = b.n_phases;
  }
  const Work wl = layout(P, n_items, o.precision, LAT_BATCH_MAX_PHASES, n_items, o.scheme);
  if (workspace_bytes < wl.total) return lat_fail(LAT_ERR_SIZE, "workspace too small");
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  const LatDev dv = make_dev(P, o.precision);
  return run_batch(P, items, stiff, nph, tol, maxit, o, (char*)workspace, wl, dv, o.plain_launches == 0, sigma_bar, iters, resid,
                   (cudaStream_t)stream);
}

namespace {

// items of basic_scheme_solve_multi grouped by plan (order of first appearance)
struct MultiGroup {
  const lat_plan* P;
  std::vector<int> inst;   // indices into the caller's items
  int n_loads;             // load cases over the group = batch items
};

int multi_groups(const lat_multi_item* items, int n, std::vector<MultiGroup>& groups) {
  groups.clear();
  for (int i = 0; i < n; ++i) {
    const lat_multi_item& b = items[i];
    if (!b.plan || !b.phase || !b.stiffness || !b.E || !b.eps)
      return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_multi: NULL item field");
    if (b.n_phases < 1 || b.n_phases > LAT_BATCH_MAX_PHASES)
      return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_multi: item n_phases not in 1..LAT_BATCH_MAX_PHASES");
    if (b.n_loads < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_multi: item n_loads < 1");
    size_t k = 0;
    while (k < groups.size() && groups[k].P != b.plan) ++k;
    if (k == groups.size()) groups.push_back(MultiGroup{b.plan, {}, 0});
    groups[k].inst.push_back(i);
    groups[k].n_loads += b.n_loads;
  }
  return LAT_OK;
}

}  // namespace

extern "C" size_t lattice_multi_workspace_bytes(const lat_multi_item* items, int n_items, int precision) {
  if (!items || n_items < 1) return 0;
  std::vector<MultiGroup> groups;
  if (multi_groups(items, n_items, groups) != LAT_OK) return 0;
  size_t total = 0;
  const int prec = ws_precision(precision), scheme = ws_scheme(precision);
  for (const MultiGroup& g : groups) {
    if (check_geometry(g.P, prec) != LAT_OK) return 0;
    total += align256(layout(g.P, g.n_loads, prec, LAT_BATCH_MAX_PHASES, (int)g.inst.size(), scheme).total);
  }
  return total;
}

extern "C" int basic_scheme_solve_multi(const lat_multi_item* items, int n_items, double tol, int maxit,
                                        const lat_solve_opts* opts, void* workspace, size_t workspace_bytes,
                                        void* stream) {
  if (!items || n_items < 1 || !workspace) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_multi: bad argument");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.resid_history) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_multi: residual histories are not kept");
  std::vector<MultiGroup> mg;
  if (int rc = multi_groups(items, n_items, mg)) return rc;
  if (workspace_bytes <
      lattice_multi_workspace_bytes(items, n_items, o.precision | (o.scheme == LAT_SCHEME_CG ? LAT_WS_CG : 0)))
    return lat_fail(LAT_ERR_SIZE, "workspace too small");
  for (int i = 0; i < n_items; ++i) {
    if (int rc = check_c0(items[i].C0)) return rc;
    if (((uintptr_t)items[i].eps & eps_align_mask(items[i].plan)) != 0)
      return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
  }
  for (const MultiGroup& g : mg) {
    if (int rc = check_common(g.P, tol, maxit, o)) return rc;
    if (int rc = lat_plan_device_check(g.P)) return rc;
  }
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<GroupRun> runs(mg.size());
  char* ws = (char*)workspace;
  size_t off = 0;
  for (size_t k = 0; k < mg.size(); ++k) {
    const MultiGroup& g = mg[k];
    const int n_c = g.P->d * (g.P->d + 1) / 2;
    std::vector<ItemHost> its;
    std::vector<const double*> stiff;
    std::vector<int> nph;
    for (size_t t = 0; t < g.inst.size(); ++t) {
      const lat_multi_item& b = items[g.inst[t]];
      for (int lc = 0; lc < b.n_loads; ++lc) {
        ItemHost it{};
        it.phase = b.phase;
        it.table = (int)t;
        it.C0[0] = b.C0[0];
        it.C0[1] = b.C0[1];
        for (int c = 0; c < 6; ++c) it.E[c] = c < n_c ? b.E[(size_t)lc * n_c + c] : 0.0;
        it.eps = b.eps + (size_t)lc * n_c * g.P->m;
        it.sigma = b.sigma ? b.sigma + (size_t)lc * n_c * g.P->m : nullptr;
        its.push_back(it);
      }
      stiff.push_back(b.stiffness);
      nph.push_back(b.n_phases);
    }
    const Work wl = layout(g.P, g.n_loads, o.precision, LAT_BATCH_MAX_PHASES, (int)g.inst.size(), o.scheme);
    const LatDev dv = make_dev(g.P, o.precision);
    if (int rc = group_prepare(g.P, its, stiff, nph, tol, maxit, o, ws + off, wl, dv, runs[k], st)) return rc;
    off += align256(wl.total);
  }
  if (int rc = run_groups(runs, o.plain_launches == 0, st)) return rc;
  int status = LAT_OK;
  for (size_t k = 0; k < mg.size(); ++k) {
    const MultiGroup& g = mg[k];
    const int n_c = g.P->d * (g.P->d + 1) / 2;
    std::vector<double> sb((size_t)g.n_loads * n_c);
    std::vector<int> it(g.n_loads);
    std::vector<double> r(g.n_loads);
    status = std::max(status, group_decode(runs[k], o, sb.data(), it.data(), r.data()));
    int j = 0;
    for (int idx : g.inst) {
      const lat_multi_item& b = items[idx];
      for (int lc = 0; lc < b.n_loads; ++lc, ++j) {
        if (b.sigma_bar)
          for (int c = 0; c < n_c; ++c) b.sigma_bar[lc * n_c + c] = sb[(size_t)j * n_c + c];
        if (b.iters) b.iters[lc] = it[j];
        if (b.resid) b.resid[lc] = r[j];
      }
    }
  }
  return status;
}

extern "C" int lattice_pass_times(const lat_plan* P, const uint8_t* phase, int n_phases, const double* stiffness,
                                  const double* C0, const double* E, int n_loads, int precision, int n_reps,
                                  double* eps, void* workspace, size_t workspace_bytes, void* stream, float* ms_out,
                                  int* n_out) {
  if (!P || !phase || !stiffness || !C0 || !E || !eps || !workspace || !ms_out || n_reps < 1 || n_loads < 1)
    return lat_fail(LAT_ERR_ARG, "lattice_pass_times: bad argument");
  if (P->nax == 0) return lat_fail(LAT_ERR_ARG, "lattice_pass_times: m = 1 has no passes");
  if (P->general) return lat_fail(LAT_ERR_UNSUPPORTED, "lattice_pass_times: power-of-two plans only");
  // one solve with maxit = 1 sets up tables, workspace and the spectrum; then time plain launches
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  o.precision = precision;
  int rc = basic_scheme_solve(P, phase, n_phases, stiffness, C0, E, n_loads, 0.0, 1, &o, eps, nullptr, nullptr,
                              nullptr, nullptr, workspace, workspace_bytes, stream);
  if (rc < 0) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = P->d, n_c = d * (d + 1) / 2;
  const int ni = n_loads;
  const Work wl = layout(P, ni, precision, kMaxPhases, 1);
  char* ws = (char*)workspace;
  const bool fp32 = (precision == LAT_MIXED);
  const LatDev dv = make_dev(P, precision);
  Geometry geo;
  memset(&geo, 0, sizeof(geo));
  if ((rc = geometry(P, n_c, fp32 ? 8 : 16, P->Rh, true, geo, ni, precision)) != LAT_OK) return rc;
  // keep the item active for every timed launch: maxit far away, tol 0
  CK(cudaMemsetAsync(ws + wl.scal, 0, (size_t)(ni + 1) * kScalBytes, st));
  RowArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.flags = ROW_UPDATE | (P->nax == 1 ? ROW_GAMMA : 0) | (fp32 ? ROW_INCREMENT | ROW_INCR_FIRST : 0);
  {  // the same material form as the solve
    bool ortho = true;
    double T[36];
    for (int p = 0; p < n_phases; ++p) {
      voigt_to_tc(stiffness + 36 * p, d, T);
      ortho = ortho && tc_ortho(T, n_c, d);
    }
    if (ortho) ra.flags |= ROW_ORTHO;
  }
  ra.rpc = geo.rpc;
  ra.items = (const ItemDev*)(ws + wl.items);
  ra.T = ws + wl.T;
  ra.TN = ws + wl.TN;
  ra.t_stride = (int64_t)(wl.t_per_lc / (fp32 ? 8 : 16));
  ra.tn_stride = (int64_t)(wl.tn_per_lc / (fp32 ? 8 : 16));
  mat_set_gscale(ra.mat, -1.0 / (double)P->m);
  ra.it.partials = (double*)(ws + wl.partials);
  ra.it.pstride = wl.pstride;
  ra.it.scal = (ItemScal*)(ws + wl.scal);
  ra.it.glob = (GlobScal*)(ws + wl.scal + (size_t)ni * kScalBytes);
  ra.it.hist = (double*)(ws + wl.hist);
  ra.it.tol = 0.0;
  ra.it.maxit = 1 << 30;
  ra.it.n_items = ni;
  ra.it.cond = 0;
  GlobScal g0;
  g0.arrivals = 0;
  g0.active = ni;
  CK(cudaMemcpyAsync(ra.it.glob, &g0, sizeof(g0), cudaMemcpyHostToDevice, st));
  ColArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.row_slots = P->Rh;
  ca.has_nyq = 1;
  ca.n_f = n_c;
  ca.T = ra.T;
  ca.TN = ra.TN;
  ca.t_stride = ra.t_stride;
  ca.tn_stride = ra.tn_stride;
  ca.scale = 1.0;
  ca.items = ra.items;
  ca.mat = ra.mat;
  const int nk = 1 + (P->ngroups > 0 ? 2 * P->ngroups - 1 : 0);
  std::vector<cudaEvent_t> ev(2 * nk);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  std::vector<double> acc(nk, 0.0);
  if (precision != LAT_FP64) launch_eps_df(ra.items, ni, n_c, P->m, 1, st);   // as inside the solve
  for (int rep = 0; rep < n_reps; ++rep) {
    int k = 0;
    CK(cudaEventRecord(ev[2 * k], st));
    by_kind(precision, [&](auto tag) {
      launch_row_pass<decltype(tag)>(dv, ra, geo.row_blocks, ni, kThreads, geo.row_smem, st);
      return 0;
    });
    CK(cudaEventRecord(ev[2 * k + 1], st));
    ++k;
    auto one = [&](int gi, int mode) {
      ColArgs c = ca;
      const LatGroup& G = P->grp[gi];
      c.mode = mode;
      c.gidx = gi;
      c.a0 = G.a0;
      c.a1 = G.a1;
      c.G = G.G;
      c.outer = G.outer;
      c.inner = G.inner;
      c.has_twiddle = G.has_twiddle;
      c.w = geo.w[gi];
      c.wN = geo.wN[gi];
      c.tiles_main = geo.tiles_main[gi];
      c.tiles_nyq = geo.tiles_nyq[gi];
      cudaEventRecord(ev[2 * k], st);
      by_kind(precision, [&](auto tag) {
        launch_col_pass<decltype(tag)>(dv, c, ni, kThreads, geo.col_smem[gi], st);
        return 0;
      });
      cudaEventRecord(ev[2 * k + 1], st);
      ++k;
    };
    for (int gi = P->ngroups - 1; gi >= 0; --gi) one(gi, gi == 0 ? COL_GAMMA : COL_FWD);
    for (int gi = 1; gi < P->ngroups; ++gi) one(gi, COL_INV);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < k; ++j) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]));
      acc[j] += ms;
    }
  }
  if (precision != LAT_FP64) launch_eps_df(ra.items, ni, n_c, P->m, 0, st);
  CK(cudaStreamSynchronize(st));
  for (auto& e : ev) cudaEventDestroy(e);
  for (int j = 0; j < 8; ++j) ms_out[j] = j < nk ? (float)(acc[j] / n_reps) : 0.0f;
  if (n_out) *n_out = nk;
  return LAT_OK;
}

extern "C" int lattice_fft(const lat_plan* P, const double* in, double* out, int n_fields, int inverse,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!P || !in || !out || n_fields < 1) return lat_fail(LAT_ERR_ARG, "lattice_fft: bad argument");
  if (in == out) return lat_fail(LAT_ERR_ARG, "lattice_fft: in and out must not overlap");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t m = P->m;
  if (P->nax == 0) {
    CK(cudaMemcpyAsync(out, in, (size_t)n_fields * 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return LAT_OK;
  }
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  const LatDev dv = make_dev(P, LAT_FP64);
  Geometry geo;
  int rc = geometry(P, 1, 16, P->Rlen, false, geo, 1);
  if (rc != LAT_OK) return rc;
  const double inv_m = 1.0 / (double)m;
  if (P->blue && (!workspace || workspace_bytes < lattice_fft_workspace_bytes(P, n_fields)))
    return lat_fail(LAT_ERR_SIZE, "lattice_fft: the chirp-z row needs lattice_fft_workspace_bytes of workspace");
  // chirp-z row (general plans): the row transforms of all fields at once, before the forward column
  // passes and after the inverse ones
  const int64_t y_lines = (int64_t)n_fields * P->nrows;
  if (P->blue && !inverse)
    blue_rows(dv, (const double2*)in, m, (double2*)out, m, (int)P->nrows, n_fields, (double2*)workspace, y_lines, 0,
              P->ngroups == 0 ? inv_m : 1.0, st);
  for (int f = 0; f < n_fields; ++f) {
    const double2* fin = (const double2*)in + (size_t)f * m;
    double2* fout = (double2*)out + (size_t)f * m;
    ColArgs base;
    memset(&base, 0, sizeof(base));
    base.row_slots = P->Rlen;
    base.has_nyq = 0;
    base.n_f = 1;
    base.T = fout;
    base.TN = nullptr;
    base.scale = 1.0;
    auto col = [&](int k, int mode, const void* tin, double scale) {
      ColArgs c = base;
      const LatGroup& G = P->grp[k];
      c.mode = mode;
      c.gidx = k;
      c.a0 = G.a0;
      c.a1 = G.a1;
      c.G = G.G;
      c.outer = G.outer;
      c.inner = G.inner;
      c.has_twiddle = G.has_twiddle;
      c.w = geo.w[k];
      c.wN = geo.wN[k];
      c.tiles_main = geo.tiles_main[k];
      c.tiles_nyq = 0;
      c.Tin = tin;
      c.scale = scale;
      c.do_scale = scale != 1.0;
      if (P->general) launch_gen_col<double>(dv, c, 1, kThreads, geo.col_smem[k], st);
      else launch_col_pass<double>(dv, c, 1, kThreads, geo.col_smem[k], st);
    };
    auto row = [&](const void* rin, int inv, double scale) {
      if (P->general) launch_gen_row_complex(dv, rin, fout, inv, scale, geo.rpc, kThreads, geo.row_smem, st);
      else launch_row_complex<double>(dv, rin, fout, 1, inv, scale, geo.rpc, kThreads, geo.row_smem, st);
    };
    if (!inverse) {
      if (!P->blue) row(fin, 0, P->ngroups == 0 ? inv_m : 1.0);
      for (int k = P->ngroups - 1; k >= 0; --k) col(k, COL_FWD, nullptr, k == 0 ? inv_m : 1.0);
    } else {
      for (int k = 0; k < P->ngroups; ++k) col(k, COL_INV, k == 0 ? (const void*)fin : nullptr, 1.0);
      if (!P->blue) row(P->ngroups == 0 ? (const void*)fin : (const void*)fout, 1, 1.0);
    }
    CK(cudaGetLastError());
  }
  if (P->blue && inverse)
    blue_rows(dv, (const double2*)(P->ngroups == 0 ? in : out), m, (double2*)out, m, (int)P->nrows, n_fields,
              (double2*)workspace, y_lines, 1, 1.0, st);
  CK(cudaGetLastError());
  return LAT_OK;
}
