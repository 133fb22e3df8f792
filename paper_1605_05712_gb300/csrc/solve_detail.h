// solve_detail.h -- launch geometry, workspace layout and the batch driver shared by the solve
// entry points (not installed).
#pragma once
#include <string>
#include <vector>

#include "kernels.cuh"

namespace latms_detail {

const size_t kMaxSmem = 232448;       // sm_100/sm_103 opt-in dynamic shared memory per block
const size_t kRowSmemTarget = 64 * 1024;
// column tiles at most ~100 KB, so that two blocks share an SM: at 128^3 the six-component Green pass ran
// 1.5x faster (mixed) than with the widest 196 KB tile, matching what lattice_autotune picks
const size_t kColSmemMax = 100 * 1024;
const int kThreads = 256;
const int kMaxPhases = 256;           // phases of the single material of basic_scheme_solve
const int kEffBlocksMax = 256;        // blocks of the effective-stress reduction per item
const size_t kScalBytes = 256;        // device scalars per item (ItemScal), plus one slot for GlobScal

struct Geometry {
  int rpc, row_blocks;
  size_t row_smem;
  int w[LAT_MAX_GROUPS], wN[LAT_MAX_GROUPS];
  int64_t tiles_main[LAT_MAX_GROUPS], tiles_nyq[LAT_MAX_GROUPS];
  size_t col_smem[LAT_MAX_GROUPS];
};

// byte offsets of the workspace regions of a batched solve
struct Work {
  size_t T, TN, items, tables, tables_f, tables_df, tables_w, tables_wf, tables_wdf, partials, scal, hist, total;
  size_t T64, TN64;   // mixed precision: binary64 spectrum of the restart (0 bytes otherwise)
  size_t cgv;         // conjugate gradients: r, p, q, w per item (0 bytes otherwise)
  size_t fld_f, fld_df;  // stiffness-field solves: binary32 and pair copies of the field (0 bytes otherwise)
  int64_t cg_stride;  // doubles per vector and item (n_c m)
  size_t t_per_lc, tn_per_lc, table_bytes;
  int64_t pstride;  // doubles of reduction partials per item
};

// host description of one item of a batch
struct ItemHost {
  const double* field;  // device 21 x m Voigt stiffness field (basic_scheme_solve_field), else NULL
  const uint8_t* phase;
  int table;        // index of its material table
  double C0[2];
  double E[6];
  double* eps;
  double* sigma;
};

int ensure_attrs();
// kind = the precision: LAT_FP64, LAT_MIXED (binary32 kernels) or LAT_DF64 (double-float kernels)
LatDev make_dev(const lat_plan* P, int kind);
// calls f(Real{}) with the kernel type of a precision
template <typename F>
int by_kind(int kind, F f) {
  if (kind == LAT_MIXED) return f(float{});
  if (kind == LAT_DF64) return f(dfloat{});
  return f(double{});
}
int geometry(const lat_plan* P, int n_f, size_t cs, int row_slots, bool nyq, Geometry& g, int n_items, int kind = -1);
int geometry_set_rpc(const lat_plan* P, int n_f, size_t cs, bool nyq, int rpc, Geometry& g);
int geometry_set_w(const lat_plan* P, int n_f, size_t cs, int row_slots, bool nyq, int k, int64_t w, Geometry& g);
int tune_bucket(int n_items);
size_t align256(size_t x);
template <typename Real>
void enqueue_col_group(const LatDev& dv, const lat_plan* P, const Geometry& g, ColArgs c, int k, int mode,
                       int n_items, cudaStream_t st);
// scheme = LAT_SCHEME_CG adds the four vectors of the conjugate-gradient iteration
// field: a per-point stiffness field (basic_scheme_solve_field) adds its binary32 / pair copies
Work layout(const lat_plan* P, int n_items, int precision, int phases_per_table, int n_tables,
            int scheme = LAT_SCHEME_BASIC, bool field = false);
void voigt_to_tc(const double* V, int d, double* out);
template <typename Real>
void enqueue_columns(const LatDev& dv, const lat_plan* P, const Geometry& g, ColArgs base, int n_items,
                     cudaStream_t st);
int check_common(const lat_plan* P, double tol, int maxit, const lat_solve_opts& o);
int check_geometry(const lat_plan* P, int precision);
int check_c0(const double* C0);
size_t eps_align_mask(const lat_plan* P);
void load_case_items(const lat_plan* P, const uint8_t* phase, const double* C0, const double* E, int n_loads,
                     double* eps, double* sigma, std::vector<ItemHost>& items);
// one batch of items on one plan, prepared for a loop that may run beside other batches
struct GroupRun {
  const lat_plan* P;
  int n_items, n_c, maxit;
  double tol;
  int kind;           // LAT_FP64, LAT_MIXED or LAT_DF64
  bool fp32, loop, want_hist;
  LatDev dv;
  Geometry geo;
  RowArgs full;       // loop body row pass (with the pause level when a restart follows)
  bool cg;            // conjugate gradients: the loop body is cg_row(B), columns, cg_row(A)
  CgArgs cga;
  ColArgs cl;
  // restart of the increment form on double-float pairs (binary64-accurate): prologue of the paused
  // items (r_pro, c64), update whose polarization is of the exact increment (r_upd), cast of the
  // spectrum to binary32, binary32 columns (cl), then the second loop (full2)
  bool restart;
  LatDev dv64;
  Geometry geo64;
  RowArgs r_pro, r_upd, full2;
  ColArgs c64;
  EffArgs ea;
  int eff_blocks;
  char* ws;
  Work wl;
  GlobScal glob0;
  std::vector<double> tabs;     // host staging, alive until the stream is synchronized
  std::vector<float> tabs_f;
  std::vector<float2> tabs_df;
  std::vector<double> tabs_w;   // (C + C0)^{-1} (Eyre-Milton)
  std::vector<float> tabs_wf;
  std::vector<float2> tabs_wdf;
  std::vector<ItemDev> hdev;
  std::vector<char> scal;       // host copy of the item scalars after the solve
  std::vector<double> hist;
};
// uploads tables and items, fills eps^(0) = E (cold start) and enqueues the prologue on `st`
int group_prepare(const lat_plan* P, const std::vector<ItemHost>& items, const std::vector<const double*>& stiff,
                  const std::vector<int>& nph, double tol, int maxit, const lat_solve_opts& o, char* ws,
                  const Work& wl, const LatDev& dv, GroupRun& g, cudaStream_t st);
// device destinations of the scalar results of an asynchronous solve (any may be NULL)
struct AsyncOut {
  double* sigma_bar;
  int* iters;
  double* resid;
  int* status;
};
// the loops of all groups (one CUDA graph with a WHILE node per group, or plain launches), then the
// effective stress and the scalars of every group; returns after synchronizing `st`, or, with aout (one
// group, graph loop), as soon as everything is enqueued, the scalars going to device memory
int run_groups(std::vector<GroupRun>& groups, bool use_graph, cudaStream_t st, const AsyncOut* aout = nullptr);
// outputs of a finished group; returns its worst status
int group_decode(const GroupRun& g, const lat_solve_opts& o, double* sigma_bar, int* iters, double* resid);
// runs a batch on workspace `ws` laid out by `wl`; dv carries the twiddle-table pointers;
// use_graph: CUDA-graph WHILE loop, else plain launches with a host check per iteration
int run_batch(const lat_plan* P, const std::vector<ItemHost>& items, const std::vector<const double*>& stiff,
              const std::vector<int>& nph, double tol, int maxit, const lat_solve_opts& o, char* ws, const Work& wl,
              const LatDev& dv, bool use_graph, double* sigma_bar, int* iters, double* resid, cudaStream_t st);
// chirp-z row transforms of a plan with lat_plan::blue (solve.cu): lines j < lines_per_item of item i at
// src + i src_stride + j p -> dst likewise (complex binary64, in place allowed); Y holds y_lines lines of
// blue_L; inverse: the unnormalized inverse DFT; scale multiplies the result
void blue_rows(const LatDev& dv, const double2* src, int64_t src_stride, double2* dst, int64_t dst_stride,
               int lines_per_item, int n_items, double2* Y, int64_t y_lines, int inverse, double scale,
               cudaStream_t st);
int lat_blue_transform_bh_impl(lat_plan* P);
// the pointwise part of a conjugate-gradient stage on a chirp-z plan (kernels_blue_cg.cu): vector updates,
// inner products, step lengths or residual report; tau = C : v except in stage A; grid nblocks x items
void launch_blue_cg_point(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items,
                          cudaStream_t st);

}  // namespace latms_detail

// host copies of the plan's twiddle tables (W_N^t, N = 2^tw_log2, and the split table
// [hi | lo]) in binary64 or binary32 pairs; returns the two table lengths in entries
int lat_host_twiddles(const lat_plan* P, int fp32, void* tw, void* stw, int64_t* n_tw, int64_t* n_stw);
// at plan creation: d_bh (the wrapped conjugate chirp) -> its DFT by the chirp-z sub-plan, on the device
int lat_blue_transform_bh(lat_plan* P);
