// solve_detail.h -- launch geometry and workspace layout shared by the solve drivers (not installed).
#pragma once
#include <string>

#include "kernels.cuh"

namespace latms_detail {

const size_t kMaxSmem = 232448;       // sm_100/sm_103 opt-in dynamic shared memory per block
const size_t kRowSmemTarget = 64 * 1024;
const size_t kColSmemMax = 200 * 1024;
const int kThreads = 256;
const int kMaxPhases = 256;
const size_t kScalBytes = 256;        // device scalars per load case

struct Geometry {
  int rpc, row_blocks;
  size_t row_smem;
  int w[LAT_MAX_GROUPS], wN[LAT_MAX_GROUPS];
  int64_t tiles_main[LAT_MAX_GROUPS], tiles_nyq[LAT_MAX_GROUPS];
  size_t col_smem[LAT_MAX_GROUPS];
};

// byte offsets of the workspace regions of a solve
struct Work {
  size_t T, TN, Dtab, Ctab, partials, scal, hist, total;
  size_t t_per_lc, tn_per_lc;
};

int ensure_attrs();
LatDev make_dev(const lat_plan* P, bool fp32);
int geometry(const lat_plan* P, int n_f, size_t cs, int row_slots, bool nyq, Geometry& g);
Work layout(const lat_plan* P, int n_loads, int precision);
void voigt_to_tc(const double* V, int d, double* out);
template <typename Real>
void enqueue_columns(const LatDev& dv, const lat_plan* P, const Geometry& g, ColArgs base, cudaStream_t st);

}  // namespace latms_detail

// host copies of the plan's twiddle tables (W_N^t, N = 2^tw_log2, and the split table
// [hi | lo]) in binary64 or binary32 pairs; returns the two table lengths in entries
int lat_host_twiddles(const lat_plan* P, int fp32, void* tw, void* stw, int64_t* n_tw, int64_t* n_stw);
