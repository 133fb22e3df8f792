// internal.h -- plan layout and kernel parameter blocks of liblatms (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lattice_ms.h"

#define LAT_MAX_AX 6
#define LAT_MAX_GROUPS 3
#define LAT_MAX_RADIX 16  // stages of a mixed-radix axis transform
#define LAT_HIST_CAP 4096  // residuals kept per item in the workspace

// One logical FFT axis in storage order (row-major, last = contiguous row).
struct LatAxis {
  int len;         // length (a power of two, or any length on a general plan)
  int log2len;
  int snf;         // elementary-divisor axis j this axis belongs to
  int64_t mult;    // k_j += mult * (spectral index on this axis)
  int64_t cv[3];   // (mult * c_j) mod e_d: contribution to v = Q^{-T} E^{-1} k * e_d
};

// One column pass: FFT over the logical axes [a0, a1) on tiles of columns.
struct LatGroup {
  int a0, a1;
  int G;            // product of the group's lengths
  int64_t outer;    // product of lengths of axes [0, a0)
  int64_t inner;    // product of lengths of axes [a1, nax-1) (row axis excluded)
  int has_twiddle;  // the split axis' n1 lies in this group (four-step twiddle before/after)
};

struct lat_plan {
  int d;
  int64_t M[3][3];
  int64_t det, m;
  int64_t Q[3][3], R[3][3], Rinv[3][3], P[3][3];  // M = Q diag(e) R, P = Q^{-T}
  int64_t e[3];
  int dM;
  int64_t ed;        // largest elementary divisor (lcm of all)
  // FFT decomposition
  int nax;           // logical axes, ax[nax-1] is the contiguous row
  LatAxis ax[LAT_MAX_AX];
  int Rlen, Rh, log2Rh;  // row length (real samples) and its half
  int64_t nrows;     // m / Rlen
  int ngroups;       // column passes; grp[0] holds axis 0 and applies Gamma0
  LatGroup grp[LAT_MAX_GROUPS];
  int split;         // 1 if the largest divisor is split into (n1, n2 = row)
  int split_n1;      // logical index of n1
  int64_t split_e;   // the split divisor e = A * B
  int split_lo_log2; // two-level twiddle table split: W_e^j = hi[j >> s] * lo[j & (2^s-1)]
  // device tables (owned)
  int tw_log2;       // twiddle table W_N^t, N = 2^tw_log2
  double2* d_tw;
  float2* d_twf;
  double2* d_stw;    // split twiddles: [hi (e >> s) | lo (2^s)]
  float2* d_stwf;
  float4* d_twdf;     // double-float copies (re hi, re lo, im hi, im lo)
  float4* d_stwdf;
  double* d_lf;       // fused multiply-add butterfly table of the binary64 kernels (power-of-two plans)
  double* d_rc;       // fused multiply-add table of their real-row pre/post-processing
  int64_t stw_hi_n, stw_lo_n;
  int device;        // device holding the tables (-1: created without a CUDA device, host-only)
  // transformed pattern (lattice_plan_set_cell): has_cell and L^{-T}
  int has_cell;
  double cell_LinvT[3][3];
  // general plans (an elementary divisor that is not a power of two): mixed-radix natural-order transforms,
  // one logical axis per column pass, full complex spectrum; radices of each logical axis and the offset
  // of its table of W_len^t in the twiddle table (the tables of all axes concatenated)
  int general;
  int ax_nrad[LAT_MAX_AX];
  uint16_t ax_rad[LAT_MAX_AX][LAT_MAX_RADIX];
  int ax_twoff[LAT_MAX_AX];
  // general plans whose largest divisor p is longer than one line in shared memory and has no split
  // into two lines that fit: the row axis (length p, not split) is transformed by Bluestein's chirp-z
  // convolution, a cyclic convolution of power-of-two length blue_L >= 2p - 1 run by blue_sub (the
  // power-of-two plan diag(1, blue_L)); d_chirp[n] = exp(-i pi n^2 / p) (n < p) and d_bh the
  // unnormalized DFT of the wrapped conjugate chirp, in blue_sub's spectral order
  int blue;
  int64_t blue_L;
  lat_plan* blue_sub;
  int blue_lgA, blue_lgB;  // blue_sub's storage order: sample n at slot (n mod A) B + n / A, A B = blue_L
  double2* d_chirp;
  double2* d_bh;
  // launch shapes picked by lattice_autotune, per precision and power-of-two bucket of the item count
  struct Tune {
    int valid;
    int rpc;                     // rows per block of the row pass
    int w[LAT_MAX_GROUPS];       // tile width (columns) of each column pass
    float ms[1 + LAT_MAX_GROUPS];  // their measured device times (ms)
  } tune[3][8];
};

// Parameters shared by the solver kernels (passed by value).
struct LatDev {
  int d, n_c, nax;
  int Rlen, Rh, log2Rh;
  int64_t m, nrows;
  int64_t ed, ed_mask;        // ed_mask = ed - 1 if ed is a power of two, else -1
  int h32;                    // 1: e_d is a power of two <= 2^31 and every |h~_i| < 2^31 (32-bit path)
  int64_t MT[3][3];           // M^T (h = M^T v' / e_d)
  int ax_len[LAT_MAX_AX], ax_log2[LAT_MAX_AX];
  int64_t ax_cv[LAT_MAX_AX][3];
  int split, split_n1, split_lo_log2;
  int64_t split_e;
  int64_t stw_hi_n;
  int tw_log2;
  const void* tw;             // twiddle table (double2 or float2, per precision)
  const void* stw;            // split twiddles [hi | lo]
  const double* lf;           // binary64 butterfly table (fft_smem.cuh, FmaTw): 8 words per t < 2^tw_log2 / 4
  const double* rc;           // binary64 real-transform table: (Re w / Im w, Im w, Im w / 2, 0), w = W_N^t, t <= N/4
  // general plan: mixed-radix axes (see lat_plan)
  int general;
  int ax_nrad[LAT_MAX_AX];
  uint16_t ax_rad[LAT_MAX_AX][LAT_MAX_RADIX];
  int ax_twoff[LAT_MAX_AX];
  // Bluestein row axis (see lat_plan): its tables, and the plan itself for the host-side launchers
  int blue;
  int64_t blue_L;
  int blue_lgA, blue_lgB;     // the sub-plan stores sample n at slot (n mod A) B + n / A (L = A B)
  const double2* blue_chirp;
  const double2* blue_bh;
  const void* blue_plan;      // host pointer (const lat_plan*), never read on the device
  // transformed pattern P_L(M) (Sec. 3.3): Gamma0 at L^{-T} h; binary64, binary32 and pair copies
  int cell;
  double cellT[3][3];
  float cellT_f[3][3], cellT_lo[3][3];
};

void lat_set_error(const std::string& s);
// LAT_OK if the plan's device tables exist on the current device (lattice_plan uploads them to the device
// current at creation); LAT_ERR_CUDA for a host-only plan, LAT_ERR_ARG for another device
int lat_plan_device_check(const lat_plan* P);
int lat_fail(int code, const std::string& s);
