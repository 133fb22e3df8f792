// kernels.cuh -- argument blocks shared by kernels.cu and solve.cu.
#pragma once
#include "internal.h"

// Row pass flags
#define ROW_LOAD_EPS 1   // take eps^(n) from the strain buffer (first iteration / warm start)
#define ROW_UPDATE 2     // inverse-transform T into eps^(n+1), residual, write eps
#define ROW_GAMMA 4      // no column axes: apply Gamma0 on the row spectrum (d_M = 1, short)
#define ROW_INCREMENT 8  // mixed precision: T carries the increment delta, eps += delta

// Column pass modes
#define COL_FWD 0
#define COL_GAMMA 1
#define COL_INV 2

struct MatArgs {
  const double* Dtab;   // n_phases x n_c x n_c, (C_p - C0) acting on tensor components
  double E[6];          // macroscopic strain, tensor components
  double lam0, mu0;
  double c1, c2;        // 1/(2 mu0), (lam0 + mu0) / (mu0 (lam0 + 2 mu0))
  double gscale;        // -1/m: the forward 1/m of F(M) and the minus sign of the update
  int boundary_zero;
  int increment;        // 1: spectrum carries an increment, k = 0 gets 0 instead of E
};

struct IterArgs {
  double* partials;     // per-block residual partial sums
  unsigned* counter;    // last-block-done counter (reset to 0 by the last block)
  int* done;            // stop flag read by the column passes
  int* iter;            // iterations performed
  double* hist;         // residual history (LAT_HIST_CAP)
  double* last_r;       // last residual
  double norm0, tol;
  int maxit;
  unsigned long long cond;  // cudaGraphConditionalHandle of the enclosing WHILE node
};

struct RowArgs {
  int flags;
  int rpc;              // rows per block
  double* eps;          // n_c planes of m binary64 (plan order)
  const uint8_t* phase;
  void* T;              // n_c planes of m/2 complex (Real2), row slots bit-reversed
  void* TN;             // n_c planes of nrows complex: the Nyquist column
  MatArgs mat;
  IterArgs it;
};

struct ColArgs {
  int mode;
  int gidx;             // group index in the plan
  int a0, a1, G;
  int64_t outer, inner; // inner excludes the row axis
  int has_twiddle;
  int w, wN;            // tile widths for T and for the Nyquist plane
  int64_t tiles_main;   // per outer index
  int64_t tiles_nyq;
  int row_slots;        // Rh (solver, half spectrum) or Rlen (complex transform)
  int has_nyq;
  int n_f;              // planes (components or fields)
  void* T;
  void* TN;
  const void* Tin;      // first pass of the complex transform reads here (else = T)
  double scale;         // multiply on store (1/m for the last forward pass of lattice_fft), 1 = none
  MatArgs mat;
  const int* done;      // NULL or stop flag
};

struct EffArgs {
  const double* eps;
  double* sigma;        // NULL or n_c planes
  const uint8_t* phase;
  const double* Ctab;   // n_phases x n_c x n_c, C_p on tensor components
  double* partials;     // blocks x n_c
  unsigned* counter;
  double* sigma_bar;    // n_c
};

template <typename Real>
void launch_row_pass(const LatDev& dv, const RowArgs& a, int nblocks, int nthreads, size_t smem,
                     cudaStream_t st);
template <typename Real>
void launch_col_pass(const LatDev& dv, const ColArgs& a, int nthreads, size_t smem, cudaStream_t st);
void launch_fill(double* eps, int n_c, int64_t m, const double* E, cudaStream_t st);
void launch_eff(const LatDev& dv, const EffArgs& a, int nblocks, cudaStream_t st);
template <typename Real>
void launch_row_complex(const LatDev& dv, const void* in, void* out, int n_f, int inverse, double scale,
                        int rpc, int nthreads, size_t smem, cudaStream_t st);
int lat_kernel_attrs(size_t max_smem);
