// kernels.cuh -- argument blocks shared by kernels.cu and the solve drivers.
#pragma once
#include "df64.cuh"
#include "internal.h"

// Shared-memory tiles of the power-of-two kernels are padded by one complex value after every 128 bytes
// (16 binary32 complex values, 8 binary64 or double-float ones): values a multiple of 128 bytes apart --
// the strided butterflies of the short FFT stages, the same slot of neighbouring lines -- then fall into
// different banks.  tile_span(n, cs) is the number of complex slots a tile of n values occupies.
__host__ __device__ inline int64_t tile_span(int64_t n, size_t cs) { return n + n / (cs == 8 ? 16 : 8) + 1; }

// Row pass flags
#define ROW_LOAD_EPS 1   // take eps^(n) from the strain buffer (first iteration / warm start)
#define ROW_UPDATE 2     // inverse-transform T into eps^(n+1), residual, write eps
#define ROW_GAMMA 4      // no column axes: apply Gamma0 on the row spectrum (d_M = 1, short)
#define ROW_INCREMENT 8  // mixed precision (binary32 kernels only): T carries the increment delta, eps += delta
#define ROW_INCR_FIRST 16  // with ROW_INCREMENT: T carries an increment from the first iteration on (cold
                           // start: the prologue mapped k = 0 to 0, so T holds G(E) - E)
#define ROW_ONLY_PAUSED 32 // restart passes: only items in state ITEM_PAUSED take part
#define ROW_TAU_DELTA 64   // with ROW_UPDATE (double-float restart): the polarization is taken of the increment
                           // eps^(n+1) - eps^(n)
#define ROW_EPS_DF 128     // the strain buffer holds double-float pairs (mixed solve): set on the double-float
                           // restart passes; the binary32 and pair kernels always read and write it so, the
                           // binary64 kernels never (none of these three flags reaches them)
#define ROW_FIELD 256      // the material is a per-point stiffness field (ItemDev::fld*), not phase tables
#define ROW_ORTHO 512      // every phase table of the batch couples no normal and shear components and has a
                           // diagonal shear block (isotropic, cubic, axis-aligned orthotropic phases): the
                           // six-component row pass reads the normal block and the shear diagonal only

// ItemScal::done
#define ITEM_ACTIVE 0
#define ITEM_DONE 1        // converged, maxit, or non-finite residual
#define ITEM_PAUSED 2      // residual fell below the restart level: waits for the binary64 restart

// Column pass modes
#define COL_FWD 0
#define COL_GAMMA 1
#define COL_INV 2

// One independent problem of a batched solve (a load case and/or a microstructure).
struct ItemDev {
  double* eps;           // n_c planes of m binary64 (plan order)
  double* sigma;         // NULL or n_c planes
  const uint8_t* phase;  // m phase ids
  const double* Dtab;    // n_phases x n_c x n_c: (C_p - C0) on tensor components
  const float* Dtab_f;   // the same in binary32 (for the binary32 kernels)
  const dfloat* Dtab_df; // the same as double-float pairs (for the double-float kernels)
  const double* Ctab;    // n_phases x n_c x n_c: C_p on tensor components
  double E[6];           // macroscopic strain, tensor components
  double c1, c2;         // Green operator constants of this item's C0
  float c1f, c2f;
  // the same constants (and C0's Lame constants) as double-float pairs: the pair kernels read them
  // instead of converting binary64 values, which runs on the binary64 pipe at 1/64 of the binary32 rate
  dfloat c1_df, c2_df, lam0_df, mu0_df;
  // Eyre-Milton iteration: (C_p + C0)^{-1} on tensor components (maps the stress-like u to the strain),
  // the reference medium's Lame constants and 2 C0 : E (tensor components)
  const double* Wtab;
  const float* Wtab_f;
  const dfloat* Wtab_df;
  double lam0, mu0;
  float lam0f, mu0f;
  double twoC0E[6];
  double norm0;          // sqrt(m) ||E||_F (1 if E = 0)
  // per-point stiffness field (basic_scheme_solve_field; NULL otherwise): 21 planes of m values, plane p the
  // upper-triangle entry p of each point's 6x6 Voigt matrix; binary64 (the caller's), binary32 and pair copies
  const double* fld;
  const float* fld_f;
  const dfloat* fld_df;
};

// Device scalars of one item (the first bytes of its 256-byte slot)
struct ItemScal {
  unsigned counter;      // last-block-done counter of the row pass (reset by the last block)
  int done;              // ITEM_ACTIVE, ITEM_DONE or ITEM_PAUSED
  int iter;              // iterations performed
  unsigned eff_counter;  // last-block counter of the effective-stress kernel
  double last_r;         // last residual
  double sigma_bar[6];   // mean stress
  // conjugate gradients: step lengths and <r, r>_C0 of the current and the previous iteration
  double cg_alpha, cg_beta, cg_gamma, cg_gamma_prev, cg_alpha_prev;
  double cg_r0;          // first residual (the rounding floor of the iteration is relative to it)
  dfloat cg_alpha_df, cg_beta_df;  // the step lengths as pairs (for the double-float kernels)
  int grow;              // consecutive iterations whose residual exceeded the previous one
  int diverged;          // 1: stopped by the divergence rule (LAT_DIVERGED)
};

// Batch-wide device scalars
struct GlobScal {
  unsigned arrivals;     // items whose row pass finished in this iteration
  int active;            // items still iterating
};

struct MatArgs {
  double gscale;         // -1/m: the forward 1/m of F(M) and the minus sign of the update
  float gscale_f;        // the same in binary32 and as a pair (set with mat_set_gscale)
  dfloat gscale_df;
  int boundary_zero;
  int increment;         // 1: spectrum carries an increment, k = 0 gets 0 instead of E
  int scheme;            // Green step of LAT_SCHEME_BASIC (also conjugate gradients) or LAT_SCHEME_EYRE_MILTON
};

struct IterArgs {
  double* partials;      // per item: row-pass block partial sums (stride pstride)
  int64_t pstride;
  ItemScal* scal;        // per item, stride 256 bytes
  GlobScal* glob;
  double* hist;          // per item residual history, stride LAT_HIST_CAP
  double tol;
  double pause_tol;      // > 0: an item whose residual falls below it (but not below tol) pauses
  int maxit;
  int n_items;
  unsigned long long cond;  // cudaGraphConditionalHandle of the enclosing WHILE node (0: none)
};

struct RowArgs {
  int flags;
  int rpc;               // rows per block
  const ItemDev* items;  // device item table
  void* T;               // per item: n_c planes of m/2 complex (Real2), row slots bit-reversed
  void* TN;              // per item: n_c planes of nrows complex, the Nyquist column
  int64_t t_stride, tn_stride;  // elements (complex) per item
  MatArgs mat;
  IterArgs it;
};

struct ColArgs {
  int mode;
  int gidx;              // group index in the plan
  int a0, a1, G;
  int64_t outer, inner;  // inner excludes the row axis
  int has_twiddle;
  int w, wN;             // tile widths for T and for the Nyquist plane
  int64_t tiles_main;    // per outer index
  int64_t tiles_nyq;
  int row_slots;         // Rh (solver, half spectrum) or Rlen (complex transform)
  int has_nyq;
  int n_f;               // planes (components or fields)
  void* T;
  void* TN;
  int64_t t_stride, tn_stride;  // per item (blockIdx.y)
  const void* Tin;       // first pass of the complex transform reads here (else = T)
  double scale;          // multiply on store (1/m for the last forward pass of lattice_fft), 1 = none
  int do_scale;          // scale != 1 (decided on the host)
  const ItemDev* items;  // solver: E and Green constants per item
  MatArgs mat;
  const ItemScal* scal;  // NULL or per-item scalars (skip items not ITEM_ACTIVE)
  int only_paused;       // with scal: process ITEM_PAUSED items only (restart passes)
};

inline void mat_set_gscale(MatArgs& m, double g) {
  m.gscale = g;
  m.gscale_f = (float)g;
  m.gscale_df = dfloat(g);
}

// Conjugate-gradient row kernel stages
#define CG_FWD_X 0   // tau = C : x, forward transform                                   (prologue)
#define CG_FULL0 1   // r = -A x from the spectrum, <r, r>_C0, ||r||; tau = C : r, forward (prologue)
#define CG_A 2       // w = A r from the spectrum, <w, r>_C0; step lengths alpha, beta
#define CG_B 3       // p, q, x, r updates, <r, r>_C0, ||r||, convergence; tau = C : r, forward

struct CgArgs {
  double* r;             // per item (stride vstride): n_c planes of m, in the strain's storage
  double* p;             // (binary64, or double-float pairs for the double-float kernels)
  double* q;             // q = A p by recurrence
  double* w;             // w = A r
  int64_t vstride;       // doubles per item
  int stage;             // CG_*
};

struct EffArgs {
  const ItemDev* items;
  double* partials;      // per item: blocks x n_c
  int64_t pstride;
  ItemScal* scal;
};

template <typename Real>
void launch_row_pass(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, int nthreads, size_t smem,
                     cudaStream_t st);
template <typename Real>
void launch_cg_row(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items, int nthreads,
                   size_t smem, cudaStream_t st);
template <typename Real>
void launch_col_pass(const LatDev& dv, const ColArgs& a, int n_items, int nthreads, size_t smem, cudaStream_t st);
void launch_fill(const ItemDev* items, int n_items, int n_c, int64_t m, cudaStream_t st);
// the per-item results of a solve to device memory (asynchronous solves): mean stress, iterations, last
// residual and the outcome (LAT_OK, LAT_NOT_CONVERGED, LAT_DIVERGED); trivial = the plan has m = 1
void launch_scalars_out(const ItemScal* scal, int n_items, int n_c, double tol, int maxit, bool trivial,
                        double* sigma_bar, int* iters, double* resid, int* status, cudaStream_t st);
void launch_eff(const LatDev& dv, const EffArgs& a, int nblocks, int n_items, cudaStream_t st);
// binary32 and pair copies of a 21 x m binary64 stiffness field (either destination may be NULL)
void launch_field_copies(const double* fld, float* fld_f, dfloat* fld_df, int64_t n, cudaStream_t st);
// n_groups (grid.y) groups of n_f fields, m apart
template <typename Real>
void launch_row_complex(const LatDev& dv, const void* in, void* out, int n_f, int inverse, double scale,
                        int rpc, int nthreads, size_t smem, cudaStream_t st, int n_groups = 1);
int lat_kernel_attrs(size_t max_smem);
// mixed-radix kernels of general plans (kernels_gen.cu): binary64 and double-float pairs; the binary32
// instantiations launch nothing (binary32 solves are refused on general plans)
template <typename Real>
void launch_gen_row(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, int nthreads, size_t smem,
                    cudaStream_t st);
template <typename Real>
void launch_gen_col(const LatDev& dv, const ColArgs& a, int n_items, int nthreads, size_t smem, cudaStream_t st);
void launch_gen_row_complex(const LatDev& dv, const void* in, void* out, int inverse, double scale, int rpc,
                            int nthreads, size_t smem, cudaStream_t st);
// the conjugate-gradient row stages (cg_row_kernel's) on a general plan: binary64 and pairs
template <typename Real>
void launch_gen_cg_row(const LatDev& dv, const RowArgs& a, const CgArgs& cg, int nblocks, int n_items, int nthreads,
                       size_t smem, cudaStream_t st);
int lat_gen_kernel_attrs(int optin);
// chirp-z rows (kernels_gen.cu, binary64): line l0 + y (y < nl) of the batch is line j = l % lines_per_item
// of item i = l / lines_per_item, p complex values at base + i stride + j p; Y holds nl lines of L in the
// sub-plan's storage order, sample n at slot(n) = (n mod A) B + n / A (A = 2^lgA, B = 2^lgB).
// pre: sample n of Y = x_n w_n (n < p; conjugated input for the inverse), 0 up to L; mul: Y[y][k] *= bh[k]
// scale; post: out_k = w_k (sample k of Y) (conjugated for the inverse) times scale, k < p
void launch_blue_pre(const double2* src, int64_t src_stride, int lines_per_item, int64_t p, int64_t L, int lgA,
                     int lgB, const double2* chirp, double2* Y, int inverse, int64_t l0, int nl, cudaStream_t st);
void launch_blue_mul(double2* Y, const double2* bh, int64_t L, int nl, double scale, cudaStream_t st);
void launch_blue_post(const double2* Y, double2* dst, int64_t dst_stride, int lines_per_item, int64_t p, int64_t L,
                      int lgA, int lgB, const double2* chirp, int inverse, double scale, int64_t l0, int nl,
                      cudaStream_t st);
// the pointwise step of a chirp-z plan's row pass (update, residual, polarization; grid nblocks x items)
// and its Green operator when the row is the only logical axis
void launch_blue_point(const LatDev& dv, const RowArgs& a, int nblocks, int n_items, cudaStream_t st);
void launch_blue_green(const LatDev& dv, const RowArgs& a, int n_items, cudaStream_t st);
// in place: binary64 strain -> double-float pairs (to_df = 1) or back (0), all items
void launch_eps_df(const ItemDev* items, int n_items, int n_c, int64_t m, int to_df, cudaStream_t st);
// restart of the increment form: glob->active = number of paused items, arrivals = 0
void launch_prep_restart(ItemScal* scal, GlobScal* glob, int n_items, cudaStream_t st);
// sets a WHILE node's condition to (glob->active > 0) from inside the graph
void launch_set_cond(const GlobScal* glob, unsigned long long cond, cudaStream_t st);
// binary64 -> binary32 copy of the spectrum (T and Nyquist planes) of every ITEM_ACTIVE item
void launch_spectrum_to_f32(const void* T64, const void* TN64, void* T32, void* TN32, int64_t t_elems,
                            int64_t tn_elems, int64_t t_stride, int64_t tn_stride, const ItemScal* scal,
                            int n_items, cudaStream_t st);

static_assert(sizeof(ItemScal) <= 256, "the device scalars of an item fill one 256-byte slot");
