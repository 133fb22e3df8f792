/*
 * lattice_ms.h -- C ABI of the GB300 lattice Basic Scheme library (liblatms.so).
 *
 * FFT-based elastic homogenization on an arbitrary sampling lattice: the
 * generalized Moulinec-Suquet Basic Scheme of Bergmann & Merkert,
 * "A framework for FFT-based homogenization on anisotropic lattices"
 * (arXiv 1605.05712), Sec. 3.2, Algorithm 1, on the pattern P(M) of a regular
 * integer matrix M (Sec. 2.1) with the pattern FFT of Sec. 2.2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: LAT_OK (0) on success, a positive LAT_* outcome for a
 *    solve that ran but did not meet the tolerance (outputs still written),
 *    a negative LAT_ERR_* code on error.  lattice_last_error() returns a
 *    thread-local message for the last failing call.
 *  - Ownership: the library allocates device memory only inside
 *    lattice_plan() (twiddle tables on the device current at that call, freed
 *    by lattice_plan_destroy()).  Every field buffer and the workspace belong
 *    to the caller; solves never allocate.  A plan's solves must run with its
 *    device current (LAT_ERR_ARG otherwise); a plan made on a machine without
 *    a CUDA device is host-only (points, frequencies, gather maps) and its
 *    solves return LAT_ERR_CUDA.
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary host memory.  `stream` is a cudaStream_t
 *    passed as void* (NULL = the legacy default stream).
 *  - Point order ("plan order"): every spatial field is an array over the m
 *    pattern points in the order reported by lattice_points().  The paper
 *    leaves the ordering free (Sec. 2.2, after Eq. FourierTransform); this
 *    library uses the storage order of its FFT (a permutation of the
 *    lexicographic lambda order when the largest elementary divisor is split
 *    for the four-step FFT).  Spectral data is in the order reported by
 *    lattice_freqs().
 *  - Tensor components: symmetric d x d tensors are stored as n_c = d(d+1)/2
 *    planes of m values ("SoA"), components ordered (11, 22, 12) for d = 2
 *    and (11, 22, 33, 23, 13, 12) for d = 3, as tensor (not engineering)
 *    components.  Stiffness matrices are 6 x 6 Voigt matrices acting on
 *    engineering strain; d = 2 is plane strain and uses the (11, 22, 12)
 *    block.
 */
#ifndef LATTICE_MS_H
#define LATTICE_MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* outcomes (>= 0) */
#define LAT_OK               0
#define LAT_NOT_CONVERGED    1   /* maxit reached with r >= tol; outputs hold the last iterate */
#define LAT_DIVERGED         2   /* the residual became non-finite, or grew for LAT_DIVERGE_STEPS
                                    consecutive iterations to above 1 (the increment larger than the
                                    start strain itself); outputs hold the last iterate */
#define LAT_DIVERGE_STEPS   16
/* errors (< 0) */
#define LAT_ERR_ARG         -1   /* NULL pointer, bad count, bad option */
#define LAT_ERR_SINGULAR    -2   /* det M == 0 */
#define LAT_ERR_DIM         -3   /* d not in {2, 3} */
#define LAT_ERR_SIZE        -4   /* m or an entry too large, workspace too small */
#define LAT_ERR_UNSUPPORTED -5   /* a divisor structure this build cannot transform */
#define LAT_ERR_CUDA        -6   /* a CUDA runtime call failed (message has the CUDA error) */

/* precision of a solve */
#define LAT_FP64   0   /* every step in IEEE binary64 */
#define LAT_MIXED  1   /* binary32 FFT / Green operator / polarization; binary64 strain,
                          residual, averages and convergence test */
#define LAT_DF64   2   /* binary64-accurate: every step on double-float pairs (hi + lo of two
                          binary32, about 48 bits) on the binary32 pipes; residual, averages and
                          convergence test in binary64.  Agrees with LAT_FP64 to ~1e-13; faster
                          where binary64 issues at a small fraction of the binary32 rate */

/* iteration (lat_solve_opts.scheme) */
#define LAT_SCHEME_BASIC 0
#define LAT_SCHEME_EYRE_MILTON 1
#define LAT_SCHEME_CG 2
/* OR into the precision argument of lattice_workspace_bytes, lattice_batch_workspace_bytes and
   lattice_multi_workspace_bytes to size the workspace of a LAT_SCHEME_CG solve (four more
   strain-sized vectors per load case) */
#define LAT_WS_CG 256

/* treatment of boundary frequencies of the symmetric cell (k with h(-k) != -h(k)) */
#define LAT_BOUNDARY_AVERAGE 0  /* Gamma0 averaged over h(k) and -h(-k): the real part of the
                                   paper's complex update (default) */
#define LAT_BOUNDARY_ZERO    1  /* those frequencies set to zero */

typedef struct lat_plan lat_plan;

/*
 * lattice_plan -- build the plan for the pattern P(M).
 *   M    host, d*d int64, row-major, det M != 0.
 *   d    2 or 3.
 *   out  receives the plan (caller frees with lattice_plan_destroy).
 * Computes the Smith normal form M = Q E R (Sec. 2.2), the pattern
 * dimension d_M, the FFT decomposition over the elementary divisors and
 * uploads twiddle tables to the current device (the plan's device; without a
 * CUDA device the plan is host-only).
 * Every regular M within the size limits below is planned: divisors that are
 * powers of two take radix-4/2 kernels with bit-reversed spectra; any other
 * divisor takes mixed-radix kernels (radix 4, 2, 3, 5 and a direct p-point
 * DFT for other primes) in natural order, with the full complex spectrum.
 * Those "general" plans run every scheme and precision the power-of-two
 * plans run and take strain buffers aligned to 8 bytes.  A largest divisor
 * longer than one pass (2048 points in 2-D, 1024 in 3-D) is split four-step
 * into two passes; when
 * no such split exists (a large prime factor) its rows are transformed by
 * Bluestein's chirp-z convolution (lattice_plan_layout reports split = 2):
 * Algorithm 1, the Eyre-Milton scheme and conjugate gradients, in LAT_FP64
 * only (LAT_DF64 and LAT_MIXED return LAT_ERR_UNSUPPORTED), and lattice_fft
 * then needs lattice_fft_workspace_bytes.
 * Errors: LAT_ERR_DIM, LAT_ERR_SINGULAR, LAT_ERR_SIZE (m > 2^28 or entries
 * beyond the exact int64 range), LAT_ERR_UNSUPPORTED (no decomposition fits:
 * a divisor other than the largest longer than one pass -- 2048 points in
 * 2-D, 1024 in 3-D, e.g. diag(4096, 4096) --, or a largest divisor that needs
 * more than two passes and is not a chirp-z row of at most 2^22 points, e.g.
 * rank-1 lattices of 2^24 points in 2-D or 2^22 in 3-D), LAT_ERR_CUDA.
 */
int lattice_plan(const int64_t* M, int d, lat_plan** out);

/* Free a plan and its device tables.  NULL is ignored. */
void lattice_plan_destroy(lat_plan* plan);

/*
 * lattice_plan_set_cell -- the transformed pattern P_L(M) = L Lambda(M) cap L [-1/2, 1/2)^d of
 * Sec. 3.3 (Def. 3.3): the microstructure lives in the cell L [-1/2, 1/2)^d, the pattern point y of
 * lattice_points sits at x = L y, and the Fourier index h stands for the physical frequency L^{-T} h,
 * where the Green operator is evaluated (the transform over the index sets is unchanged).  Phase
 * fields are to be sampled at x = L y.  Strains and stresses are Cartesian components in the x frame.
 *   L  host, d*d row-major, regular; NULL restores the unit cube.
 * Returns LAT_ERR_ARG for non-finite entries, LAT_ERR_SINGULAR for a singular L.  Applies to solves
 * started after the call (not to lattice_fft, which has no Green operator).
 */
int lattice_plan_set_cell(lat_plan* plan, const double* L);

/*
 * lattice_gather_map -- subsampling and rearrangement between patterns.  For M = J N (J integral),
 * Lambda(N) is a sublattice of Lambda(M) and P(N) a subpattern of P(M) (Sec. 2.1); for
 * pattern-congruent matrices (P(M1) = P(M2), e.g. M2 = Q M1 with Q unimodular, Sec. 2.2) the two
 * point sets coincide and only the order differs.  map (host, to->m int32) receives, for every point
 * of `to` in its plan order, the plan-order slot of the same point in `from`.  Host computation
 * (exact integer matching of the point numerators); O(from->m) memory.
 * Returns LAT_ERR_ARG if a point of P(to) is not in P(from) (or the dimensions differ),
 * LAT_ERR_SIZE if from->m >= 2^31.
 */
int lattice_gather_map(const lat_plan* from, const lat_plan* to, int32_t* map);

/*
 * lattice_gather -- out[f][s] = in[f][map[s]] for s < n_out and f < n_fields (device): samples
 * fields given on P(from) onto P(to) with a map of lattice_gather_map (copied to the device by the
 * caller).  elem_bytes 1 (phase ids), 2, 4, 8 (binary64) or 16; in_plane / out_plane are the plane
 * strides in elements.  Buffers aligned to the element size; in and out must not overlap.
 * Asynchronous on `stream`.
 */
int lattice_gather(const void* in, void* out, const int32_t* map, int64_t n_out, int elem_bytes,
                   int n_fields, int64_t in_plane, int64_t out_plane, void* stream);

/*
 * lattice_plan_info -- m = |det M|, d_M = #{e_j > 1} and the d elementary
 * divisors e_1 | e_2 | ... (Sec. 2.2).  Any output pointer may be NULL.
 */
int lattice_plan_info(const lat_plan* plan, int64_t* m, int* d_M, int64_t* divisors);

/*
 * lattice_points -- the pattern P(M) in plan order (Sec. 2.1): p is host,
 * m*d int64, point i is y_i = p[i*d .. i*d+d-1] / m, every coordinate in
 * [-1/2, 1/2).  (m y is integral because m M^{-1} = +-adj M.)
 */
int lattice_points(const lat_plan* plan, int64_t* p);

/*
 * lattice_freqs -- the generating set G(M^T) in spectral order (Sec. 2.1):
 * h is host, m*d int64, M^{-T} h in [-1/2, 1/2)^d.
 */
int lattice_freqs(const lat_plan* plan, int64_t* h);

/* Thread-local description of the last error (never NULL). */
const char* lattice_last_error(void);

/*
 * lattice_fft -- the Fourier transform on the pattern, Eq. (Fouriermatrix):
 * forward  a_hat = F(M) a      (carries the 1/m),
 * inverse  a     = F(M)^{-1} a_hat (no scaling).
 *   in, out   device, n_fields * m complex binary64, interleaved (re, im);
 *             forward: in is in plan order and out in spectral order;
 *             inverse: the reverse.  in and out must not overlap.
 *   workspace device, at least lattice_fft_workspace_bytes(plan, n_fields).
 * Asynchronous on `stream`.
 */
size_t lattice_fft_workspace_bytes(const lat_plan* plan, int n_fields);
int lattice_fft(const lat_plan* plan, const double* in, double* out, int n_fields,
                int inverse, void* workspace, size_t workspace_bytes, void* stream);

typedef struct lat_solve_opts {
  int precision;        /* LAT_FP64, LAT_MIXED or LAT_DF64 */
  int boundary;         /* LAT_BOUNDARY_AVERAGE or LAT_BOUNDARY_ZERO */
  int warm_start;       /* 0: eps^(0) = E (Algorithm 1); 1: eps holds eps^(0) on entry */
  double* resid_history;/* host or NULL: n_loads * maxit residuals r_0, r_1, ... (rest untouched) */
  int mixed_increment;  /* LAT_MIXED only: 1 = binary32 kernels carry the increment
                           eps^(n+1) - eps^(n) (accumulated into the strain, which the solve holds
                           as double-float pairs), 0 = they carry the strain itself */
  int mixed_restart;    /* LAT_MIXED increment form: 0 (default) = when an item's residual first
                           falls below sqrt(tol), one binary64-accurate iteration (double-float
                           pairs, as LAT_DF64) restarts the increment recurrence; binary32
                           rounding otherwise stays in the fixed point as an offset of up to
                           1/(1 - rate) times the accumulated rounding.  Negative = no restart.
                           The restart counts as an iteration. */
  int plain_launches;   /* 0: the iteration is a CUDA-graph WHILE loop (one replay per solve);
                           nonzero: plain kernel launches with a host read of the convergence
                           state after every iteration, same results (for profilers that do not
                           trace kernels inside graphs with conditional nodes) */
  int scheme;           /* LAT_SCHEME_BASIC (0, Algorithm 1) or LAT_SCHEME_EYRE_MILTON (1):
                           the accelerated iteration u = (C + C0) eps <- (I - 2 C0 Gamma0)
                           (C - C0) eps, <u> = <(C - C0) eps> + 2 C0 E (Sec. 6 notes that such
                           schemes carry over to patterns).  Same discrete solution as Algorithm 1
                           at the same C0, converging for any positive C0, fastest at the
                           geometric mean of the phase extremes (rate (sqrt(k)-1)/(sqrt(k)+1)
                           against (k-1)/(k+1)).  Not with LAT_BOUNDARY_ZERO.
                           LAT_SCHEME_CG (2): conjugate gradients on the same discrete equation
                           (Sec. 6; the paper cites Zeman et al. 2010) in the inner product
                           sum_y a : C0 : c, where Gamma0 C is self-adjoint and positive on the
                           compatible zero-mean fields.  Its residual r = -Gamma0 : sigma(eps) is
                           Algorithm 1's increment, so tol means the same; one iteration is one
                           forward and one inverse transform.  The solution does not depend on C0;
                           iterations grow with the square root of the contrast.  LAT_FP64 or
                           LAT_DF64 only, cold start only, and LAT_BOUNDARY_ZERO on lattices with an
                           even largest divisor (there Gamma0 C0 is a projector only with the
                           boundary frequencies zeroed); LAT_ERR_ARG otherwise.  The workspace
                           query takes LAT_WS_CG. */
} lat_solve_opts;

/*
 * lattice_workspace_bytes -- device workspace a solve with n_loads load
 * cases needs (spectrum buffers, reduction partials, device scalars).
 * Returns 0 for invalid arguments or when a row or column tile of the plan
 * does not fit in shared memory at this precision (the solve would return
 * LAT_ERR_UNSUPPORTED); the same holds for the batch and multi variants.
 */
size_t lattice_workspace_bytes(const lat_plan* plan, int n_loads, int precision);

/*
 * basic_scheme_solve -- Algorithm 1 (Sec. 3.2) for n_loads macroscopic strains:
 *   eps^(0) = E; repeat  tau = (C_y - C0) : eps_y ;  tau_hat = F(M) tau ;
 *   eps_hat_h = -Gamma0(h) : tau_hat_h (h != 0), eps_hat_0 = E ;
 *   eps = F(M)^{-1} eps_hat  until r_n < tol or n = maxit,
 * with the Cauchy residual of Sec. 5.2, r_n = ||eps^(n+1) - eps^(n)|| /
 * (sqrt(m) ||E||_F) (l2 over points of the Frobenius norm; 1 replaces the
 * denominator when E = 0), then sigma_y = C_y : eps_y and its mean
 * sigma_bar = C^eff : E (Sec. 3.1).  Gamma0 is the isotropic closed form
 * evaluated at the integer frequency h in G(M^T).
 *   phase      device, m uint8, phase id per point in plan order (< n_phases).
 *   n_phases   1..256.
 *   stiffness  host, n_phases * 36 binary64: 6x6 Voigt matrix per phase (row-major).
 *   C0         host, {lambda0, mu0}: isotropic reference medium (mu0 > 0, lambda0 + 2 mu0 > 0).
 *   E          host, n_loads * n_c binary64 tensor components.
 *   tol, maxit Cauchy threshold and iteration cap (maxit >= 0).
 *   opts       may be NULL (= FP64, average, cold start, no history).
 *   eps        device, n_loads * n_c * m binary64 (output; input too for a warm start).
 *   sigma      device or NULL, n_loads * n_c * m binary64: the stress field.
 *   sigma_bar  host or NULL, n_loads * n_c: mean stress per load case.
 *   iters      host or NULL, n_loads: iterations performed.
 *   resid      host or NULL, n_loads: last residual r.
 *   workspace  device, >= lattice_workspace_bytes(plan, n_loads, precision).
 * Runs on `stream` and returns after synchronizing it (host outputs valid).
 * The load cases are solved together (one batch, see basic_scheme_solve_batch);
 * each stops on its own residual.  Residual histories keep at most 4096
 * entries per load case.  Returns LAT_OK when every load case met tol, else
 * the worst outcome.
 */
int basic_scheme_solve(const lat_plan* plan, const uint8_t* phase, int n_phases,
                       const double* stiffness, const double* C0,
                       const double* E, int n_loads, double tol, int maxit,
                       const lat_solve_opts* opts,
                       double* eps, double* sigma, double* sigma_bar,
                       int* iters, double* resid,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * basic_scheme_solve_async -- basic_scheme_solve (Algorithm 1, Sec. 3.2) without the final host
 * synchronization: everything is enqueued on `stream` (the iteration is the CUDA-graph loop) and the
 * call returns at once; the scalar results are written to device memory at the end of the solve.
 *   sigma_bar_d  device or NULL, n_loads x n_c binary64: mean stress per load case
 *   iters_d      device or NULL, n_loads int32: iterations performed
 *   resid_d      device or NULL, n_loads binary64: last Cauchy residual
 *   status_d     device or NULL, n_loads int32: LAT_OK, LAT_NOT_CONVERGED or LAT_DIVERGED per load case
 * Other arguments as for basic_scheme_solve; opts->resid_history must be NULL and plain_launches 0
 * (LAT_ERR_ARG otherwise).  phase, eps, sigma, the workspace and the result arrays must stay valid
 * until the stream has passed the solve.  Host-side argument errors are returned before anything is
 * enqueued; the return value is LAT_OK once the solve is enqueued (its outcome is in status_d).
 */
int basic_scheme_solve_async(const lat_plan* plan, const uint8_t* phase, int n_phases,
                             const double* stiffness, const double* C0,
                             const double* E, int n_loads, double tol, int maxit,
                             const lat_solve_opts* opts, double* eps, double* sigma,
                             double* sigma_bar_d, int* iters_d, double* resid_d, int* status_d,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * basic_scheme_solve_field -- Algorithm 1 (Sec. 3.2) with a per-point stiffness field C(y) instead of
 * phases (Sec. 3.1: the Lippmann-Schwinger equation holds for any field C(x); the polarization is
 * tau_y = C_y : eps_y - C0 : eps_y):
 *   voigt   device, 21 x m binary64, 16-byte aligned: plane p holds entry p of the row-major upper
 *           triangle of each point's 6x6 Voigt matrix ((0,0), (0,1), ..., (0,5), (1,1), ..., (5,5);
 *           Voigt order 11, 22, 33, 23, 13, 12 on engineering strain) in plan order; d = 2 reads the
 *           plane-strain block (11, 22, 12).  Read-only; shared by all load cases.
 *   workspace  device, >= lattice_field_workspace_bytes(plan, n_loads, precision) (it also holds the
 *           binary32 / pair copies of the field the LAT_MIXED and LAT_DF64 kernels read)
 * Other arguments and outputs as for basic_scheme_solve.  Algorithm 1 only (opts->scheme must be
 * LAT_SCHEME_BASIC: LAT_ERR_ARG otherwise).  Per iteration the kernels read the field (168 bytes per
 * point in binary64, 84 in binary32) where the phase form reads one byte.
 */
size_t lattice_field_workspace_bytes(const lat_plan* plan, int n_loads, int precision);
int basic_scheme_solve_field(const lat_plan* plan, const double* voigt, const double* C0,
                             const double* E, int n_loads, double tol, int maxit,
                             const lat_solve_opts* opts, double* eps, double* sigma,
                             double* sigma_bar, int* iters, double* resid,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * Batches of independent microstructures on one lattice (shared plan): each
 * item has its own phase field, material, reference medium, macroscopic
 * strain and outputs, and stops on its own residual.  All items run in the
 * same kernel launches (one CUDA-graph loop); finished items drop out.
 */
#define LAT_BATCH_MAX_PHASES 16
typedef struct lat_batch_item {
  const uint8_t* phase;     /* device, m phase ids in plan order (< n_phases) */
  int n_phases;             /* 1..LAT_BATCH_MAX_PHASES */
  const double* stiffness;  /* host, n_phases * 36: 6x6 Voigt matrix per phase */
  double C0[2];             /* isotropic reference medium (lambda0, mu0) */
  const double* E;          /* host, n_c tensor components */
  double* eps;              /* device, n_c * m (output) */
  double* sigma;            /* device or NULL, n_c * m */
} lat_batch_item;

/* workspace of basic_scheme_solve_batch for n_items items */
size_t lattice_batch_workspace_bytes(const lat_plan* plan, int n_items, int precision);

/*
 * basic_scheme_solve_batch -- Algorithm 1 (Sec. 3.2) for n_items independent
 * problems sharing the lattice of `plan`; per item as basic_scheme_solve with
 * one load case.  Host outputs are n_items (x n_c) arrays.  Returns the worst
 * outcome over the items.
 */
int basic_scheme_solve_batch(const lat_plan* plan, const lat_batch_item* items, int n_items,
                             double tol, int maxit, const lat_solve_opts* opts,
                             double* sigma_bar, int* iters, double* resid,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * basic_scheme_solve_multi -- Algorithm 1 (Sec. 3.2) for independent problems
 * on different lattices (any mix of d, M and load-case counts) in one call.
 * Items that share a plan run as one batch (as basic_scheme_solve_batch, all
 * their load cases in the same kernel launches); the batches of different
 * plans run concurrently as the parallel branches of one CUDA graph, each with
 * its own WHILE loop, so small lattices do not wait for large ones.
 *   items      host array of n_items; per item:
 *     plan       the item's lattice (lattice_plan); items with the same pointer batch together
 *     phase      device, m phase ids in plan order (< n_phases)
 *     n_phases   1..LAT_BATCH_MAX_PHASES; stiffness host, n_phases * 36 Voigt
 *     C0         isotropic reference medium (lambda0, mu0), lambda0 + 2 mu0 > 0, mu0 > 0
 *     E, n_loads host, n_loads x n_c macroscopic strains (tensor components), n_loads >= 1
 *     eps        device, n_loads x n_c x m binary64, 16-byte aligned (8 bytes on plans with a divisor that
 *                is not a power of two) (output; input with warm_start)
 *     sigma      device or NULL, n_loads x n_c x m
 *     sigma_bar, iters, resid  host or NULL, n_loads (x n_c) outputs per item
 *   opts       as basic_scheme_solve; resid_history must be NULL (LAT_ERR_ARG otherwise)
 *   workspace  device, >= lattice_multi_workspace_bytes(items, n_items, precision), carved per plan
 *              in order of first appearance
 * Runs on `stream` and returns after synchronizing it.  Returns the worst outcome over all load
 * cases of all items; argument errors are reported before anything runs.
 */
typedef struct lat_multi_item {
  const lat_plan* plan;
  const uint8_t* phase;
  int n_phases;
  const double* stiffness;
  double C0[2];
  const double* E;
  int n_loads;
  double* eps;
  double* sigma;
  double* sigma_bar;
  int* iters;
  double* resid;
} lat_multi_item;
size_t lattice_multi_workspace_bytes(const lat_multi_item* items, int n_items, int precision);
int basic_scheme_solve_multi(const lat_multi_item* items, int n_items, double tol, int maxit,
                             const lat_solve_opts* opts, void* workspace, size_t workspace_bytes,
                             void* stream);

/*
 * basic_scheme_solve_noalloc -- basic_scheme_solve for callers that cannot
 * allocate device memory (the paper has no counterpart: this is a property of
 * the library, not of the method).  A serving loop with a fixed device-memory
 * budget, a runtime whose own allocator owns all device memory, or code that
 * must not allocate while it sets up work around a later stream capture cannot
 * call cudaMalloc for the workspace basic_scheme_solve wants.  This variant
 * takes no workspace and allocates nothing: its scratch is one static device
 * array of LAT_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which loads the
 * library holds until the process exits.  The caller still owns and passes the
 * inputs and outputs, with the meaning they have for basic_scheme_solve; the
 * twiddle tables are the plan's (lattice_plan made them).
 *  - Limit: returns LAT_ERR_SIZE (message gives the bytes needed) when the
 *    solve's workspace exceeds the array, e.g. binary64 m = 262144 in 2-D fits
 *    two load cases, not three.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and keeps it; concurrent first calls from several
 *    host threads are serialized.
 *  - Every call shares the one array; each call clears what it reads before
 *    use, but calls that overlap on the GPU (other streams or host threads)
 *    race on it.
 *  - The iteration uses plain kernel launches and reads the convergence flag
 *    back after every iteration (a stream synchronization) instead of a
 *    CUDA-graph loop; the results equal basic_scheme_solve's.  It must
 *    therefore not be called on a stream that is being captured: that returns
 *    LAT_ERR_ARG before anything is enqueued.
 */
#define LAT_NOALLOC_SCRATCH_BYTES (16u << 20)
int basic_scheme_solve_noalloc(const lat_plan* plan, const uint8_t* phase, int n_phases,
                               const double* stiffness, const double* C0,
                               const double* E, int n_loads, double tol, int maxit,
                               const lat_solve_opts* opts,
                               double* eps, double* sigma, double* sigma_bar,
                               int* iters, double* resid, void* stream);

/*
 * Learned warm start (not in the paper; an addition measured against the
 * plain scheme): a periodic 3-D U-Net, 4 levels x 32 channels, BF16 weights
 * and activations with FP32 accumulation, mapping the stiffness field of a
 * cubic n^3 tensor grid (M = diag(n, n, n), plan order = grid order) to the
 * strain-localization field A, eps^(0) = A : E with <A> = I, so that
 * basic_scheme_solve can start warm and run to the same tolerance.
 * Device buffers are the caller's:
 *   params  lat_wsnet_param_bytes(): fp32 parameters, gradients, Adam moments,
 *           bf16 copies of the convolution weights;
 *   work    lat_wsnet_work_bytes(n): activations and gradients of one n^3 sample
 *           (n in 16..256, divisible by 8).
 * Parameter vector (lat_wsnet_num_params floats): for each of the 7 convolutions
 * (c0 c1 c2 c3 d2 d1 d0) W[27][32][32] (taps (dz,dy,dx) lexicographic, ci, co)
 * then b[32]; then the 1x1 head H[32][36] and hb[36].
 * Feature table: per phase 21 floats, the upper triangle of its Voigt matrix / mu0.
 * Errors: LAT_ERR_SIZE / LAT_ERR_ARG for bad sizes or pointers, LAT_ERR_CUDA for
 * a failed launch or copy.  The tensor-core convolutions bound their waits on
 * their own products; one that ran out writes NaN outputs and raises a device
 * flag, which the calls that synchronize (get_params, get_activation,
 * train_step with loss_out) report as LAT_ERR_CUDA and clear.
 */
size_t lat_wsnet_param_bytes(void);
int64_t lat_wsnet_num_params(void);
size_t lat_wsnet_work_bytes(int n);
int lat_wsnet_set_params(void* params, const float* host_params, void* stream);      /* also resets Adam */
int lat_wsnet_get_params(const void* params, float* host_params, float* host_grads, void* stream);
int lat_wsnet_features(const uint8_t* phase, const float* table, int n, void* work, size_t work_bytes,
                       void* stream);
/* forward of the features in `work`; y_out (device, n^3 x 36 fp32, channel 6 i + j = A'_ij) or NULL */
int lat_wsnet_forward(const void* params, int n, float* y_out, void* work, size_t work_bytes, void* stream);
/* backward after lat_wsnet_forward on the same work: parameter gradients from dL/dy (device n^3 x 36) */
int lat_wsnet_backward(void* params, int n, const float* dy, void* work, size_t work_bytes, void* stream);
/* one Adam step on the centred relative squared error sum (y~ - t~)^2 / (sum t~^2 + N 1e-6), x~ = x minus
 * its spatial mean per channel (the prediction's mean is discarded when it is used), against the
 * localization t of the six unit load cases (loss_out: host, that ratio, before the step):
 * eps_unit device, 6 x 6 x n^3 binary64 (load case, component, point), as basic_scheme_solve writes */
int lat_wsnet_train_step(void* params, const uint8_t* phase, const float* table, const double* eps_unit,
                         int n, float lr, int step, double* loss_out, void* work, size_t work_bytes,
                         void* stream);
/* copy a forward activation of `work` to host fp32 (n_l^3 x 32, n_l = n >> level): which = 0 features,
 * 1..4 encoder outputs s0..s3, 5..7 pooled inputs p1..p3, 8/9 level-0 decoder input/output, 10/11
 * level 1, 12/13 level 2 (for inspecting and checking the network) */
int lat_wsnet_get_activation(const void* work, size_t work_bytes, int n, int which, float* host_out,
                             void* stream);
/* eps0 (device, n_loads x 6 x n^3 binary64) = E + (A' - <A'>) : E for n_loads macroscopic strains */
int lat_wsnet_predict(const void* params, const uint8_t* phase, const float* table, int n,
                      const double* E, int n_loads, double* eps0, void* work, size_t work_bytes,
                      void* stream);

/*
 * lattice_start_filter -- two-iteration filter of an initial strain (an
 * addition to the paper, used with the warm start): out = (G^2(eps0) -
 * rho^2 eps0) / (1 - rho^2), where G^2(eps0) is the iterate after two plain
 * iterations from eps0 (basic_scheme_solve with maxit = 2, tol = 0).  Since
 * G is affine with fixed point eps*, the error of out is p(T) (eps0 - eps*)
 * with T the linear part of G and p(t) = (t^2 - rho^2) / (1 - rho^2): the
 * solution is kept (p(1) = 1) and the error components of eigenvalue +-rho,
 * the slowest ones, are removed.  For phases whose stiffness is a multiple
 * c_p C0 of the reference, rho = max_p |c_p - 1| and those components are
 * the compatible strains confined to one phase; the exact solution has none
 * (equilibrium in each phase), a predicted start in general has.
 *   out, eps_g2, eps0  device, count binary64 each; out may alias either input.
 *   rho               in [0, 1).
 * Returns LAT_ERR_ARG for NULL pointers or rho outside [0, 1); asynchronous.
 */
int lattice_start_filter(double* out, const double* eps_g2, const double* eps0, double rho, size_t count,
                         void* stream);

/*
 * lattice_autotune -- pick the launch shapes of a solve on this plan by timing them on the device
 * (not in the paper): the rows per block of the row pass and the tile width of every column pass,
 * one kernel at a time, each candidate over 5 iterations of a homogeneous test problem with n_items
 * items (load cases x problems).  The fastest are kept in the plan for solves of this precision
 * whose item count falls in the same power-of-two bucket (1, 2-3, 4-7, ..., >= 128); they change
 * how lines are grouped into blocks, never the arithmetic of a line, so the fields are the same.
 *   workspace  device, >= lattice_autotune_workspace_bytes(plan, n_items, precision)
 * Synchronizes `stream`.  Not thread-safe with solves on the same plan.
 */
size_t lattice_autotune_workspace_bytes(const lat_plan* plan, int n_items, int precision);
int lattice_autotune(lat_plan* plan, int n_items, int precision, void* workspace, size_t workspace_bytes,
                     void* stream);
/* the tuned shapes of a bucket: returns 1 and fills rpc, w[n_groups] and ms[1 + n_groups] (device
 * times of the row pass and of each column group) if the bucket is tuned, else 0; n_groups is always
 * set (w and ms need 3 and 4 entries: a plan has at most 3 column groups) */
int lattice_tune_info(const lat_plan* plan, int n_items, int precision, int* rpc, int* w, float* ms,
                      int* n_groups);

/*
 * lattice_pass_times -- profiling helper: average device time of each kernel
 * of one Basic Scheme iteration (no counterpart in the paper; it measures
 * the passes the solve above runs inside its CUDA graph).  Runs the
 * prologue once and then n_reps iterations of the n_loads load cases as one
 * batch (the launches basic_scheme_solve makes: every kernel covers all load
 * cases) with plain launches, a CUDA event pair around every launch on
 * `stream`.  Arguments as for basic_scheme_solve (E holds n_loads x n_c
 * values; eps, n_loads x n_c x m, is overwritten).
 *   ms_out  host, >= 8 floats: [0] row pass, [1..] column passes in
 *           launch order (forward mid groups, Gamma group, inverse mid groups),
 *           unused entries set to 0.
 *   n_out   receives the number of kernels per iteration.
 */
int lattice_pass_times(const lat_plan* plan, const uint8_t* phase, int n_phases,
                       const double* stiffness, const double* C0, const double* E, int n_loads,
                       int precision, int n_reps, double* eps,
                       void* workspace, size_t workspace_bytes, void* stream,
                       float* ms_out, int* n_out);

/*
 * lattice_plan_layout -- the FFT decomposition a plan chose for the pattern
 * DFT of Sec. 2.2 (its d_M-dimensional DFT over the elementary divisors),
 * for cost models and profiling (no counterpart in the paper).
 *   nax        number of logical axes in storage order; the last one is the
 *              contiguous row (a divisor axis may be split four-step into
 *              two logical axes).
 *   ax_len     host, >= 6 ints: their lengths.
 *   ngroups    column passes per transform direction: group g covers the
 *              logical axes [grp[2g], grp[2g+1]) (host, >= 6 ints); group 0
 *              also applies the Green operator.
 *   split      1 if the largest divisor is split four-step; 2 if the row (the
 *              largest divisor, not split) is transformed by Bluestein's
 *              chirp-z convolution (general plans whose largest divisor has no
 *              split into two lines of at most 2048 points in 2-D, 1024 in 3-D).
 * Any output pointer may be NULL.
 */
int lattice_plan_layout(const lat_plan* plan, int* nax, int* ax_len, int* ngroups, int* grp, int* split);

#ifdef __cplusplus
}
#endif
#endif /* LATTICE_MS_H */
