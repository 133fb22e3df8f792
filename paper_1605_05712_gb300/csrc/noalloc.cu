// noalloc.cu -- basic_scheme_solve_noalloc: the Basic Scheme solve for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being captured into a
// CUDA graph, code inside a serving loop with a fixed memory budget, or host runtimes whose
// allocator owns all device memory.  For them this entry point takes no workspace argument and
// allocates nothing.  Its scratch memory (spectrum buffers, reduction partials, device scalars,
// material and twiddle tables) lives in one file-scope static __device__ array of
// LAT_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until the process exits.
//
// Host code may not pass the array's name to a kernel: in host code that name is a host-side
// stand-in, not a device address.  The first call on each device therefore asks the runtime for
// the device address with cudaGetSymbolAddress (with that device current) and keeps it; that first
// call should come before any stream capture.  Every call shares the one array and leaves its
// contents behind, so each call clears the device scalars it reads before use, and calls that
// overlap on the GPU (two streams, two host threads) race on the array.
//
// The iteration runs with plain launches instead of the CUDA graph of basic_scheme_solve (a graph
// is not instantiated here); after each iteration the convergence flag is read back.  The kernels
// and their arithmetic are the same, so the results equal basic_scheme_solve's.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "solve_detail.h"

using namespace latms_detail;

static __device__ __align__(256) unsigned char g_lat_scratch[LAT_NOALLOC_SCRATCH_BYTES];

namespace {

const int kMaxDev = 64;
void* g_scratch_ptr[kMaxDev] = {nullptr};

#define CK_NA(x)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// device address of the static scratch on the current device (set up once per device)
int scratch_ptr(char** out) {
  int dev = 0;
  CK_NA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: device index >= 64");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    CK_NA(cudaGetSymbolAddress(&p, g_lat_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = (char*)g_scratch_ptr[dev];
  return LAT_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int basic_scheme_solve_noalloc(const lat_plan* P, const uint8_t* phase, int n_phases,
                                          const double* stiffness, const double* C0, const double* E, int n_loads,
                                          double tol, int maxit, const lat_solve_opts* opts, double* eps,
                                          double* sigma, double* sigma_bar, int* iters, double* resid,
                                          void* stream) {
  if (!P || !phase || !stiffness || !C0 || !E || !eps)
    return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: NULL argument");
  if (n_phases < 1 || n_phases > kMaxPhases) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: n_phases not in 1..256");
  if (n_loads < 1 || maxit < 0 || !(tol >= 0)) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: bad n_loads/maxit/tol");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precision != LAT_FP64 && o.precision != LAT_MIXED) return lat_fail(LAT_ERR_ARG, "bad precision");
  if (o.boundary != LAT_BOUNDARY_AVERAGE && o.boundary != LAT_BOUNDARY_ZERO) return lat_fail(LAT_ERR_ARG, "bad boundary");
  const double lam0 = C0[0], mu0 = C0[1];
  if (!(mu0 > 0) || !(lam0 + 2 * mu0 > 0)) return lat_fail(LAT_ERR_ARG, "C0 must have mu0 > 0 and lam0 + 2 mu0 > 0");
  if (((uintptr_t)eps & 15) != 0) return lat_fail(LAT_ERR_ARG, "eps must be 16-byte aligned");
  const bool fp32 = (o.precision == LAT_MIXED);
  // scratch layout: [solve workspace | twiddle table | split twiddle table]
  const Work wl = layout(P, n_loads, o.precision);
  int64_t n_tw = 0, n_stw = 0;
  if (P->nax > 0) lat_host_twiddles(P, fp32, nullptr, nullptr, &n_tw, &n_stw);
  const size_t es = fp32 ? sizeof(float2) : sizeof(double2);
  const size_t off_tw = up256(wl.total), off_stw = up256(off_tw + n_tw * es);
  const size_t need = up256(off_stw + n_stw * es);
  if (need > (size_t)LAT_NOALLOC_SCRATCH_BYTES)
    return lat_fail(LAT_ERR_SIZE, "basic_scheme_solve_noalloc: this solve needs " + std::to_string(need) +
                                      " bytes of scratch, more than the static " +
                                      std::to_string((size_t)LAT_NOALLOC_SCRATCH_BYTES) +
                                      " (use basic_scheme_solve with a caller-allocated workspace)");
  char* ws = nullptr;
  if (int rc = scratch_ptr(&ws)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  cudaStream_t st = (cudaStream_t)stream;
  const int d = P->d, n_c = d * (d + 1) / 2;
  const int64_t m = P->m;

  // tables: material (C_p - C0 and C_p in tensor-component form) and this plan's twiddles
  std::vector<double> D(n_phases * n_c * n_c), Cc(n_phases * n_c * n_c);
  double C0v[36];
  memset(C0v, 0, sizeof(C0v));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C0v[i * 6 + j] = lam0;
    C0v[i * 6 + i] = lam0 + 2 * mu0;
    C0v[(i + 3) * 6 + (i + 3)] = mu0;
  }
  double c0tc[36];
  voigt_to_tc(C0v, d, c0tc);
  for (int p = 0; p < n_phases; ++p) {
    voigt_to_tc(stiffness + 36 * p, d, &Cc[p * n_c * n_c]);
    for (int k = 0; k < n_c * n_c; ++k) D[p * n_c * n_c + k] = Cc[p * n_c * n_c + k] - c0tc[k];
  }
  CK_NA(cudaMemcpyAsync(ws + wl.Dtab, D.data(), D.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CK_NA(cudaMemcpyAsync(ws + wl.Ctab, Cc.data(), Cc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<char> htw(n_tw * es), hstw(n_stw * es);
  if (P->nax > 0) {
    lat_host_twiddles(P, fp32, htw.data(), hstw.data(), nullptr, nullptr);
    CK_NA(cudaMemcpyAsync(ws + off_tw, htw.data(), htw.size(), cudaMemcpyHostToDevice, st));
    if (n_stw) CK_NA(cudaMemcpyAsync(ws + off_stw, hstw.data(), hstw.size(), cudaMemcpyHostToDevice, st));
  }
  // the scalars left by an earlier call must start from zero
  CK_NA(cudaMemsetAsync(ws + wl.scal, 0, (size_t)n_loads * kScalBytes, st));

  LatDev dv = make_dev(P, fp32);
  dv.tw = ws + off_tw;
  dv.stw = ws + off_stw;
  Geometry geo;
  memset(&geo, 0, sizeof(geo));
  if (P->nax > 0) {
    int rc = geometry(P, n_c, fp32 ? 8 : 16, P->Rh, true, geo);
    if (rc != LAT_OK) return rc;
  }
  const int eff_blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (m + 255) / 256));
  for (int lc = 0; lc < n_loads; ++lc) {
    char* sc = ws + wl.scal + (size_t)lc * kScalBytes;
    double* eps_lc = eps + (size_t)lc * n_c * m;
    const double* E_lc = E + (size_t)lc * n_c;
    double nE2 = 0;
    for (int c = 0; c < n_c; ++c) nE2 += (c >= d ? 2.0 : 1.0) * E_lc[c] * E_lc[c];
    const double norm0 = nE2 > 0 ? sqrt((double)m * nE2) : 1.0;
    if (!o.warm_start) launch_fill(eps_lc, n_c, m, E_lc, st);
    CK_NA(cudaGetLastError());
    if (P->nax > 0 && maxit > 0) {
      RowArgs ra;
      memset(&ra, 0, sizeof(ra));
      ra.rpc = geo.rpc;
      ra.eps = eps_lc;
      ra.phase = phase;
      ra.T = ws + wl.T + lc * wl.t_per_lc;
      ra.TN = ws + wl.TN + lc * wl.tn_per_lc;
      ra.mat.Dtab = (const double*)(ws + wl.Dtab);
      for (int c = 0; c < 6; ++c) ra.mat.E[c] = c < n_c ? E_lc[c] : 0.0;
      ra.mat.lam0 = lam0;
      ra.mat.mu0 = mu0;
      ra.mat.c1 = 0.5 / mu0;
      ra.mat.c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
      ra.mat.gscale = -1.0 / (double)m;
      ra.mat.boundary_zero = o.boundary == LAT_BOUNDARY_ZERO;
      ra.it.partials = (double*)(ws + wl.partials);
      ra.it.counter = (unsigned*)(sc + 0);
      ra.it.done = (int*)(sc + 4);
      ra.it.iter = (int*)(sc + 8);
      ra.it.last_r = (double*)(sc + 16);
      ra.it.hist = (double*)(ws + wl.hist) + (size_t)lc * LAT_HIST_CAP;
      ra.it.norm0 = norm0;
      ra.it.tol = tol;
      ra.it.maxit = maxit;
      ra.it.cond = 0;  // no graph: the kernel only raises the done flag
      ColArgs ca;
      memset(&ca, 0, sizeof(ca));
      ca.row_slots = P->Rh;
      ca.has_nyq = 1;
      ca.n_f = n_c;
      ca.T = ra.T;
      ca.TN = ra.TN;
      ca.scale = 1.0;
      ca.mat = ra.mat;
      const bool gamma_in_row = (P->nax == 1);
      RowArgs first = ra;
      first.flags = ROW_LOAD_EPS | (gamma_in_row ? ROW_GAMMA : 0);
      RowArgs full = ra;
      full.flags = ROW_UPDATE | (gamma_in_row ? ROW_GAMMA : 0);
      ColArgs c0 = ca;
      c0.done = nullptr;
      ca.done = ra.it.done;
      if (fp32) {
        launch_row_pass<float>(dv, first, geo.row_blocks, kThreads, geo.row_smem, st);
        enqueue_columns<float>(dv, P, geo, c0, st);
      } else {
        launch_row_pass<double>(dv, first, geo.row_blocks, kThreads, geo.row_smem, st);
        enqueue_columns<double>(dv, P, geo, c0, st);
      }
      CK_NA(cudaGetLastError());
      for (int n = 0; n < maxit; ++n) {
        if (fp32) {
          launch_row_pass<float>(dv, full, geo.row_blocks, kThreads, geo.row_smem, st);
          enqueue_columns<float>(dv, P, geo, ca, st);
        } else {
          launch_row_pass<double>(dv, full, geo.row_blocks, kThreads, geo.row_smem, st);
          enqueue_columns<double>(dv, P, geo, ca, st);
        }
        CK_NA(cudaGetLastError());
        int done = 0;
        CK_NA(cudaMemcpyAsync(&done, ra.it.done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK_NA(cudaStreamSynchronize(st));
        if (done) break;
      }
    }
    EffArgs ea;
    ea.eps = eps_lc;
    ea.sigma = sigma ? sigma + (size_t)lc * n_c * m : nullptr;
    ea.phase = phase;
    ea.Ctab = (const double*)(ws + wl.Ctab);
    ea.partials = (double*)(ws + wl.partials);
    ea.counter = (unsigned*)(sc + 24);
    ea.sigma_bar = (double*)(sc + 32);
    launch_eff(dv, ea, eff_blocks, st);
    CK_NA(cudaGetLastError());
  }
  std::vector<char> scal((size_t)n_loads * kScalBytes);
  CK_NA(cudaMemcpyAsync(scal.data(), ws + wl.scal, scal.size(), cudaMemcpyDeviceToHost, st));
  std::vector<double> hist;
  if (o.resid_history && maxit > 0) {
    hist.resize((size_t)n_loads * LAT_HIST_CAP);
    CK_NA(cudaMemcpyAsync(hist.data(), ws + wl.hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK_NA(cudaStreamSynchronize(st));
  int status = LAT_OK;
  for (int lc = 0; lc < n_loads; ++lc) {
    const char* sc = scal.data() + (size_t)lc * kScalBytes;
    int it = *(const int*)(sc + 8);
    double r = *(const double*)(sc + 16);
    if (P->nax == 0) {
      it = (maxit > 0 && tol > 0) ? 1 : maxit;
      r = maxit > 0 ? 0.0 : NAN;
    } else if (maxit == 0) {
      r = NAN;
    }
    if (iters) iters[lc] = it;
    if (resid) resid[lc] = r;
    if (sigma_bar)
      for (int c = 0; c < n_c; ++c) sigma_bar[lc * n_c + c] = ((const double*)(sc + 32))[c];
    if (o.resid_history && maxit > 0) {
      if (P->nax == 0)
        for (int k = 0; k < it; ++k) o.resid_history[(size_t)lc * maxit + k] = 0.0;
      for (int k = 0; k < std::min(it, std::min(maxit, LAT_HIST_CAP)) && P->nax > 0; ++k)
        o.resid_history[(size_t)lc * maxit + k] = hist[(size_t)lc * LAT_HIST_CAP + k];
    }
    int s = LAT_OK;
    if (!isfinite(r) && maxit > 0) s = LAT_DIVERGED;
    else if (!(r < tol)) s = LAT_NOT_CONVERGED;
    status = std::max(status, s);
  }
  return status;
}
