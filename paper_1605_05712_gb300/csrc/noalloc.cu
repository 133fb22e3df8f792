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
// is not instantiated here); after each iteration the number of unfinished load cases is read
// back.  The kernels and their arithmetic are the same, so the results equal basic_scheme_solve's.
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
  if (n_loads < 1) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: n_loads < 1");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  if (int rc = check_c0(C0)) return rc;
  if (((uintptr_t)eps & 15) != 0) return lat_fail(LAT_ERR_ARG, "eps must be 16-byte aligned");
  const bool fp32 = (o.precision == LAT_MIXED);
  // scratch layout: [solve workspace | twiddle table | split twiddle table]
  const Work wl = layout(P, n_loads, o.precision, n_phases, 1, o.scheme);
  int64_t n_tw = 0, n_stw = 0;
  if (P->nax > 0) lat_host_twiddles(P, o.precision, nullptr, nullptr, &n_tw, &n_stw);
  const size_t es = fp32 ? sizeof(float2) : o.precision == LAT_DF64 ? sizeof(float4) : sizeof(double2);
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
  // this plan's twiddles go into the scratch too (the plan's own device tables are not needed)
  std::vector<char> htw(n_tw * es), hstw(n_stw * es);
  if (P->nax > 0) {
    lat_host_twiddles(P, o.precision, htw.data(), hstw.data(), nullptr, nullptr);
    CK_NA(cudaMemcpyAsync(ws + off_tw, htw.data(), htw.size(), cudaMemcpyHostToDevice, st));
    if (n_stw) CK_NA(cudaMemcpyAsync(ws + off_stw, hstw.data(), hstw.size(), cudaMemcpyHostToDevice, st));
  }
  LatDev dv = make_dev(P, o.precision);
  dv.tw = ws + off_tw;
  dv.stw = ws + off_stw;
  std::vector<ItemHost> items;
  load_case_items(P, phase, C0, E, n_loads, eps, sigma, items);
  // run_batch clears the device scalars left by an earlier call before the kernels read them
  return run_batch(P, items, {stiffness}, {n_phases}, tol, maxit, o, ws, wl, dv, false, sigma_bar, iters, resid, st);
}
