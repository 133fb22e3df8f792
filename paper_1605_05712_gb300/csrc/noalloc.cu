// noalloc.cu -- basic_scheme_solve_noalloc: the Basic Scheme solve for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc around a solve: a serving loop that runs under a fixed device-memory
// budget, a host runtime whose own allocator owns all device memory, or code that prepares a stream for
// a later CUDA-graph capture and must not allocate while doing so.  For them this entry point takes no
// workspace argument and allocates nothing.  Its scratch memory (spectrum buffers, reduction partials,
// device scalars, material tables) lives in one file-scope static __device__ array of
// LAT_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until the process exits.  The
// twiddle tables are the plan's own (lattice_plan uploads them), so the scratch only holds the solve's
// workspace.
//
// Host code may not pass the array's name to a kernel: in host code that name is a host-side stand-in,
// not a device address.  The first call on each device therefore asks the runtime for the device address
// with cudaGetSymbolAddress (with that device current) and keeps it; the lookup is serialized by a mutex,
// so host threads making their first calls at the same time do not race on the cache.  Every call shares
// the one array and leaves its contents behind, so each call clears the device scalars it reads before
// use, and calls that overlap on the GPU (two streams, two host threads) race on the array.
//
// The iteration runs with plain launches instead of the CUDA graph of basic_scheme_solve (a graph is
// not instantiated here); after each iteration the number of unfinished load cases is read back, with a
// stream synchronization.  A call on a stream that is being captured is therefore refused (LAT_ERR_ARG)
// before anything is enqueued.  The kernels and their arithmetic are the same as basic_scheme_solve's,
// so the results equal its results.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "solve_detail.h"

using namespace latms_detail;

static __device__ __align__(256) unsigned char g_lat_scratch[LAT_NOALLOC_SCRATCH_BYTES];

namespace {

const int kMaxDev = 64;
void* g_scratch_ptr[kMaxDev] = {nullptr};
std::mutex g_scratch_mu;

#define CK_NA(x)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// device address of the static scratch on the current device (looked up once per device, under a lock)
int scratch_ptr(char** out) {
  int dev = 0;
  CK_NA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: device index >= 64");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
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
  cudaStream_t st = (cudaStream_t)stream;
  {  // the plain-launch loop synchronizes the stream every iteration: not possible inside a capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK_NA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return lat_fail(LAT_ERR_ARG, "basic_scheme_solve_noalloc: the stream is being captured (the call "
                                   "synchronizes it every iteration); call it outside the capture");
  }
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (int rc = check_common(P, tol, maxit, o)) return rc;
  if (int rc = check_c0(C0)) return rc;
  if (((uintptr_t)eps & eps_align_mask(P)) != 0) return lat_fail(LAT_ERR_ARG, "eps misaligned (16 bytes; 8 on general plans)");
  if (int rc = lat_plan_device_check(P)) return rc;
  const Work wl = layout(P, n_loads, o.precision, n_phases, 1, o.scheme);
  const size_t need = up256(wl.total);
  if (need > (size_t)LAT_NOALLOC_SCRATCH_BYTES)
    return lat_fail(LAT_ERR_SIZE, "basic_scheme_solve_noalloc: this solve needs " + std::to_string(need) +
                                      " bytes of scratch, more than the static " +
                                      std::to_string((size_t)LAT_NOALLOC_SCRATCH_BYTES) +
                                      " (use basic_scheme_solve with a caller-allocated workspace)");
  char* ws = nullptr;
  if (int rc = scratch_ptr(&ws)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  const LatDev dv = make_dev(P, o.precision);
  std::vector<ItemHost> items;
  load_case_items(P, phase, C0, E, n_loads, eps, sigma, items);
  // run_batch clears the device scalars left by an earlier call before the kernels read them
  return run_batch(P, items, {stiffness}, {n_phases}, tol, maxit, o, ws, wl, dv, false, sigma_bar, iters, resid, st);
}
