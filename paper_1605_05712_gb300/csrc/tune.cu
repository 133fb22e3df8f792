// tune.cu -- autotuner of the launch shapes of the iteration: rows per block of the row pass and the
// tile width (columns per block) of every column pass, timed on the device for one plan, precision
// and item count.  Not in the paper (its FFT is Matlab's); the choices change the grouping of lines
// into blocks only, never the arithmetic of a line, so tuned and untuned solves give the same fields.
#include <string.h>

#include <algorithm>
#include <vector>

#include "solve_detail.h"

using namespace latms_detail;

#define CKT(x)                                                                                 \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

struct TuneWs {
  Work wl;
  size_t off_eps, off_phase, total;
};

TuneWs tune_layout(const lat_plan* P, int n_items, int precision) {
  TuneWs t;
  t.wl = layout(P, n_items, precision, 1, 1);
  const int n_c = P->d * (P->d + 1) / 2;
  t.off_eps = align256(t.wl.total);
  t.off_phase = align256(t.off_eps + (size_t)n_items * n_c * P->m * sizeof(double));
  t.total = align256(t.off_phase + (size_t)P->m);
  return t;
}

// one iteration (row pass + column passes) with geometry `geo`; events around kernel `which`
// (0 = row pass, 1 + k = every launch of column group k) accumulate its device time
template <typename Real>
int timed_iteration(const GroupRun& g, const Geometry& geo, int which, cudaEvent_t* ev, float* ms,
                    cudaStream_t st) {
  const lat_plan* P = g.P;
  RowArgs full = g.full;
  full.rpc = geo.rpc;
  full.it.cond = 0;
  *ms = 0.f;
  int n_ev = 0;
  auto begin = [&](bool on) {
    if (on) cudaEventRecord(ev[2 * n_ev], st);
  };
  auto end = [&](bool on) {
    if (on) {
      cudaEventRecord(ev[2 * n_ev + 1], st);
      ++n_ev;
    }
  };
  begin(which == 0);
  launch_row_pass<Real>(g.dv, full, geo.row_blocks, g.n_items, kThreads, geo.row_smem, st);
  end(which == 0);
  for (int k = P->ngroups - 1; k >= 0; --k) {
    begin(which == 1 + k);
    enqueue_col_group<Real>(g.dv, P, geo, g.cl, k, k == 0 ? COL_GAMMA : COL_FWD, g.n_items, st);
    end(which == 1 + k);
  }
  for (int k = 1; k < P->ngroups; ++k) {
    begin(which == 1 + k);
    enqueue_col_group<Real>(g.dv, P, geo, g.cl, k, COL_INV, g.n_items, st);
    end(which == 1 + k);
  }
  CKT(cudaGetLastError());
  CKT(cudaStreamSynchronize(st));
  for (int i = 0; i < n_ev; ++i) {
    float t = 0.f;
    CKT(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
    *ms += t;
  }
  return LAT_OK;
}

// the median of `reps` timed iterations after one untimed one
template <typename Real>
int time_kernel(const GroupRun& g, const Geometry& geo, int which, cudaEvent_t* ev, int reps, float* out,
                cudaStream_t st) {
  float t = 0.f;
  if (int rc = timed_iteration<Real>(g, geo, which, ev, &t, st)) return rc;
  std::vector<float> v;
  for (int r = 0; r < reps; ++r) {
    if (int rc = timed_iteration<Real>(g, geo, which, ev, &t, st)) return rc;
    v.push_back(t);
  }
  std::sort(v.begin(), v.end());
  *out = v[v.size() / 2];
  return LAT_OK;
}

template <typename Real>
int tune_kernels(lat_plan* P, GroupRun& g, int n_c, size_t cs, lat_plan::Tune& best, cudaStream_t st) {
  std::vector<cudaEvent_t> ev(2 * 4);
  for (auto& e : ev) CKT(cudaEventCreate(&e));
  Geometry cur = g.geo;
  const int reps = 5;
  int rc = LAT_OK;
  // row pass: rows per block
  {
    float bt = 1e30f;
    int brpc = cur.rpc;
    for (int rpc = 1; rpc <= P->nrows && rc == LAT_OK; rpc *= 2) {
      Geometry cand = cur;
      if (geometry_set_rpc(P, n_c, cs, true, rpc, cand) != LAT_OK) continue;
      float t = 0.f;
      if ((rc = time_kernel<Real>(g, cand, 0, ev.data(), reps, &t, st)) != LAT_OK) break;
      if (t < bt) bt = t, brpc = rpc;
    }
    if (rc == LAT_OK) {
      geometry_set_rpc(P, n_c, cs, true, brpc, cur);
      best.rpc = brpc;
      best.ms[0] = bt;
    }
  }
  // column passes: tile width of each group
  for (int k = 0; k < P->ngroups && rc == LAT_OK; ++k) {
    float bt = 1e30f;
    int bw = cur.w[k];
    const int64_t ic = P->grp[k].inner * (int64_t)P->Rh;
    for (int64_t w = 1; w <= std::min<int64_t>(ic, 128) && rc == LAT_OK; w *= 2) {
      Geometry cand = cur;
      if (geometry_set_w(P, n_c, cs, P->Rh, true, k, w, cand) != LAT_OK) continue;
      float t = 0.f;
      if ((rc = time_kernel<Real>(g, cand, 1 + k, ev.data(), reps, &t, st)) != LAT_OK) break;
      if (t < bt) bt = t, bw = (int)w;
    }
    if (rc == LAT_OK) {
      geometry_set_w(P, n_c, cs, P->Rh, true, k, bw, cur);
      best.w[k] = bw;
      best.ms[1 + k] = bt;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

}  // namespace

extern "C" size_t lattice_autotune_workspace_bytes(const lat_plan* P, int n_items, int precision) {
  if (!P || n_items < 1 || check_geometry(P, precision) != LAT_OK) return 0;
  return tune_layout(P, n_items, precision).total;
}

extern "C" int lattice_autotune(lat_plan* P, int n_items, int precision, void* workspace, size_t workspace_bytes,
                                void* stream) {
  if (!P || !workspace || n_items < 1) return lat_fail(LAT_ERR_ARG, "lattice_autotune: bad argument");
  lat_solve_opts o;
  memset(&o, 0, sizeof(o));
  o.precision = precision;
  o.mixed_increment = 1;
  o.mixed_restart = -1;
  if (int rc = check_common(P, 0.0, 1, o)) return rc;
  const TuneWs tw = tune_layout(P, n_items, precision);
  if (workspace_bytes < tw.total) return lat_fail(LAT_ERR_SIZE, "lattice_autotune: workspace too small");
  if (P->nax == 0) return LAT_OK;
  if (P->general) return lat_fail(LAT_ERR_UNSUPPORTED, "lattice_autotune: power-of-two plans only");
  if (int rc = lat_plan_device_check(P)) return rc;
  if (int rc = ensure_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString((cudaError_t)rc));
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int n_c = P->d * (P->d + 1) / 2;
  // a homogeneous medium (one phase, C != C0) under a unit load: timing only, the data stay bounded
  CKT(cudaMemsetAsync(ws + tw.off_phase, 0, (size_t)P->m, st));
  std::vector<ItemHost> items(n_items);
  for (int i = 0; i < n_items; ++i) {
    ItemHost& it = items[i];
    it.phase = (const uint8_t*)(ws + tw.off_phase);
    it.table = 0;
    it.C0[0] = 5.5;
    it.C0[1] = 5.5;
    for (int c = 0; c < 6; ++c) it.E[c] = (c == 0) ? 1.0 : 0.0;
    it.eps = (double*)(ws + tw.off_eps) + (size_t)i * n_c * P->m;
    it.sigma = nullptr;
  }
  double stiff[36];
  memset(stiff, 0, sizeof(stiff));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) stiff[i * 6 + j] = 1.0;
    stiff[i * 6 + i] = 3.0;
    stiff[(i + 3) * 6 + (i + 3)] = 1.0;
  }
  lat_plan::Tune& slot = P->tune[precision][tune_bucket(n_items)];
  slot.valid = 0;  // the prologue runs with the untuned shapes
  GroupRun g;
  const LatDev dv = make_dev(P, precision);
  if (int rc = group_prepare(P, items, {stiff}, {1}, 0.0, 1 << 30, o, ws, tw.wl, dv, g, st)) return rc;
  lat_plan::Tune best;
  memset(&best, 0, sizeof(best));
  const size_t cs = precision == LAT_MIXED ? 8 : 16;
  int rc = by_kind(precision, [&](auto tag) { return tune_kernels<decltype(tag)>(P, g, n_c, cs, best, st); });
  CKT(cudaStreamSynchronize(st));
  if (rc != LAT_OK) return rc;
  best.valid = 1;
  slot = best;
  return LAT_OK;
}

extern "C" int lattice_tune_info(const lat_plan* P, int n_items, int precision, int* rpc, int* w, float* ms,
                                 int* n_groups) {
  if (!P || n_items < 1 || precision < 0 || precision > 2) return lat_fail(LAT_ERR_ARG, "lattice_tune_info: bad argument");
  const lat_plan::Tune& t = P->tune[precision][tune_bucket(n_items)];
  if (n_groups) *n_groups = P->ngroups;
  if (!t.valid) return 0;
  if (rpc) *rpc = t.rpc;
  for (int k = 0; k < P->ngroups; ++k) {
    if (w) w[k] = t.w[k];
    if (ms) ms[1 + k] = t.ms[1 + k];
  }
  if (ms) ms[0] = t.ms[0];
  return 1;
}
