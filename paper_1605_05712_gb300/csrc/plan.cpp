// plan.cpp -- lattice_plan: Smith normal form, FFT decomposition, index maps, twiddles.
//
// Sec. 2.1-2.2 of arXiv 1605.05712: the pattern P(M) of a regular integer
// matrix M, its Smith normal form M = Q E R (E = diag(e), e_j | e_{j+1}), and
// the statement that with lexicographic addressing lambda of P(M) and k of
// G(M^T) the pattern DFT is an ordinary d_M-dimensional DFT over the e_j > 1:
//   h(k)^T y(lambda) = sum_j k_j lambda_j / e_j  (mod 1),
//   y(lambda) = R^{-1} E^{-1} lambda (mod 1),  h(k) = R^T k (mod M^T Z^d).
// The frequency in the symmetric cell is found from the fractional coordinates
//   M^{-T} R^T k = Q^{-T} E^{-1} k = v / e_d,  v = sum_j k_j (e_d / e_j) P e_j,
// P = Q^{-T}: reduce v into [-e_d/2, e_d/2) componentwise and h = M^T v / e_d.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "solve_detail.h"

static thread_local std::string g_err;
void lat_set_error(const std::string& s) { g_err = s; }
int lat_fail(int code, const std::string& s) {
  g_err = s;
  return code;
}
extern "C" const char* lattice_last_error(void) { return g_err.c_str(); }

typedef __int128 i128;

namespace {

struct Mat {
  int d;
  i128 a[3][3];
};

Mat ident(int d) {
  Mat I;
  I.d = d;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) I.a[i][j] = (i == j);
  return I;
}

i128 det(const Mat& A) {
  if (A.d == 2) return A.a[0][0] * A.a[1][1] - A.a[0][1] * A.a[1][0];
  return A.a[0][0] * (A.a[1][1] * A.a[2][2] - A.a[1][2] * A.a[2][1]) -
         A.a[0][1] * (A.a[1][0] * A.a[2][2] - A.a[1][2] * A.a[2][0]) +
         A.a[0][2] * (A.a[1][0] * A.a[2][1] - A.a[1][1] * A.a[2][0]);
}

// adjugate: adj(A) A = det(A) I
Mat adjugate(const Mat& A) {
  Mat B;
  B.d = A.d;
  if (A.d == 2) {
    B.a[0][0] = A.a[1][1];
    B.a[0][1] = -A.a[0][1];
    B.a[1][0] = -A.a[1][0];
    B.a[1][1] = A.a[0][0];
    return B;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
      B.a[i][j] = A.a[r0][c0] * A.a[r1][c1] - A.a[r0][c1] * A.a[r1][c0];
    }
  return B;
}

i128 iabs(i128 x) { return x < 0 ? -x : x; }

// floor(a / b) for b != 0
i128 floordiv(i128 a, i128 b) {
  i128 q = a / b, r = a % b;
  if (r != 0 && ((r < 0) != (b < 0))) --q;
  return q;
}
i128 mod(i128 a, i128 b) {  // b > 0, result in [0, b)
  i128 r = a % b;
  return r < 0 ? r + b : r;
}

// Smith normal form by textbook elimination: U A V = diag(e), returns Q = U^-1, R = V^-1.
bool smith(const Mat& M, Mat& Q, i128 e[3], Mat& R) {
  const int d = M.d;
  Mat A = M, U = ident(d), V = ident(d);
  const i128 LIM = ((i128)1) << 100;
  for (int t = 0; t < d; ++t) {
    for (int guard = 0; guard < 100000; ++guard) {
      int bi = -1, bj = -1;
      for (int i = t; i < d; ++i)
        for (int j = t; j < d; ++j)
          if (A.a[i][j] != 0 && (bi < 0 || iabs(A.a[i][j]) < iabs(A.a[bi][bj]))) bi = i, bj = j;
      if (bi < 0) return false;
      if (bi != t)
        for (int j = 0; j < d; ++j) std::swap(A.a[bi][j], A.a[t][j]), std::swap(U.a[bi][j], U.a[t][j]);
      if (bj != t)
        for (int i = 0; i < d; ++i) std::swap(A.a[i][bj], A.a[i][t]), std::swap(V.a[i][bj], V.a[i][t]);
      const i128 p = A.a[t][t];
      bool clean = true;
      for (int i = t + 1; i < d; ++i) {
        i128 q = floordiv(A.a[i][t], p);
        if (q != 0)
          for (int j = 0; j < d; ++j) A.a[i][j] -= q * A.a[t][j], U.a[i][j] -= q * U.a[t][j];
        if (A.a[i][t] != 0) clean = false;
      }
      for (int j = t + 1; j < d; ++j) {
        i128 q = floordiv(A.a[t][j], p);
        if (q != 0)
          for (int i = 0; i < d; ++i) A.a[i][j] -= q * A.a[i][t], V.a[i][j] -= q * V.a[i][t];
        if (A.a[t][j] != 0) clean = false;
      }
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
          if (iabs(A.a[i][j]) > LIM || iabs(U.a[i][j]) > LIM || iabs(V.a[i][j]) > LIM) return false;
      if (!clean) continue;
      int bad = -1;
      for (int i = t + 1; i < d && bad < 0; ++i)
        for (int j = t + 1; j < d; ++j)
          if (A.a[i][j] % p != 0) {
            bad = i;
            break;
          }
      if (bad >= 0) {
        for (int j = 0; j < d; ++j) A.a[t][j] += A.a[bad][j], U.a[t][j] += U.a[bad][j];
        continue;
      }
      break;
    }
    if (A.a[t][t] < 0)
      for (int j = 0; j < d; ++j) A.a[t][j] = -A.a[t][j], U.a[t][j] = -U.a[t][j];
  }
  for (int i = 0; i < d; ++i) e[i] = A.a[i][i];
  // inverses of unimodular U, V: adj * det (det = +-1)
  i128 du = det(U), dv = det(V);
  if (iabs(du) != 1 || iabs(dv) != 1) return false;
  Q = adjugate(U);
  R = adjugate(V);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Q.a[i][j] *= du, R.a[i][j] *= dv;
  return true;
}

int ilog2(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}
bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

// W_N^t = exp(-2 pi i t / N) with octant reduction so that cos/sin only see |angle| <= pi/4
void twiddle(int64_t t, int64_t N, double* re, double* im) {
  t = (int64_t)mod(t, N);
  // angle = 2 pi t / N = pi * (8t/N) / 4 ; octant o = floor(8t / N)
  int64_t o8 = 8 * t;
  int64_t o = o8 / N;
  // residual fraction r = 8t/N - o in [0,1); angle = (o + r) * pi/4
  double r = (double)(o8 - o * N) / (double)N;
  double c, s;
  int oo = (int)(o & 7);
  // reduce to phi in [0, pi/4]
  double phi = (oo & 1) ? (1.0 - r) * M_PI / 4 : r * M_PI / 4;
  double cp = cos(phi), sp = sin(phi);
  // angle = k*pi/4 + (+-)phi, map through octant symmetries
  switch (oo) {
    case 0: c = cp; s = sp; break;     // [0, pi/4)
    case 1: c = sp; s = cp; break;     // [pi/4, pi/2): angle = pi/2 - phi
    case 2: c = -sp; s = cp; break;    // angle = pi/2 + phi
    case 3: c = -cp; s = sp; break;    // angle = pi - phi
    case 4: c = -cp; s = -sp; break;   // angle = pi + phi
    case 5: c = -sp; s = -cp; break;   // angle = 3pi/2 - phi
    case 6: c = sp; s = -cp; break;    // angle = 3pi/2 + phi
    default: c = cp; s = -sp; break;   // angle = 2pi - phi
  }
  *re = c;
  *im = -s;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// radices of a mixed-radix transform of length L: 4s, a 2, then the odd primes ascending
static int factor_radices(int64_t L, uint16_t* rad) {
  int n = 0;
  while (L % 4 == 0 && n < LAT_MAX_RADIX) rad[n++] = 4, L /= 4;
  while (L % 2 == 0 && n < LAT_MAX_RADIX) rad[n++] = 2, L /= 2;
  for (int64_t p = 3; L > 1 && n < LAT_MAX_RADIX; p += 2)
    while (L % p == 0 && n < LAT_MAX_RADIX) rad[n++] = (uint16_t)p, L /= p;
  return L == 1 ? n : -1;
}

static void set_cv(lat_plan* P) {
  for (int t = 0; t < P->nax; ++t) {
    LatAxis& a = P->ax[t];
    int j = a.snf;
    for (int r = 0; r < P->d; ++r) {
      i128 c = (i128)(P->ed / P->e[j]) * P->P[r][j];
      a.cv[r] = (int64_t)mod((i128)a.mult * mod(c, P->ed), P->ed);
    }
  }
}

// Layout of a general plan (some divisor is not a power of two): every divisor axis is one logical axis
// transformed in one pass; the last one (the contiguous row) is split four-step as A B when longer than
// a line may be.  A line of every logical axis, all n_c planes, twice (ping-pong), must fit in shared
// memory: 2 x n_c x L x 16 B <= 196 KB.  A largest divisor with no such split (a large prime, or a
// large prime times a small factor) stays one row transformed by Bluestein's chirp-z convolution.
static int choose_layout_general(lat_plan* P, const std::vector<int>& paxes) {
  const int d = P->d, n_c = d * (d + 1) / 2;
  const int64_t LMAX = (n_c == 3) ? 2048 : 1024;
  P->general = 1;
  for (size_t i = 0; i + 1 < paxes.size(); ++i)
    if (P->e[paxes[i]] > LMAX)
      return lat_fail(LAT_ERR_UNSUPPORTED, "elementary divisor " + std::to_string((long long)P->e[paxes[i]]) +
                                               " is longer than one mixed-radix pass (" + std::to_string((long long)LMAX) +
                                               " points) and not the largest");
  const int jL = paxes.back();
  const int64_t eL = P->e[jL];
  int64_t B = eL;
  if (eL > LMAX) {   // four-step: B (row) and A = eL / B both <= LMAX, B nearest sqrt(eL), the larger on the row
    B = -1;
    double best = 1e300;
    for (int64_t b = 2; b <= LMAX; ++b)
      if (eL % b == 0 && eL / b <= LMAX && b >= eL / b) {
        const double dist = fabs(log((double)b) - 0.5 * log((double)eL));
        if (dist < best) best = dist, B = b;
      }
    if (B < 0) B = eL, P->blue = 1;   // no split into two lines that fit: Bluestein on the whole row
  }
  int na = 0;
  for (size_t i = 0; i + 1 < paxes.size(); ++i) {
    LatAxis& a = P->ax[na++];
    a.len = (int)P->e[paxes[i]];
    a.snf = paxes[i];
    a.mult = 1;
  }
  P->split = (B != eL);
  if (P->split) {
    LatAxis& a = P->ax[na++];
    a.len = (int)(eL / B);
    a.snf = jL;
    a.mult = B;  // k = k2 + B k1
    P->split_n1 = na - 1;
    P->split_e = eL;
    P->split_lo_log2 = (ilog2(eL) + 1) / 2;
  }
  {
    LatAxis& a = P->ax[na++];
    a.len = (int)B;
    a.snf = jL;
    a.mult = 1;
  }
  P->nax = na;
  int off = 0;
  for (int i = 0; i < na; ++i) {
    P->ax[i].log2len = ilog2(P->ax[i].len);
    const bool row = i == na - 1;
    P->ax_nrad[i] = (row && P->blue) ? 0 : factor_radices(P->ax[i].len, P->ax_rad[i]);
    if (P->ax_nrad[i] < 0 && row && !P->split) P->blue = 1, P->ax_nrad[i] = 0;   // more stages than a pass holds
    if (P->ax_nrad[i] < 0) return lat_fail(LAT_ERR_UNSUPPORTED, "axis length with too many prime factors");
    P->ax_twoff[i] = off;
    if (!(row && P->blue)) off += P->ax[i].len;   // the Bluestein row has no table of W_p^t
  }
  if (P->blue) {
    // Bluestein (chirp-z): X_k = w_k sum_n (x_n w_n) conj(w_{k-n}), w_n = exp(-i pi n^2 / p), a cyclic
    // convolution of length L >= 2p - 1 (power of two), transformed by the power-of-two plan diag(1, L)
    int64_t L = 1;
    while (L < 2 * eL - 1) L <<= 1;
    if (L > (int64_t(1) << 23))
      return lat_fail(LAT_ERR_UNSUPPORTED, "elementary divisor " + std::to_string((long long)eL) +
                                               " has no split into two lines of at most " + std::to_string((long long)LMAX) +
                                               " points and is longer than a chirp-z transform of 2^23 points allows");
    P->blue_L = L;
  }
  P->Rlen = (int)B;
  P->Rh = (int)(B / 2);
  P->log2Rh = ilog2(std::max<int64_t>(P->Rh, 1));
  P->nrows = P->m / B;
  P->ngroups = na - 1;
  for (int k = 0; k < na - 1; ++k) {
    LatGroup& G = P->grp[k];
    G.a0 = k;
    G.a1 = k + 1;
    G.G = P->ax[k].len;
    G.outer = 1;
    for (int t = 0; t < k; ++t) G.outer *= P->ax[t].len;
    G.inner = 1;
    for (int t = k + 1; t < na - 1; ++t) G.inner *= P->ax[t].len;
    G.has_twiddle = P->split && k == P->split_n1;
  }
  set_cv(P);
  return LAT_OK;
}

static int choose_layout(lat_plan* P) {
  const int d = P->d;
  std::vector<int> paxes;
  for (int j = 0; j < d; ++j)
    if (P->e[j] > 1) paxes.push_back(j);
  P->dM = (int)paxes.size();
  for (int j : paxes)
    if (!is_pow2(P->e[j])) return choose_layout_general(P, paxes);
  if (P->dM == 0) {  // m == 1
    P->nax = 0;
    P->ngroups = 0;
    return LAT_OK;
  }
  const int n_c = d * (d + 1) / 2;
  // shared-memory budgets, sized for binary64 complex (16 B)
  const int64_t RH_MAX = (n_c == 3) ? 2048 : 1024;          // row half-length
  const int64_t G_MAX = (n_c == 3) ? 2048 : 1024;           // column group length
  const int jL = paxes.back();
  const int64_t eL = P->e[jL];
  const int lgL = ilog2(eL);
  // candidate row lengths B (power of two dividing eL, B <= 2*RH_MAX); B = eL means no split
  int best_groups = 1 << 30;
  int64_t bestB = -1;
  double best_dist = 1e300;
  std::vector<int64_t> cands;
  for (int lb = (lgL + 1) / 2; lb < lgL; ++lb) {
    int64_t B = int64_t(1) << lb;
    if (B <= 2 * RH_MAX && B >= 2) cands.push_back(B);
  }
  // no split only where it leaves work for several blocks (at least 32 rows) or the rows are short: a
  // single long row (a small rank-1 pattern, m <= 4096) would run as one block per item on one SM, where
  // the split's two passes spread it over m / B blocks
  if (eL <= 2 * RH_MAX && (P->m / eL >= 32 || eL <= 128)) cands.push_back(eL);
  for (int64_t B : cands) {
    std::vector<int64_t> lens;
    for (size_t i = 0; i + 1 < paxes.size(); ++i) lens.push_back(P->e[paxes[i]]);
    if (B != eL) lens.push_back(eL / B);
    // greedy grouping from the left
    int ng = 0;
    size_t i = 0;
    bool ok = true;
    while (i < lens.size()) {
      int64_t g = 1;
      size_t j = i;
      while (j < lens.size() && g * lens[j] <= G_MAX) g *= lens[j++];
      if (j == i) {
        ok = false;
        break;
      }
      ++ng;
      i = j;
    }
    if (!ok) continue;
    // fewest column passes first; then rows and columns balanced (B close to sqrt(2m)),
    // ties to the shorter row
    const double target = 0.5 * log2(2.0 * (double)P->m);
    const double dist = fabs(log2((double)B) - target);
    if (ng < best_groups || (ng == best_groups && dist < best_dist - 1e-9)) best_groups = ng, bestB = B, best_dist = dist;
  }
  if (bestB < 0) return lat_fail(LAT_ERR_UNSUPPORTED, "no FFT decomposition fits shared memory");
  const int64_t B = bestB;
  // logical axes
  int na = 0;
  for (size_t i = 0; i + 1 < paxes.size(); ++i) {
    LatAxis& a = P->ax[na++];
    a.len = (int)P->e[paxes[i]];
    a.snf = paxes[i];
    a.mult = 1;
  }
  P->split = (B != eL);
  if (P->split) {
    LatAxis& a = P->ax[na++];
    a.len = (int)(eL / B);
    a.snf = jL;
    a.mult = B;  // k = k2 + B k1
    P->split_n1 = na - 1;
    P->split_e = eL;
    P->split_lo_log2 = (lgL + 1) / 2;
  }
  {
    LatAxis& a = P->ax[na++];
    a.len = (int)B;
    a.snf = jL;
    a.mult = 1;
  }
  P->nax = na;
  for (int i = 0; i < na; ++i) P->ax[i].log2len = ilog2(P->ax[i].len);
  P->Rlen = (int)B;
  P->Rh = (int)(B / 2);
  P->log2Rh = ilog2(P->Rh);
  P->nrows = P->m / B;
  // groups
  P->ngroups = 0;
  int i = 0;
  while (i < na - 1) {
    int64_t g = 1;
    int j = i;
    while (j < na - 1 && g * P->ax[j].len <= G_MAX) g *= P->ax[j++].len;
    LatGroup& G = P->grp[P->ngroups++];
    G.a0 = i;
    G.a1 = j;
    G.G = (int)g;
    G.outer = 1;
    for (int t = 0; t < i; ++t) G.outer *= P->ax[t].len;
    G.inner = 1;
    for (int t = j; t < na - 1; ++t) G.inner *= P->ax[t].len;
    G.has_twiddle = P->split && (P->split_n1 >= i && P->split_n1 < j);
    i = j;
  }
  set_cv(P);   // v contributions
  return LAT_OK;
}

int lat_host_twiddles(const lat_plan* P, int fp32, void* tw, void* stw, int64_t* n_tw, int64_t* n_stw);

// Host part of the twiddle tables: their sizes (the device copies are made by lat_upload_tables).
static void set_table_sizes(lat_plan* P) {
  int lg = 1;
  for (int i = 0; i < P->nax; ++i) lg = std::max(lg, P->ax[i].log2len);
  P->tw_log2 = lg;
  if (P->split) {
    P->stw_lo_n = int64_t(1) << P->split_lo_log2;
    P->stw_hi_n = ((P->split_e - 1) >> P->split_lo_log2) + 1;
  }
}

// binary64, binary32 and double-float copies of both twiddle tables on the current device
static int lat_upload_tables(lat_plan* P) {
  if (P->nax == 0) return LAT_OK;
  int64_t n_tw = 0, n_stw = 0;
  lat_host_twiddles(P, 0, nullptr, nullptr, &n_tw, &n_stw);
  void** dst_tw[3] = {(void**)&P->d_tw, (void**)&P->d_twf, (void**)&P->d_twdf};
  void** dst_stw[3] = {(void**)&P->d_stw, (void**)&P->d_stwf, (void**)&P->d_stwdf};
  const size_t es[3] = {sizeof(double2), sizeof(float2), sizeof(float4)};
  for (int k = 0; k < 3; ++k) {
    std::vector<char> htw(n_tw * es[k]), hstw(std::max<int64_t>(n_stw, 1) * es[k]);
    lat_host_twiddles(P, k, htw.data(), P->split ? hstw.data() : nullptr, nullptr, nullptr);
    cudaError_t err;
    if ((err = cudaMalloc(dst_tw[k], htw.size())) != cudaSuccess ||
        (err = cudaMemcpy(*dst_tw[k], htw.data(), htw.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return lat_fail(LAT_ERR_CUDA, std::string("twiddle upload: ") + cudaGetErrorString(err));
    if (P->split && n_stw > 0) {
      const size_t nb = n_stw * es[k];
      if ((err = cudaMalloc(dst_stw[k], nb)) != cudaSuccess ||
          (err = cudaMemcpy(*dst_stw[k], hstw.data(), nb, cudaMemcpyHostToDevice)) != cudaSuccess)
        return lat_fail(LAT_ERR_CUDA, std::string("split twiddle upload: ") + cudaGetErrorString(err));
    }
  }
  if (!P->general) {   // butterfly table of the binary64 kernels (FmaTw in fft_smem.cuh)
    const int64_t N = int64_t(1) << P->tw_log2, n = std::max<int64_t>(N / 4, 1);
    int lgn = 0;
    while ((int64_t(1) << lgn) < n) ++lgn;
    std::vector<double> lf((size_t)n * 12, 0.0);
    for (int64_t t = 0; t < n; ++t) {
      double e[6];   // t1, t3, tau2, s1, sx2, r (with the form bit)
      int64_t swap = 0;
      if (t == 0) {   // identity twiddles: the plain additions, exactly
        e[0] = e[1] = e[2] = 0.0;
        e[3] = e[4] = e[5] = 1.0;
      } else {
        double r1, i1, r2, i2, r3, i3;
        twiddle(t, N, &r1, &i1);
        twiddle(2 * t, N, &r2, &i2);
        twiddle(3 * t, N, &r3, &i3);
        e[0] = i1 / r1;   // 0 < t < N/4: cos of t, 3t (of 2 pi / N) are nonzero
        e[1] = i3 / r3;
        e[3] = r1;
        e[5] = r3 / r1;
        if (std::fabs(r2) >= std::fabs(i2)) {
          e[2] = i2 / r2;
          e[4] = r2;
        } else {
          e[2] = -r2 / i2;
          e[4] = -i2;
          swap = 1;
        }
      }
      uint64_t rb;
      memcpy(&rb, &e[5], sizeof(rb));
      rb = (rb & ~uint64_t(1)) | (uint64_t)swap;
      memcpy(&e[5], &rb, sizeof(rb));
      uint64_t u = 0;   // bit-reversed position of t over lgn bits
      for (int k = 0; k < lgn; ++k) u |= (uint64_t)((t >> k) & 1) << (lgn - 1 - k);
      for (int k = 0; k < 6; ++k) {
        lf[(size_t)k * n + t] = e[k];
        lf[(size_t)(6 + k) * n + u] = e[k];
      }
    }
    // table of the real-row pre/post-processing (kernels.cu): for w = W_N^t, 0 < t <= N/4 (where Im w != 0),
    // c = Re w / Im w, Im w and Im w / 2, so that w b = Im w (c b.x - b.y, c b.y + b.x)
    std::vector<double> rc((size_t)(N / 4 + 1) * 4, 0.0);
    for (int64_t t = 1; t <= N / 4; ++t) {
      double re, im;
      twiddle(t, N, &re, &im);
      rc[(size_t)t * 4] = re / im;
      rc[(size_t)t * 4 + 1] = im;
      rc[(size_t)t * 4 + 2] = 0.5 * im;
    }
    cudaError_t err;
    if ((err = cudaMalloc((void**)&P->d_lf, lf.size() * sizeof(double))) != cudaSuccess ||
        (err = cudaMemcpy(P->d_lf, lf.data(), lf.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMalloc((void**)&P->d_rc, rc.size() * sizeof(double))) != cudaSuccess ||
        (err = cudaMemcpy(P->d_rc, rc.data(), rc.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
      return lat_fail(LAT_ERR_CUDA, std::string("butterfly table upload: ") + cudaGetErrorString(err));
  }
  return LAT_OK;
}

// Bluestein row (general plans, see lat_plan): the power-of-two plan diag(1, L), the chirp
// w_n = exp(-i pi n^2 / p) (n^2 reduced mod 2p exactly) and the unnormalized DFT of the wrapped
// conjugate chirp b (b_j = conj(w_|j|) at j mod L for |j| < p, 0 elsewhere), transformed on the device
// by the sub-plan's own forward passes so that its spectral order is the one the solver multiplies in
static int lat_blue_tables(lat_plan* P) {
  const int64_t p = P->Rlen, L = P->blue_L;
  const int64_t Msub[4] = {1, 0, 0, L};
  if (int rc = lattice_plan(Msub, 2, &P->blue_sub)) return rc;
  const lat_plan* S = P->blue_sub;
  if (S->general || S->device != P->device || S->nax != (S->split ? 2 : 1))
    return lat_fail(LAT_ERR_CUDA, "chirp-z sub-plan: unexpected layout or device");
  // the sub-plan's storage order (lattice_points): a split row holds sample n = n1 + A n2 at n1 B + n2
  const int64_t A = S->split ? S->ax[S->split_n1].len : 1;
  P->blue_lgA = ilog2(A);
  P->blue_lgB = ilog2(L / A);
  auto slot = [&](int64_t n) { return ((n & (A - 1)) << P->blue_lgB) + (n >> P->blue_lgA); };
  std::vector<double2> w(p), b(L, make_double2(0.0, 0.0));
  for (int64_t n = 0; n < p; ++n) {
    double re, im;
    twiddle((int64_t)((i128)n * n % (2 * p)), 2 * p, &re, &im);
    w[n] = make_double2(re, im);
    b[slot(n)] = make_double2(re, -im);
    if (n > 0) b[slot(L - n)] = make_double2(re, -im);
  }
  cudaError_t err;
  if ((err = cudaMalloc((void**)&P->d_chirp, p * sizeof(double2))) != cudaSuccess ||
      (err = cudaMemcpy(P->d_chirp, w.data(), p * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMalloc((void**)&P->d_bh, L * sizeof(double2))) != cudaSuccess ||
      (err = cudaMemcpy(P->d_bh, b.data(), L * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return lat_fail(LAT_ERR_CUDA, std::string("chirp-z table upload: ") + cudaGetErrorString(err));
  return lat_blue_transform_bh(P);
}

int lat_plan_device_check(const lat_plan* P) {
  if (P->nax == 0) return LAT_OK;   // m = 1: no transform, no tables
  if (P->device < 0)
    return lat_fail(LAT_ERR_CUDA, "the plan was created without a CUDA device (host-only plan: points, "
                                  "frequencies and gather maps only)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != P->device)
    return lat_fail(LAT_ERR_ARG, "the plan's tables live on device " + std::to_string(P->device) +
                                     " but the current device is " + std::to_string(dev));
  return LAT_OK;
}

extern "C" int lattice_plan(const int64_t* Min, int d, lat_plan** out) {
  if (!Min || !out) return lat_fail(LAT_ERR_ARG, "lattice_plan: NULL argument");
  *out = nullptr;
  if (d != 2 && d != 3) return lat_fail(LAT_ERR_DIM, "lattice_plan: d must be 2 or 3");
  Mat M;
  M.d = d;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      if (Min[i * d + j] > (int64_t(1) << 40) || Min[i * d + j] < -(int64_t(1) << 40))
        return lat_fail(LAT_ERR_SIZE, "lattice_plan: |M_ij| > 2^40");
      M.a[i][j] = Min[i * d + j];
    }
  i128 D = det(M);
  if (D == 0) return lat_fail(LAT_ERR_SINGULAR, "lattice_plan: det M = 0");
  if (iabs(D) > (((i128)1) << 28)) return lat_fail(LAT_ERR_SIZE, "lattice_plan: m = |det M| > 2^28");
  Mat Q, R;
  i128 e[3];
  if (!smith(M, Q, e, R)) return lat_fail(LAT_ERR_SIZE, "lattice_plan: Smith normal form left the exact range");
  lat_plan* P = new lat_plan();
  memset(P, 0, sizeof(lat_plan));
  P->d = d;
  P->det = (int64_t)D;
  P->m = (int64_t)iabs(D);
  Mat Rinv = adjugate(R);
  i128 dR = det(R);
  Mat Qinv = adjugate(Q);
  i128 dQ = det(Q);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      bool in = i < d && j < d;
      P->M[i][j] = in ? (int64_t)M.a[i][j] : 0;
      P->Q[i][j] = in ? (int64_t)Q.a[i][j] : 0;
      P->R[i][j] = in ? (int64_t)R.a[i][j] : 0;
      P->Rinv[i][j] = in ? (int64_t)(Rinv.a[i][j] * dR) : 0;
      P->P[i][j] = in ? (int64_t)(Qinv.a[j][i] * dQ) : 0;  // Q^{-T}
    }
  P->ed = 1;
  for (int j = 0; j < d; ++j) P->e[j] = (int64_t)e[j], P->ed = std::max(P->ed, P->e[j]);
  for (int j = d; j < 3; ++j) P->e[j] = 1;
  int rc = choose_layout(P);
  if (rc != LAT_OK) {
    lattice_plan_destroy(P);
    return rc;
  }
  set_table_sizes(P);
  // the twiddle tables go to the current device now, so that no solve allocates; without a CUDA device
  // the plan stays host-only (points, frequencies, gather maps) and solves report LAT_ERR_CUDA
  P->device = -1;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) == cudaSuccess && n_dev > 0) {
    if (cudaGetDevice(&P->device) != cudaSuccess) P->device = -1;
  }
  cudaGetLastError();   // a machine without a device leaves a (non-sticky) error behind
  if (P->device >= 0 && (rc = lat_upload_tables(P)) == LAT_OK && P->blue) rc = lat_blue_tables(P);
  if (P->device >= 0 && rc != LAT_OK) {
    lattice_plan_destroy(P);
    return rc;
  }
  *out = P;
  return LAT_OK;
}

int lat_host_twiddles(const lat_plan* P, int fp32, void* tw, void* stw, int64_t* n_tw, int64_t* n_stw) {
  int lg = 1;
  for (int i = 0; i < P->nax; ++i) lg = std::max(lg, P->ax[i].log2len);
  // power-of-two plans: one table of W_N^t, N = 2^lg; general plans: the tables of W_len^t of every
  // logical axis, concatenated
  int64_t N = int64_t(1) << lg;
  if (P->general) {
    N = 0;
    for (int i = 0; i < P->nax; ++i) N += (P->blue && i == P->nax - 1) ? 0 : P->ax[i].len;
  }
  int64_t lo_n = 0, hi_n = 0;
  if (P->split) {
    lo_n = int64_t(1) << P->split_lo_log2;
    hi_n = ((P->split_e - 1) >> P->split_lo_log2) + 1;
  }
  if (n_tw) *n_tw = N;
  if (n_stw) *n_stw = hi_n + lo_n;
  // kind (the fp32 argument): 0 binary64 (double2), 1 binary32 (float2), 2 double-float pairs
  // (float4: re hi, re lo, im hi, im lo)
  auto put = [&](void* dst, int64_t i, double re, double im) {
    if (fp32 == 1) {
      ((float2*)dst)[i] = make_float2((float)re, (float)im);
    } else if (fp32 == 2) {
      const float rh = (float)re, ih = (float)im;
      ((float4*)dst)[i] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
    } else {
      ((double2*)dst)[i] = make_double2(re, im);
    }
  };
  if (tw && !P->general)
    for (int64_t t = 0; t < N; ++t) {
      double re, im;
      twiddle(t, N, &re, &im);
      put(tw, t, re, im);
    }
  if (tw && P->general)
    for (int i = 0; i < P->nax; ++i)
      for (int64_t t = 0; t < ((P->blue && i == P->nax - 1) ? 0 : P->ax[i].len); ++t) {
        double re, im;
        twiddle(t, P->ax[i].len, &re, &im);
        put(tw, P->ax_twoff[i] + t, re, im);
      }
  if (stw && P->split) {
    for (int64_t j = 0; j < hi_n; ++j) {
      double re, im;
      twiddle(j << P->split_lo_log2, P->split_e, &re, &im);
      put(stw, j, re, im);
    }
    for (int64_t j = 0; j < lo_n; ++j) {
      double re, im;
      twiddle(j, P->split_e, &re, &im);
      put(stw, hi_n + j, re, im);
    }
  }
  return LAT_OK;
}

extern "C" void lattice_plan_destroy(lat_plan* P) {
  if (!P) return;
  if (P->d_tw) cudaFree(P->d_tw);
  if (P->d_twf) cudaFree(P->d_twf);
  if (P->d_stw) cudaFree(P->d_stw);
  if (P->d_stwf) cudaFree(P->d_stwf);
  if (P->d_twdf) cudaFree(P->d_twdf);
  if (P->d_stwdf) cudaFree(P->d_stwdf);
  if (P->d_lf) cudaFree(P->d_lf);
  if (P->d_rc) cudaFree(P->d_rc);
  if (P->d_chirp) cudaFree(P->d_chirp);
  if (P->d_bh) cudaFree(P->d_bh);
  if (P->blue_sub) lattice_plan_destroy(P->blue_sub);
  delete P;
}

extern "C" int lattice_plan_set_cell(lat_plan* P, const double* L) {
  if (!P) return lat_fail(LAT_ERR_ARG, "lattice_plan_set_cell: NULL plan");
  if (!L) {
    P->has_cell = 0;
    return LAT_OK;
  }
  const int d = P->d;
  double A[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double scale = 0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      if (!std::isfinite(L[i * d + j])) return lat_fail(LAT_ERR_ARG, "lattice_plan_set_cell: L not finite");
      A[i][j] = L[i * d + j];
      scale = std::max(scale, std::fabs(A[i][j]));
    }
  // inverse by cofactors (d <= 3); L^{-T}_ij = cof_ij / det
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale))
    return lat_fail(LAT_ERR_SINGULAR, "lattice_plan_set_cell: L is singular");
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      P->cell_LinvT[i][j] = (A[i1][j1] * A[i2][j2] - A[i1][j2] * A[i2][j1]) / det;
    }
  P->has_cell = 1;
  return LAT_OK;
}

extern "C" int lattice_plan_layout(const lat_plan* P, int* nax, int* ax_len, int* ngroups, int* grp, int* split) {
  if (!P) return lat_fail(LAT_ERR_ARG, "lattice_plan_layout: NULL plan");
  if (nax) *nax = P->nax;
  if (ax_len)
    for (int a = 0; a < LAT_MAX_AX; ++a) ax_len[a] = a < P->nax ? P->ax[a].len : 0;
  if (ngroups) *ngroups = P->ngroups;
  if (grp)
    for (int g = 0; g < LAT_MAX_GROUPS; ++g) {
      grp[2 * g] = g < P->ngroups ? P->grp[g].a0 : 0;
      grp[2 * g + 1] = g < P->ngroups ? P->grp[g].a1 : 0;
    }
  if (split) *split = P->blue ? 2 : P->split;
  return LAT_OK;
}

extern "C" int lattice_plan_info(const lat_plan* P, int64_t* m, int* d_M, int64_t* divisors) {
  if (!P) return lat_fail(LAT_ERR_ARG, "lattice_plan_info: NULL plan");
  if (m) *m = P->m;
  if (d_M) *d_M = P->dM;
  if (divisors)
    for (int j = 0; j < P->d; ++j) divisors[j] = P->e[j];
  return LAT_OK;
}

// storage slot -> lambda (spatial).  Split axis: lambda = n1 + A * n2.
static void slot_lambda(const lat_plan* P, int64_t slot, int64_t lam[3]) {
  lam[0] = lam[1] = lam[2] = 0;
  int64_t rest = slot;
  for (int a = P->nax - 1; a >= 0; --a) {
    int64_t idx = rest % P->ax[a].len;
    rest /= P->ax[a].len;
    int64_t smult = 1;
    if (P->split && a == P->nax - 1) smult = P->ax[P->split_n1].len;  // n2 carries A
    lam[P->ax[a].snf] += smult * idx;
  }
}

extern "C" int lattice_points(const lat_plan* P, int64_t* p) {
  if (!P || !p) return lat_fail(LAT_ERR_ARG, "lattice_points: NULL argument");
  const int d = P->d;
  const int64_t m = P->m;
  for (int64_t s = 0; s < m; ++s) {
    int64_t lam[3];
    slot_lambda(P, s, lam);
    for (int i = 0; i < d; ++i) {
      i128 acc = 0;
      for (int j = 0; j < d; ++j) acc += (i128)P->Rinv[i][j] * lam[j] * (m / P->e[j]);
      i128 r = mod(acc, m);
      if (2 * r >= m) r -= m;
      p[s * d + i] = (int64_t)r;
    }
  }
  return LAT_OK;
}

namespace {
struct PointKey {
  int64_t c[3];
  bool operator==(const PointKey& o) const { return c[0] == o.c[0] && c[1] == o.c[1] && c[2] == o.c[2]; }
};
struct PointHash {
  size_t operator()(const PointKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) h = (h ^ (uint64_t)k.c[i]) * 1099511628211ull;
    return (size_t)(h ^ (h >> 29));
  }
};
}  // namespace

extern "C" int lattice_gather_map(const lat_plan* from, const lat_plan* to, int32_t* map) {
  if (!from || !to || !map) return lat_fail(LAT_ERR_ARG, "lattice_gather_map: NULL argument");
  if (from->d != to->d) return lat_fail(LAT_ERR_ARG, "lattice_gather_map: plans of different dimension");
  if (from->m >= (int64_t(1) << 31)) return lat_fail(LAT_ERR_SIZE, "lattice_gather_map: m of the source >= 2^31");
  if (from->m % to->m != 0)
    return lat_fail(LAT_ERR_ARG, "lattice_gather_map: |det| of the target does not divide the source's: not a subpattern");
  const int d = from->d;
  std::vector<int64_t> pf((size_t)from->m * d), pt((size_t)to->m * d);
  lattice_points(from, pf.data());
  lattice_points(to, pt.data());
  // y = p_from / m_from = p_to / m_to: both in [-1/2, 1/2)^d, so equal points have equal scaled numerators
  const int64_t scale = from->m / to->m;
  std::unordered_map<PointKey, int32_t, PointHash> where;
  where.reserve((size_t)from->m * 2);
  for (int64_t s = 0; s < from->m; ++s) {
    PointKey k = {{0, 0, 0}};
    for (int i = 0; i < d; ++i) k.c[i] = pf[(size_t)s * d + i];
    where.emplace(k, (int32_t)s);
  }
  for (int64_t s = 0; s < to->m; ++s) {
    PointKey k = {{0, 0, 0}};
    for (int i = 0; i < d; ++i) k.c[i] = pt[(size_t)s * d + i] * scale;
    auto it = where.find(k);
    if (it == where.end())
      return lat_fail(LAT_ERR_ARG, "lattice_gather_map: a point of the target pattern is not in the source pattern");
    map[s] = it->second;
  }
  return LAT_OK;
}

// spectral slot of the complex transform (bit-reversed positions on every axis of a power-of-two plan,
// natural positions on a general plan) -> k
static void slot_k(const lat_plan* P, int64_t slot, int64_t k[3]) {
  k[0] = k[1] = k[2] = 0;
  int64_t rest = slot;
  for (int a = P->nax - 1; a >= 0; --a) {
    int64_t pos = rest % P->ax[a].len;
    rest /= P->ax[a].len;
    int lg = P->ax[a].log2len;
    int64_t kk = 0;
    if (P->general) {
      kk = pos;   // mixed-radix transforms keep natural order
    } else {
      for (int b = 0; b < lg; ++b)
        if (pos & (int64_t(1) << b)) kk |= int64_t(1) << (lg - 1 - b);
    }
    k[P->ax[a].snf] += P->ax[a].mult * kk;
  }
}

extern "C" int lattice_freqs(const lat_plan* P, int64_t* h) {
  if (!P || !h) return lat_fail(LAT_ERR_ARG, "lattice_freqs: NULL argument");
  const int d = P->d;
  Mat MT;
  MT.d = d;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) MT.a[i][j] = P->M[j][i];
  Mat A = adjugate(MT);
  const i128 D = P->det;
  for (int64_t s = 0; s < P->m; ++s) {
    int64_t k[3];
    slot_k(P, s, k);
    i128 g[3], u[3], z[3];
    for (int i = 0; i < d; ++i) {
      g[i] = 0;
      for (int j = 0; j < d; ++j) g[i] += (i128)P->R[j][i] * k[j];  // R^T k
    }
    for (int i = 0; i < d; ++i) {
      u[i] = 0;
      for (int j = 0; j < d; ++j) u[i] += A.a[i][j] * g[j];
      z[i] = floordiv(2 * u[i] + D, 2 * D);  // floor(u/D + 1/2)
    }
    for (int i = 0; i < d; ++i) {
      i128 acc = g[i];
      for (int j = 0; j < d; ++j) acc -= MT.a[i][j] * z[j];
      h[s * d + i] = (int64_t)acc;
    }
  }
  return LAT_OK;
}
