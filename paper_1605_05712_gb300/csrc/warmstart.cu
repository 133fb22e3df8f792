// warmstart.cu -- the learned warm start: a periodic 3-D U-Net (4 levels, 32 channels) that maps the
// stiffness field to the strain-localization field A (eps^(0) = A : E), trained and run by these
// kernels.  BF16 weights and activations, FP32 accumulation (BF16 tensor cores for the 3x3x3
// convolutions: implicit GEMM over the 27 taps, one block per contiguous row with the 9 neighbour
// rows and their periodic halo staged in shared memory; rows shorter than 16 voxels use CUDA cores).
//
// Layout: channels-last, voxel v = (z n1 + y) n2 + x, 32 channels per voxel (BF16 activations,
// FP32 gradients).  Convolution weights: FP32 master [27][ci][co], BF16 copies Wf[27][co][ci]
// (forward: B operand col-major with k = ci) and Wb[27][ci][co] (backward data: k = co).
// Taps t in lexicographic (dz, dy, dx) order; conv3(x)[v, co] = b[co] + sum_t sum_ci W[t,ci,co] x[v + off_t, ci].
#include <cuda_bf16.h>
#include <mma.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "conv_tc05.cuh"
#include "warmstart.h"

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

namespace {

constexpr float kLeak = 0.1f;   // slope of the leaky ReLU for negative inputs

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ------------------------------------------------------------------ 3x3x3 convolution, tensor cores
// in: [V][32] bf16; W: [27][32 n][32 k] bf16 (B operand, col-major with leading dimension 32);
// out_mode 0: bf16 act(acc + bias), act = leaky ReLU; 1: fp32 acc (no bias); neg: taps -off (backward data)
__global__ void __launch_bounds__(128) conv3_tc_kernel(const bf16* __restrict__ in, const bf16* __restrict__ W,
                                                       const float* __restrict__ bias, void* out, int n0, int n1,
                                                       int n2, int out_mode, int neg) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int L2 = n2 + 2;
  bf16* rows = (bf16*)smem;                       // [9][n2 + 2][32]
  bf16* wsm = rows + 9 * L2 * 32;                 // [32][32]
  const int row = blockIdx.x;                     // (z, y)
  const int z = row / n1, y = row - z * n1;
  const int tid = threadIdx.x;
  // stage the 9 neighbour rows with periodic halo: 4 x 16-byte chunks per voxel
  const int nchunk = 9 * L2 * 4;
  for (int i = tid; i < nchunk; i += blockDim.x) {
    const int q = i & 3, vx = (i >> 2) % L2, r = (i >> 2) / L2;
    const int dz = r / 3 - 1, dy = r % 3 - 1;
    const int zz = wrap(z + (neg ? -dz : dz), n0), yy = wrap(y + (neg ? -dy : dy), n1);
    const int xs = wrap(vx - 1, n2);
    const uint4 val = *((const uint4*)(in + ((size_t)(zz * n1 + yy) * n2 + xs) * 32) + q);
    *((uint4*)(rows + ((size_t)r * L2 + vx) * 32) + q) = val;
  }
  const int warp = tid >> 5, nw = blockDim.x >> 5;
  const int mt = n2 >> 4;                         // M tiles of 16 voxels
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];  // up to 2 M tiles per warp (n2 <= 128)
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) wmma::fill_fragment(acc[a][b], 0.0f);
  for (int t = 0; t < 27; ++t) {
    __syncthreads();
    for (int i = tid; i < 128; i += blockDim.x) ((uint4*)wsm)[i] = ((const uint4*)(W + (size_t)t * 1024))[i];
    __syncthreads();
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int r = (dz + 1) * 3 + (dy + 1);
    const int ox = neg ? -dx : dx;
    for (int j = 0; j < 2; ++j) {
      const int mi = warp + j * nw;
      if (mi >= mt) break;
      for (int ks = 0; ks < 2; ++ks) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa;
        wmma::load_matrix_sync(fa, rows + ((size_t)r * L2 + mi * 16 + ox + 1) * 32 + ks * 16, 32);
        for (int ni = 0; ni < 2; ++ni) {
          wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> fb;
          wmma::load_matrix_sync(fb, wsm + ni * 16 * 32 + ks * 16, 32);
          wmma::mma_sync(acc[j][ni], fa, fb, acc[j][ni]);
        }
      }
    }
  }
  __syncthreads();
  float* osm = (float*)smem;                      // [n2][32] fp32 staging (reuses the rows)
  for (int j = 0; j < 2; ++j) {
    const int mi = warp + j * nw;
    if (mi >= mt) break;
    for (int ni = 0; ni < 2; ++ni)
      wmma::store_matrix_sync(osm + (size_t)mi * 16 * 32 + ni * 16, acc[j][ni], 32, wmma::mem_row_major);
  }
  __syncthreads();
  const size_t base = (size_t)row * n2 * 32;
  for (int i = tid; i < n2 * 32; i += blockDim.x) {
    float v = osm[i];
    if (out_mode == 0) {
      v += bias[i & 31];
      ((bf16*)out)[base + i] = __float2bfloat16(v > 0.f ? v : kLeak * v);
    } else {
      ((float*)out)[base + i] = v;
    }
  }
}

// dW[t][ci][co] += sum_v x[v + off_t][ci] dpre[v][co]; grid (chunks of rows, 27 taps); db for the centre tap
__global__ void __launch_bounds__(128) conv3_dw_tc_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dp,
                                                          float* dW, float* db, int n0, int n1, int n2,
                                                          int rows_per_cta) {
  extern __shared__ __align__(128) unsigned char smem[];
  bf16* xs = (bf16*)smem;                         // [n2][32]
  bf16* ds = xs + n2 * 32;                        // [n2][32]
  float* red = (float*)(ds + n2 * 32);            // [32][32] fp32 staging, then db partial
  const int t = blockIdx.y;
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mi = warp >> 1, ni = warp & 1;        // 4 warps: output tiles (ci 16 x co 16)
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
  wmma::fill_fragment(acc, 0.0f);
  float dbacc = 0.f;
  const int nrows = n0 * n1;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(nrows, r0 + rows_per_cta);
  for (int row = r0; row < r1; ++row) {
    const int z = row / n1, y = row - z * n1;
    const int zz = wrap(z + dz, n0), yy = wrap(y + dy, n1);
    __syncthreads();
    for (int i = tid; i < n2 * 4; i += blockDim.x) {
      const int q = i & 3, vx = i >> 2;
      const int xsrc = wrap(vx + dx, n2);
      ((uint4*)(xs + vx * 32))[q] = ((const uint4*)(x + ((size_t)(zz * n1 + yy) * n2 + xsrc) * 32))[q];
      ((uint4*)(ds + vx * 32))[q] = ((const uint4*)(dp + ((size_t)row * n2 + vx) * 32))[q];
    }
    __syncthreads();
    for (int ks = 0; ks < (n2 >> 4); ++ks) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> fa;   // (ci, v): ptr[v*32 + ci]
      wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;   // (v, co): ptr[v*32 + co]
      wmma::load_matrix_sync(fa, xs + ks * 16 * 32 + mi * 16, 32);
      wmma::load_matrix_sync(fb, ds + ks * 16 * 32 + ni * 16, 32);
      wmma::mma_sync(acc, fa, fb, acc);
    }
    if (t == 13 && tid < 32)
      for (int v = 0; v < n2; ++v) dbacc += __bfloat162float(ds[v * 32 + tid]);
  }
  __syncthreads();
  wmma::store_matrix_sync(red + mi * 16 * 32 + ni * 16, acc, 32, wmma::mem_row_major);
  __syncthreads();
  for (int i = tid; i < 1024; i += blockDim.x) atomicAdd(dW + (size_t)t * 1024 + i, red[i]);
  if (t == 13 && tid < 32) atomicAdd(db + tid, dbacc);
}

// ------------------------------------------------------------------ 3x3x3 convolution, CUDA cores (short rows)
// forward (neg = 0): out[v, co] = sum_t sum_ci in[v + off_t, ci] W[t][ci][co]
// backward data (neg = 1): out[u, ci] = sum_t sum_co in[u - off_t, co] W[t][ci][co]; Wm is [27][ci][co] bf16
__global__ void conv3_cc_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Wm,
                                const float* __restrict__ bias, void* out, int n0, int n1, int n2, int out_mode,
                                int neg) {
  const int64_t V = (int64_t)n0 * n1 * n2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 32) return;
  const int oc = (int)(idx & 31);
  const int64_t v = idx >> 5;
  const int x = (int)(v % n2), y = (int)((v / n2) % n1), z = (int)(v / ((int64_t)n1 * n2));
  float acc = 0.f;
  for (int t = 0; t < 27; ++t) {
    int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    if (neg) dz = -dz, dy = -dy, dx = -dx;
    const int64_t u = ((int64_t)wrap(z + dz, n0) * n1 + wrap(y + dy, n1)) * n2 + wrap(x + dx, n2);
    const bf16* ip = in + u * 32;
    for (int c = 0; c < 32; ++c) {
      const float w = neg ? __bfloat162float(Wm[(size_t)t * 1024 + oc * 32 + c])   // W[t][ci=oc][co=c]
                          : __bfloat162float(Wm[(size_t)t * 1024 + c * 32 + oc]);  // W[t][ci=c][co=oc]
      acc += __bfloat162float(ip[c]) * w;
    }
  }
  if (out_mode == 0) {
    acc += bias[oc];
    ((bf16*)out)[idx] = __float2bfloat16(acc > 0.f ? acc : kLeak * acc);
  } else {
    ((float*)out)[idx] = acc;
  }
}

__global__ void conv3_dw_cc_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dp, float* dW, float* db,
                                   int n0, int n1, int n2) {
  const int t = blockIdx.x, ci = threadIdx.x >> 5, co = threadIdx.x & 31;  // block of 1024 threads per tap
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  float acc = 0.f, dba = 0.f;
  for (int z = 0; z < n0; ++z)
    for (int y = 0; y < n1; ++y)
      for (int xx = 0; xx < n2; ++xx) {
        const int64_t v = ((int64_t)z * n1 + y) * n2 + xx;
        const int64_t u = ((int64_t)wrap(z + dz, n0) * n1 + wrap(y + dy, n1)) * n2 + wrap(xx + dx, n2);
        const float g = __bfloat162float(dp[v * 32 + co]);
        acc += __bfloat162float(x[u * 32 + ci]) * g;
        if (t == 13 && ci == 0) dba += g;
      }
  atomicAdd(dW + (size_t)t * 1024 + ci * 32 + co, acc);
  if (t == 13 && ci == 0) atomicAdd(db + co, dba);
}

// ------------------------------------------------------------------ elementwise pieces
__global__ void pool_fwd_kernel(const bf16* in, bf16* out, int m0, int m1, int m2) {  // out dims m = n/2
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t V = (int64_t)m0 * m1 * m2;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  const int x = (int)(v % m2), y = (int)((v / m2) % m1), z = (int)(v / ((int64_t)m1 * m2));
  const int n1 = 2 * m1, n2 = 2 * m2;
  float s = 0.f;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int e = 0; e < 2; ++e)
        s += __bfloat162float(in[(((int64_t)(2 * z + a) * n1 + 2 * y + b) * n2 + 2 * x + e) * 32 + c]);
  out[idx] = __float2bfloat16(0.125f * s);
}

// out (fine, n) = up(coarse) + skip   (bf16)
__global__ void up_add_kernel(const bf16* coarse, const bf16* skip, bf16* out, int n0, int n1, int n2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t V = (int64_t)n0 * n1 * n2;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  const int x = (int)(v % n2), y = (int)((v / n2) % n1), z = (int)(v / ((int64_t)n1 * n2));
  const int64_t u = ((int64_t)(z / 2) * (n1 / 2) + y / 2) * (n2 / 2) + x / 2;
  out[idx] = __float2bfloat16(__bfloat162float(coarse[u * 32 + c]) + __bfloat162float(skip[idx]));
}

// g_coarse[u] (+)= sum of the 8 fine children of u (scale 1: up, 1/8: pool)
__global__ void restrict_kernel(const float* fine, float* coarse, int m0, int m1, int m2, float scale, int accum) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t V = (int64_t)m0 * m1 * m2;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  const int x = (int)(v % m2), y = (int)((v / m2) % m1), z = (int)(v / ((int64_t)m1 * m2));
  const int n1 = 2 * m1, n2 = 2 * m2;
  float s = 0.f;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int e = 0; e < 2; ++e) s += fine[(((int64_t)(2 * z + a) * n1 + 2 * y + b) * n2 + 2 * x + e) * 32 + c];
  coarse[idx] = scale * s + (accum ? coarse[idx] : 0.f);
}

// fine[v] += scale * coarse[parent(v)]   (gradient of the pool: scale 1/8)
__global__ void prolong_add_kernel(const float* coarse, float* fine, int n0, int n1, int n2, float scale) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t V = (int64_t)n0 * n1 * n2;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  const int x = (int)(v % n2), y = (int)((v / n2) % n1), z = (int)(v / ((int64_t)n1 * n2));
  const int64_t u = ((int64_t)(z / 2) * (n1 / 2) + y / 2) * (n2 / 2) + x / 2;
  fine[idx] += scale * coarse[u * 32 + c];
}

// dpre = g * act'(y), to bf16 (act = leaky ReLU of the conv output; y keeps the sign of its input)
__global__ void relu_mask_kernel(const float* g, const bf16* y, bf16* dpre, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dpre[i] = __float2bfloat16(__bfloat162float(y[i]) > 0.f ? g[i] : kLeak * g[i]);
}

// head: y[v][j] = hb[j] + sum_c u[v][c] H[c][j]  (36 outputs, fp32)
__global__ void head_fwd_kernel(const bf16* u, const float* H, const float* hb, float* y, int64_t V) {
  __shared__ float Hs[32 * 36 + 36];
  for (int i = threadIdx.x; i < 32 * 36; i += blockDim.x) Hs[i] = H[i];
  for (int i = threadIdx.x; i < 36; i += blockDim.x) Hs[32 * 36 + i] = hb[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 36) return;
  const int j = (int)(idx % 36);
  const int64_t v = idx / 36;
  float acc = Hs[32 * 36 + j];
  for (int c = 0; c < 32; ++c) acc += __bfloat162float(u[v * 32 + c]) * Hs[c * 36 + j];
  y[idx] = acc;
}

// head backward, input gradient: du[v][c] = sum_j H[c][j] dy[v][j]
__global__ void head_bwd_dx_kernel(const float* H, const float* dy, float* du, int64_t V) {
  __shared__ float Hs[32 * 36];
  for (int i = threadIdx.x; i < 32 * 36; i += blockDim.x) Hs[i] = H[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  float s = 0.f;
  for (int j = 0; j < 36; ++j) s += Hs[c * 36 + j] * dy[v * 36 + j];
  du[idx] = s;
}

// head backward, weights: dH[c][j] += sum_v u[v][c] dy[v][j], dhb[j] += sum_v dy[v][j];
// each block reduces a chunk of voxels staged in shared memory, then one atomic per output
__global__ void __launch_bounds__(256) head_bwd_dw_kernel(const bf16* u, const float* dy, float* dH, float* dhb,
                                                          int64_t V, int64_t chunk) {
  __shared__ float us[64 * 32];
  __shared__ float ds[64 * 36];
  float acc[5] = {0, 0, 0, 0, 0};
  float bacc = 0.f;
  const int64_t v0 = (int64_t)blockIdx.x * chunk, v1 = min(V, v0 + chunk);
  for (int64_t vb = v0; vb < v1; vb += 64) {
    const int nv = (int)min((int64_t)64, v1 - vb);
    __syncthreads();
    for (int i = threadIdx.x; i < nv * 32; i += blockDim.x) us[i] = __bfloat162float(u[vb * 32 + i]);
    for (int i = threadIdx.x; i < nv * 36; i += blockDim.x) ds[i] = dy[vb * 36 + i];
    __syncthreads();
    for (int k = 0; k < 5; ++k) {
      const int o = threadIdx.x + k * 256;
      if (o >= 32 * 36) break;
      const int c = o / 36, j = o % 36;
      float a = 0.f;
      for (int v = 0; v < nv; ++v) a += us[v * 32 + c] * ds[v * 36 + j];
      acc[k] += a;
    }
    if (threadIdx.x < 36)
      for (int v = 0; v < nv; ++v) bacc += ds[v * 36 + threadIdx.x];
  }
  for (int k = 0; k < 5; ++k) {
    const int o = threadIdx.x + k * 256;
    if (o < 32 * 36) atomicAdd(dH + o, acc[k]);
  }
  if (threadIdx.x < 36) atomicAdd(dhb + threadIdx.x, bacc);
}

// sum of squares of the targets (per-sample normalisation of the loss)
__global__ void sumsq_kernel(const float* t, double* out, int64_t n) {
  __shared__ double red[256];
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)t[i] * t[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// a[v][c] -= sums[c] / V for the 36 output channels (projection onto zero spatial mean)
__global__ void center_kernel(float* a, const double* sums, int64_t V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 36) return;
  a[idx] -= (float)(sums[idx % 36] / (double)V);
}

// relative squared error: loss = sum (y - t)^2 / (sum t^2 + n eps0), dy = 2 (y - t) / (sum t^2 + n eps0)
__global__ void rel_mse_kernel(const float* y, const float* t, const double* tss, float* dy, double* loss, int64_t n,
                               double eps0) {
  __shared__ double red[256];
  const double den = *tss + (double)n * eps0;
  const float inv = (float)(1.0 / den);
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d * inv;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / den);
}

// Adam on fp32 masters; refresh the bf16 copies of conv weights (forward Wf[t][co][ci], backward Wb[t][ci][co])
__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

__global__ void refresh_bf16_kernel(const float* Wm, bf16* Wf, bf16* Wb) {  // one conv layer: 27 x 32 x 32
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * 1024) return;
  const int t = i / 1024, ci = (i / 32) % 32, co = i % 32;
  const bf16 w = __float2bfloat16(Wm[i]);
  Wf[(size_t)t * 1024 + co * 32 + ci] = w;
  Wb[(size_t)t * 1024 + ci * 32 + co] = w;
}

// features: x0[v][c] = table[phase(v)][c] for c < 21, else 0 (bf16)
__global__ void features_kernel(const uint8_t* phase, const float* table, bf16* x0, int64_t V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 32) return;
  const int c = (int)(idx & 31);
  const int64_t v = idx >> 5;
  x0[idx] = __float2bfloat16(c < 21 ? table[(int)phase[v] * 21 + c] : 0.f);
}

// targets: t[v][6 i + j] = eps_j[i][v] - E_j[i]  (unit load cases j, strain components i)
__global__ void targets_kernel(const double* eps, const double* Eu, float* t, int64_t V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 36) return;
  const int ch = (int)(idx % 36);
  const int64_t v = idx / 36;
  const int i = ch / 6, j = ch % 6;
  t[idx] = (float)(eps[((int64_t)j * 6 + i) * V + v] - Eu[j * 6 + i]);
}

// channel sums of y (36) for the mean projection
__global__ void chan_sum_kernel(const float* y, double* sums, int64_t V) {
  __shared__ double red[36];
  if (threadIdx.x < 36) red[threadIdx.x] = 0;
  __syncthreads();
  double acc[36];
  for (int j = 0; j < 36; ++j) acc[j] = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
    for (int j = 0; j < 36; ++j) acc[j] += y[v * 36 + j];
  for (int j = 0; j < 36; ++j) atomicAdd(&red[j], acc[j]);
  __syncthreads();
  if (threadIdx.x < 36) atomicAdd(&sums[threadIdx.x], red[threadIdx.x]);
}

// eps0[l][i][v] = E_l[i] + sum_j (y[v][6 i + j] - mean_ij) Eu_l[j]   (Eu: E with engineering shear)
__global__ void predict_strain_kernel(const float* y, const double* sums, const double* E, int n_loads, double* eps0,
                                      int64_t V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * 6 * n_loads) return;
  const int64_t v = idx % V;
  const int i = (int)((idx / V) % 6);
  const int l = (int)(idx / (V * 6));
  const double* El = E + l * 6;
  double s = El[i];
  for (int j = 0; j < 6; ++j) {
    const double Eu = El[j] * (j >= 3 ? 2.0 : 1.0);
    s += ((double)y[v * 36 + 6 * i + j] - sums[6 * i + j] / (double)V) * Eu;
  }
  eps0[idx] = s;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------------------------- host side
namespace latws {

size_t conv3_smem(int n2) { return (size_t)9 * (n2 + 2) * 32 * 2 + 2048 > (size_t)n2 * 32 * 4 ? (size_t)9 * (n2 + 2) * 32 * 2 + 2048 : (size_t)n2 * 32 * 4; }
size_t dw_smem(int n2) { return (size_t)n2 * 32 * 2 * 2 + 32 * 32 * 4; }

int set_attrs() {
  static bool done = false;
  if (done) return 0;
  cudaError_t e = cudaFuncSetAttribute(conv3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc05::conv3_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(std::max(tc05::smem_bytes(16), tc05::smem_bytes(32)), tc05::smem_bytes(64)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc05::conv3_tc05_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc05::ring_smem_bytes(128));
  if (e == cudaSuccess)   // the whole shared memory of an SM: two blocks of 86-105 KB
    e = cudaFuncSetAttribute(tc05::conv3_tc05_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv3_dw_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) done = true;
  return (int)e;
}

// tcgen05 paths: rows of 128 voxels with the sliding window, rows of 16, 32 or 64 packed into 128-voxel tiles
bool tc05_fits(int n0, int n1, int n2) {   // the tile kernel
  return (n2 == 16 || n2 == 32 || n2 == 64) && n1 % (128 / n2) == 0 && ((int64_t)n0 * n1 * n2) % 128 == 0;
}
// persistent blocks: as many as are resident at once (by shared memory: one or two per SM), at most one
// per tile
bool tc05_ring(int n1, int n2) { return n2 == 128 && n1 % std::min(n1, tc05::kRingRows) == 0; }   // the ring kernel
unsigned tc05_grid(int n0, int n1, int n2) {
  static int sms = 0, smem_sm = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || sms <= 0)
      sms = 1, smem_sm = 0;
  }
  // blocks never wait on one another, so a count above what is resident only queues blocks
  if (tc05_ring(n1, n2)) {   // work items of kRingRows rows
    const int per_sm = std::max(1, smem_sm / (int)(tc05::ring_smem_bytes(n2) + 1024));
    const int64_t items = (int64_t)n0 * (n1 / std::min(n1, tc05::kRingRows));
    return (unsigned)std::min<int64_t>(items, (int64_t)per_sm * sms);
  }
  const int per_sm = std::max(1, smem_sm / (int)(tc05::smem_bytes(n2) + 1024));
  const int64_t tiles = (int64_t)n0 * n1 * n2 / 128;
  return (unsigned)std::min<int64_t>(tiles, (int64_t)per_sm * sms);
}

void conv3_forward(const void* in, const void* Wf, const void* Wb, const float* bias, void* out, int n0, int n1,
                   int n2, int out_mode, cudaStream_t st) {
  if (tc05_ring(n1, n2))
    tc05::conv3_tc05_ring_kernel<<<tc05_grid(n0, n1, n2), 128, tc05::ring_smem_bytes(n2), st>>>(
        (const bf16*)in, (const bf16*)Wf, bias, out, n0, n1, n2, out_mode, 0, kLeak);
  else if (tc05_fits(n0, n1, n2))
    tc05::conv3_tc05_kernel<<<tc05_grid(n0, n1, n2), 128, tc05::smem_bytes(n2), st>>>(
        (const bf16*)in, (const bf16*)Wf, bias, out, n0, n1, n2, out_mode, 0, kLeak);
  else if (n2 >= 16 && n2 % 16 == 0 && n2 <= 128)
    conv3_tc_kernel<<<n0 * n1, 128, conv3_smem(n2), st>>>((const bf16*)in, (const bf16*)Wf, bias, out, n0, n1, n2,
                                                          out_mode, 0);
  else
    conv3_cc_kernel<<<nblk((int64_t)n0 * n1 * n2 * 32, 256), 256, 0, st>>>((const bf16*)in, (const bf16*)Wb, bias,
                                                                           out, n0, n1, n2, out_mode, 0);
}

void conv3_backward_data(const void* dpre, const void* Wb, float* out, int n0, int n1, int n2, cudaStream_t st) {
  // din[u, ci] = sum_t sum_co W[t][ci][co] dpre[u - off_t, co]: B operand (k = co, n = ci) col-major is Wb
  if (tc05_ring(n1, n2))
    tc05::conv3_tc05_ring_kernel<<<tc05_grid(n0, n1, n2), 128, tc05::ring_smem_bytes(n2), st>>>(
        (const bf16*)dpre, (const bf16*)Wb, nullptr, out, n0, n1, n2, 1, 1, kLeak);
  else if (tc05_fits(n0, n1, n2))
    tc05::conv3_tc05_kernel<<<tc05_grid(n0, n1, n2), 128, tc05::smem_bytes(n2), st>>>(
        (const bf16*)dpre, (const bf16*)Wb, nullptr, out, n0, n1, n2, 1, 1, kLeak);
  else if (n2 >= 16 && n2 % 16 == 0 && n2 <= 128)
    conv3_tc_kernel<<<n0 * n1, 128, conv3_smem(n2), st>>>((const bf16*)dpre, (const bf16*)Wb, nullptr, out, n0, n1,
                                                          n2, 1, 1);
  else
    conv3_cc_kernel<<<nblk((int64_t)n0 * n1 * n2 * 32, 256), 256, 0, st>>>((const bf16*)dpre, (const bf16*)Wb,
                                                                           nullptr, out, n0, n1, n2, 1, 1);
}

void conv3_backward_weight(const void* x, const void* dpre, float* dW, float* db, int n0, int n1, int n2,
                           cudaStream_t st) {
  if (n2 >= 16 && n2 % 16 == 0 && n2 <= 128) {
    const int rows = n0 * n1;
    const int rpc = rows >= 256 ? (rows + 255) / 256 : 1;   // about 256 chunks x 27 taps
    dim3 grid((rows + rpc - 1) / rpc, 27);
    conv3_dw_tc_kernel<<<grid, 128, dw_smem(n2), st>>>((const bf16*)x, (const bf16*)dpre, dW, db, n0, n1, n2, rpc);
  } else {
    conv3_dw_cc_kernel<<<27, 1024, 0, st>>>((const bf16*)x, (const bf16*)dpre, dW, db, n0, n1, n2);
  }
}

}  // namespace latws

using namespace latws;

// ---------------------------------------------------------------------------------------------- network
namespace {

const int kConvs = 7;                 // c0 c1 c2 c3 d2 d1 d0
const int64_t kConvW = 27 * 1024, kConvP = kConvW + 32;
const int64_t kHeadP = 32 * 36 + 36;
const int64_t kNParams = kConvs * kConvP + kHeadP;

// parameter block: [fp32 params | fp32 grads | adam m | adam v | bf16 Wf x7 | bf16 Wb x7 | fp32 feature table? no]
struct ParamView {
  float *p, *g, *m1, *m2;
  bf16 *Wf, *Wb;
};
ParamView view(void* blk) {
  ParamView v;
  float* f = (float*)blk;
  v.p = f;
  v.g = f + kNParams;
  v.m1 = f + 2 * kNParams;
  v.m2 = f + 3 * kNParams;
  bf16* b = (bf16*)(f + 4 * kNParams);
  v.Wf = b;
  v.Wb = b + kConvs * kConvW;
  return v;
}
float* convW(const ParamView& v, float* base, int l) { return base + l * kConvP; }
float* convb(const ParamView& v, float* base, int l) { return base + l * kConvP + kConvW; }

// activation workspace of one sample of n^3 (n0 = n1 = n2 = n, n divisible by 8)
struct Acts {
  int n[4];
  int64_t V[4];
  bf16 *x0, *s[4], *p[4], *i_[3], *u[3];   // p[1..3] pooled inputs, i_[l] = up + skip at level l, u[l] outputs
  float* y;                              // [V0][36]
  float* tgt;                            // [V0][36]
  float* dy;
  float *ga[4], *gb[4];                  // fp32 gradient buffers per level
  bf16* dpre;                            // bf16 scratch (level 0 size)
  double* scal;                          // loss, channel sums (36)
  size_t total;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

Acts layout_acts(char* base, int n) {
  Acts a;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  for (int l = 0; l < 4; ++l) {
    a.n[l] = n >> l;
    a.V[l] = (int64_t)a.n[l] * a.n[l] * a.n[l];
  }
  a.x0 = (bf16*)take(a.V[0] * 64);
  for (int l = 0; l < 4; ++l) a.s[l] = (bf16*)take(a.V[l] * 64);
  a.p[0] = nullptr;
  for (int l = 1; l < 4; ++l) a.p[l] = (bf16*)take(a.V[l] * 64);
  for (int l = 0; l < 3; ++l) a.i_[l] = (bf16*)take(a.V[l] * 64), a.u[l] = (bf16*)take(a.V[l] * 64);
  a.y = (float*)take(a.V[0] * 36 * 4);
  a.tgt = (float*)take(a.V[0] * 36 * 4);
  a.dy = (float*)take(a.V[0] * 36 * 4);
  for (int l = 0; l < 4; ++l) a.ga[l] = (float*)take(a.V[l] * 128), a.gb[l] = (float*)take(a.V[l] * 128);
  a.dpre = (bf16*)take(a.V[0] * 64);
  a.scal = (double*)take(128 * 8);
  a.total = off;
  return a;
}

void forward(const ParamView& P, const Acts& a, cudaStream_t st) {
  // encoder
  conv3_forward(a.x0, P.Wf + 0 * kConvW, P.Wb + 0 * kConvW, convb(P, P.p, 0), a.s[0], a.n[0], a.n[0], a.n[0], 0, st);
  for (int l = 1; l < 4; ++l) {
    pool_fwd_kernel<<<nblk(a.V[l] * 32, 256), 256, 0, st>>>(a.s[l - 1], a.p[l], a.n[l], a.n[l], a.n[l]);
    conv3_forward(a.p[l], P.Wf + l * kConvW, P.Wb + l * kConvW, convb(P, P.p, l), a.s[l], a.n[l], a.n[l], a.n[l], 0,
                  st);
  }
  // decoder: level 2, 1, 0 (conv layers 4, 5, 6)
  const bf16* coarse = a.s[3];
  for (int l = 2; l >= 0; --l) {
    const int layer = 6 - l;
    up_add_kernel<<<nblk(a.V[l] * 32, 256), 256, 0, st>>>(coarse, a.s[l], a.i_[l], a.n[l], a.n[l], a.n[l]);
    conv3_forward(a.i_[l], P.Wf + layer * kConvW, P.Wb + layer * kConvW, convb(P, P.p, layer), a.u[l], a.n[l],
                  a.n[l], a.n[l], 0, st);
    coarse = a.u[l];
  }
  const float* H = P.p + kConvs * kConvP;
  head_fwd_kernel<<<nblk(a.V[0] * 36, 256), 256, 0, st>>>(a.u[0], H, H + 32 * 36, a.y, a.V[0]);
}

// gradients of all parameters into P.g (zeroed here) from a.dy
void backward(const ParamView& P, const Acts& a, cudaStream_t st) {
  cudaMemsetAsync(P.g, 0, kNParams * sizeof(float), st);
  const float* H = P.p + kConvs * kConvP;
  float* gH = P.g + kConvs * kConvP;
  head_bwd_dx_kernel<<<nblk(a.V[0] * 32, 256), 256, 0, st>>>(H, a.dy, a.ga[0], a.V[0]);
  {
    const int64_t chunk = std::max<int64_t>(64, (a.V[0] + 511) / 512);
    head_bwd_dw_kernel<<<nblk(a.V[0], (int)chunk), 256, 0, st>>>(a.u[0], a.dy, gH, gH + 32 * 36, a.V[0], chunk);
  }
  // decoder backwards: level 0, 1, 2; ga[l] holds dL/du_l on entry
  for (int l = 0; l <= 2; ++l) {
    const int layer = 6 - l;
    const int n = a.n[l];
    relu_mask_kernel<<<nblk(a.V[l] * 32, 256), 256, 0, st>>>(a.ga[l], a.u[l], a.dpre, a.V[l] * 32);
    conv3_backward_weight(a.i_[l], a.dpre, convW(P, P.g, layer), convb(P, P.g, layer), n, n, n, st);
    conv3_backward_data(a.dpre, P.Wb + layer * kConvW, a.gb[l], n, n, n, st);   // dL/di_l = skip grad of s_l
    // dL/du_{l+1} (or dL/ds_3) = up-adjoint of dL/di_l
    restrict_kernel<<<nblk(a.V[l + 1] * 32, 256), 256, 0, st>>>(a.gb[l], a.ga[l + 1], a.n[l + 1], a.n[l + 1],
                                                                   a.n[l + 1], 1.0f, 0);
  }
  // encoder backwards: level 3 (ga[3] = dL/ds3), then 2, 1, 0 with the skip gradients gb[l]
  for (int l = 3; l >= 0; --l) {
    const int n = a.n[l];
    float* gs = (l == 3) ? a.ga[3] : a.gb[l];   // dL/ds_l (skip part already in gb[l], pool part added below)
    relu_mask_kernel<<<nblk(a.V[l] * 32, 256), 256, 0, st>>>(gs, a.s[l], a.dpre, a.V[l] * 32);
    const bf16* xin = (l == 0) ? a.x0 : a.p[l];
    conv3_backward_weight(xin, a.dpre, convW(P, P.g, l), convb(P, P.g, l), n, n, n, st);
    if (l > 0) {
      conv3_backward_data(a.dpre, P.Wb + l * kConvW, a.ga[l], n, n, n, st);   // dL/dp_l
      // pool adjoint: dL/ds_{l-1} += dL/dp_l / 8 at every child
      prolong_add_kernel<<<nblk(a.V[l - 1] * 32, 256), 256, 0, st>>>(a.ga[l], a.gb[l - 1], a.n[l - 1], a.n[l - 1],
                                                                      a.n[l - 1], 0.125f);
    }
  }
}

}  // namespace

#define CKW(x)                                                                                     \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" size_t lat_wsnet_param_bytes(void) {
  return align_up(4 * kNParams * sizeof(float)) + 2 * kConvs * kConvW * sizeof(bf16);
}
extern "C" int64_t lat_wsnet_num_params(void) { return kNParams; }

extern "C" size_t lat_wsnet_work_bytes(int n) {
  if (n < 16 || n % 8 != 0 || n > 256) return 0;
  return layout_acts(nullptr, n).total;
}

// a tcgen05 convolution whose mbarrier wait ran out wrote NaN outputs and set tc05::g_timeout: reported
// (and cleared) by the entry points that synchronize
static int tc05_check() {
  int f = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&f, tc05::g_timeout, sizeof(int));
  if (e != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("warm start: ") + cudaGetErrorString(e));
  if (f) {
    const int zero = 0;
    cudaMemcpyToSymbol(tc05::g_timeout, &zero, sizeof(int));
    return lat_fail(LAT_ERR_CUDA, "warm start: a tensor-core convolution timed out waiting for its products "
                                  "(its outputs are NaN)");
  }
  return LAT_OK;
}

extern "C" int lat_wsnet_set_params(void* params, const float* host_params, void* stream) {
  if (!params || !host_params) return lat_fail(LAT_ERR_ARG, "lat_wsnet_set_params: NULL");
  cudaStream_t st = (cudaStream_t)stream;
  ParamView P = view(params);
  CKW(cudaMemcpyAsync(P.p, host_params, kNParams * sizeof(float), cudaMemcpyHostToDevice, st));
  CKW(cudaMemsetAsync(P.m1, 0, 2 * kNParams * sizeof(float), st));
  for (int l = 0; l < kConvs; ++l)
    refresh_bf16_kernel<<<nblk(kConvW, 256), 256, 0, st>>>(convW(P, P.p, l), P.Wf + l * kConvW, P.Wb + l * kConvW);
  CKW(cudaGetLastError());
  return LAT_OK;
}

extern "C" int lat_wsnet_get_params(const void* params, float* host_params, float* host_grads, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  ParamView P = view((void*)params);
  if (host_params) CKW(cudaMemcpyAsync(host_params, P.p, kNParams * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (host_grads) CKW(cudaMemcpyAsync(host_grads, P.g, kNParams * sizeof(float), cudaMemcpyDeviceToHost, st));
  CKW(cudaStreamSynchronize(st));
  return tc05_check();
}

static int prepare(void* work, size_t work_bytes, int n, Acts& a) {
  if (n < 16 || n % 8 != 0 || n > 256) return lat_fail(LAT_ERR_SIZE, "warm start: grid size must be 16..256, divisible by 8");
  a = layout_acts((char*)work, n);
  if (!work || work_bytes < a.total) return lat_fail(LAT_ERR_SIZE, "warm start: work buffer too small");
  if (int rc = set_attrs()) return lat_fail(LAT_ERR_CUDA, std::string("warm start attributes: ") + cudaGetErrorString((cudaError_t)rc));
  return LAT_OK;
}

extern "C" int lat_wsnet_features(const uint8_t* phase, const float* table, int n, void* work, size_t work_bytes,
                                  void* stream) {
  Acts a;
  if (int rc = prepare(work, work_bytes, n, a)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  features_kernel<<<nblk(a.V[0] * 32, 256), 256, 0, st>>>(phase, table, a.x0, a.V[0]);
  CKW(cudaGetLastError());
  return LAT_OK;
}

extern "C" int lat_wsnet_forward(const void* params, int n, float* y_out, void* work, size_t work_bytes,
                                 void* stream) {
  Acts a;
  if (int rc = prepare(work, work_bytes, n, a)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  forward(view((void*)params), a, st);
  if (y_out) CKW(cudaMemcpyAsync(y_out, a.y, a.V[0] * 36 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  CKW(cudaGetLastError());
  return LAT_OK;
}

extern "C" int lat_wsnet_backward(void* params, int n, const float* dy, void* work, size_t work_bytes, void* stream) {
  Acts a;
  if (int rc = prepare(work, work_bytes, n, a)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  CKW(cudaMemcpyAsync(a.dy, dy, a.V[0] * 36 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  backward(view(params), a, st);
  CKW(cudaGetLastError());
  return LAT_OK;
}

extern "C" int lat_wsnet_train_step(void* params, const uint8_t* phase, const float* table, const double* eps_unit,
                                    int n, float lr, int step, double* loss_out, void* work, size_t work_bytes,
                                    void* stream) {
  Acts a;
  if (int rc = prepare(work, work_bytes, n, a)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  ParamView P = view(params);
  features_kernel<<<nblk(a.V[0] * 32, 256), 256, 0, st>>>(phase, table, a.x0, a.V[0]);
  // unit load cases in tensor components: E_j[i] = delta_ij (1/2 for shear)
  double Eu[36];
  for (int j = 0; j < 6; ++j)
    for (int i = 0; i < 6; ++i) Eu[j * 6 + i] = (i == j) ? (i >= 3 ? 0.5 : 1.0) : 0.0;
  double* dEu = a.scal + 8;
  CKW(cudaMemcpyAsync(dEu, Eu, sizeof(Eu), cudaMemcpyHostToDevice, st));
  targets_kernel<<<nblk(a.V[0] * 36, 256), 256, 0, st>>>(eps_unit, dEu, a.tgt, a.V[0]);
  forward(P, a, st);
  // loss on the zero-mean parts of prediction and target (the prediction's mean is discarded when it is
  // used, and the target's is zero up to rounding); y - t is then mean-free, so dy needs no projection
  double* sums = a.scal + 48;   // 36 channel sums of y, then 36 of t
  CKW(cudaMemsetAsync(a.scal, 0, 2 * sizeof(double), st));
  CKW(cudaMemsetAsync(sums, 0, 72 * sizeof(double), st));
  chan_sum_kernel<<<256, 256, 0, st>>>(a.y, sums, a.V[0]);
  chan_sum_kernel<<<256, 256, 0, st>>>(a.tgt, sums + 36, a.V[0]);
  center_kernel<<<nblk(a.V[0] * 36, 256), 256, 0, st>>>(a.y, sums, a.V[0]);
  center_kernel<<<nblk(a.V[0] * 36, 256), 256, 0, st>>>(a.tgt, sums + 36, a.V[0]);
  sumsq_kernel<<<512, 256, 0, st>>>(a.tgt, a.scal + 1, a.V[0] * 36);
  rel_mse_kernel<<<512, 256, 0, st>>>(a.y, a.tgt, a.scal + 1, a.dy, a.scal, a.V[0] * 36, 1e-6);
  backward(P, a, st);
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<nblk(kNParams, 256), 256, 0, st>>>(P.p, P.g, P.m1, P.m2, kNParams, lr, b1, b2, 1e-8f, c1, c2);
  for (int l = 0; l < kConvs; ++l)
    refresh_bf16_kernel<<<nblk(kConvW, 256), 256, 0, st>>>(convW(P, P.p, l), P.Wf + l * kConvW, P.Wb + l * kConvW);
  CKW(cudaGetLastError());
  if (loss_out) {
    CKW(cudaMemcpyAsync(loss_out, a.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKW(cudaStreamSynchronize(st));
    return tc05_check();
  }
  return LAT_OK;
}

extern "C" int lat_wsnet_get_activation(const void* work, size_t work_bytes, int n, int which, float* host_out,
                                        void* stream) {
  Acts a;
  if (int rc = prepare((void*)work, work_bytes, n, a)) return rc;
  // which: 0 x0, 1..4 s0..s3, 5..7 p1..p3, 8 i0, 9 u0, 10 i1, 11 u1, 12 i2, 13 u2
  const bf16* src = nullptr;
  int level = 0;
  if (which == 0) src = a.x0;
  else if (which <= 4) src = a.s[which - 1], level = which - 1;
  else if (which <= 7) src = a.p[which - 4], level = which - 4;
  else if (which <= 13) {
    const int l = (which - 8) / 2;
    src = ((which - 8) % 2) ? a.u[l] : a.i_[l];
    level = l;
  } else {
    return lat_fail(LAT_ERR_ARG, "lat_wsnet_get_activation: which not in 0..13");
  }
  const int64_t cnt = a.V[level] * 32;
  std::vector<uint16_t> tmp(cnt);
  cudaStream_t st = (cudaStream_t)stream;
  CKW(cudaMemcpyAsync(tmp.data(), src, cnt * 2, cudaMemcpyDeviceToHost, st));
  CKW(cudaStreamSynchronize(st));
  if (int rc = tc05_check()) return rc;
  for (int64_t i = 0; i < cnt; ++i) {
    const uint32_t b = (uint32_t)tmp[i] << 16;
    float f;
    memcpy(&f, &b, 4);
    host_out[i] = f;
  }
  return LAT_OK;
}

namespace {
__global__ void start_filter_kernel(double* out, const double* g2, const double* e0, double a, double b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a * g2[i] - b * e0[i];
}
}  // namespace

extern "C" int lattice_start_filter(double* out, const double* eps_g2, const double* eps0, double rho, size_t count,
                                    void* stream) {
  if (!out || !eps_g2 || !eps0) return lat_fail(LAT_ERR_ARG, "lattice_start_filter: NULL");
  if (!(rho >= 0.0 && rho < 1.0)) return lat_fail(LAT_ERR_ARG, "lattice_start_filter: rho not in [0, 1)");
  if (count == 0) return LAT_OK;
  const double a = 1.0 / (1.0 - rho * rho), b = rho * rho * a;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
  start_filter_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, eps_g2, eps0, a, b, count);
  CKW(cudaGetLastError());
  return LAT_OK;
}

extern "C" int lat_wsnet_predict(const void* params, const uint8_t* phase, const float* table, int n,
                                 const double* E, int n_loads, double* eps0, void* work, size_t work_bytes,
                                 void* stream) {
  Acts a;
  if (int rc = prepare(work, work_bytes, n, a)) return rc;
  if (n_loads < 1 || n_loads > 6) return lat_fail(LAT_ERR_ARG, "lat_wsnet_predict: n_loads not in 1..6");
  cudaStream_t st = (cudaStream_t)stream;
  features_kernel<<<nblk(a.V[0] * 32, 256), 256, 0, st>>>(phase, table, a.x0, a.V[0]);
  forward(view((void*)params), a, st);
  double* sums = a.scal + 8;
  double* dE = a.scal + 8 + 36;
  CKW(cudaMemsetAsync(sums, 0, 36 * sizeof(double), st));
  CKW(cudaMemcpyAsync(dE, E, n_loads * 6 * sizeof(double), cudaMemcpyHostToDevice, st));
  chan_sum_kernel<<<256, 256, 0, st>>>(a.y, sums, a.V[0]);
  predict_strain_kernel<<<nblk(a.V[0] * 6 * n_loads, 256), 256, 0, st>>>(a.y, sums, dE, n_loads, eps0, a.V[0]);
  CKW(cudaGetLastError());
  return LAT_OK;
}
