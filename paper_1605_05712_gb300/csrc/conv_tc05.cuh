// conv_tc05.cuh -- the 3x3x3 convolution of the warm-start network on the fifth-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), included by warmstart.cu.
//
// Implicit GEMM per block of 128 consecutive voxels (the MMA's M): D[v][co] = sum over the 27 taps and the
// 32 input channels of A_t[v][ci] W[t][ci][co], as 27 x 2 MMAs of M = 128, N = 32, K = 16 (BF16 operands,
// FP32 accumulator in 32 TMEM columns).  Both operands are read from shared memory in the canonical
// no-swizzle K-major layout: "core matrices" of 8 rows x 16 bytes (8 rows x 8 BF16 along K) stored as 128
// contiguous bytes; the descriptor's stride-byte offset (SBO) steps to the next 8 rows, its leading-byte
// offset (LBO) to the next 8 elements of K.
//
// A (activations): staged as [channel group cg (4 x 8 channels)][row][voxel x][8 channels], 16 bytes per
// (cg, row, x).  Consecutive voxels are 16 bytes apart, so the 8 rows of a core matrix are 8 consecutive
// voxels and SBO = 128; a shift of the tap by one voxel is a 16-byte shift of the start address (no copy per
// tap).  Two kernels:
//   - conv3_tc05_ring_kernel, rows of 128 voxels: one row per tile with its periodic halo, a sliding
//     window of staged rows over consecutive tiles (below);
//   - conv3_tc05_kernel, rows of 16, 32 or 64 voxels: a tile is k = 128 / n2 consecutive rows of one z
//     layer, staged as rows of exactly n2 voxels so that the k rows follow each other at the MMA's uniform
//     stride; the x shift is built into three staged copies, one per dx.  The taps run as three rounds
//     per tile, one per dz: stage that layer's rows, issue its 18 MMAs from one thread, commit them to an
//     mbarrier, wait, then stage the next round into the same buffer.
// Every mbarrier wait has an iteration limit, then an error flag and NaN outputs: no hang.
// B (weights): all 27 taps staged once as [tap][k group (4)][co (32)][8 ci]: SBO = 128, LBO = 512.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tc05 {

__device__ int g_timeout;   // set when an mbarrier wait ran out (the outputs of that block are NaN)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units, descriptor version 1,
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kIdescBf16M128N32 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescBf16M128N32), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(bar), "r"(phase)
      : "memory");
  return done != 0;
}
// waits for the given phase of the barrier; false after the iteration limit (about a second)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < (1 << 24); ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
// 16-byte asynchronous copy global -> shared (many in flight per thread; completed by cp_wait_all)
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane (32x32b shape, warp w reads lanes 32 w .. 32 w + 31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kWBytes = 27 * 4 * 32 * 16;          // all 27 taps of B in the canonical layout
constexpr int kTmemCols = 32;                     // the FP32 accumulator: N = 32 columns x 128 lanes

// staged activation bytes of conv3_tc05_kernel for rows of n2 < 128 voxels: 3 copies x 4 channel groups x
// (k + 2) rows x n2 voxels x 16 bytes
__host__ __device__ inline int a_bytes(int n2) { return 3 * 4 * (128 / n2 + 2) * n2 * 16; }
// its dynamic shared memory: weights, activations, the mbarrier and the TMEM address slot
__host__ __device__ inline size_t smem_bytes(int n2) { return (size_t)kWBytes + (size_t)a_bytes(n2) + 16; }

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// in: [V][32] BF16 (channels last); W: [27][32 n][32 k] BF16 (n the output channel); out_mode 0: BF16
// leaky-ReLU(acc + bias), 1: FP32 acc; neg: taps at -offset (backward data).  Blocks of 128 threads,
// persistent: a block stages the weights once and then loops over tiles of 128 consecutive voxels
// (blockIdx.x, + gridDim.x, ...); n2 in {16, 32, 64}, n1 divisible by 128 / n2; smem_bytes(n2) of
// dynamic shared memory (86-105 KB: two blocks per SM).
__global__ void __launch_bounds__(128) conv3_tc05_kernel(const __nv_bfloat16* __restrict__ in,
                                                         const __nv_bfloat16* __restrict__ W,
                                                         const float* __restrict__ bias, void* out, int n0, int n1,
                                                         int n2, int out_mode, int neg, float leak) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = 128 / n2;                          // rows per tile
  const int nrow = k + 2;                          // staged rows per copy
  unsigned char* wsm = smem;
  unsigned char* asmem = smem + kWBytes;
  const int abytes = 3 * 4 * nrow * n2 * 16;       // = a_bytes(n2)
  uint64_t* bar = (uint64_t*)(asmem + abytes);     // 16-byte aligned
  uint32_t* tslot = (uint32_t*)(bar + 1);

  for (int i = tid; i < 27 * 32 * 4; i += 128) {   // B: chunk (tap, co, kg) -> [tap][kg][co]
    const int kg = i & 3, co = (i >> 2) & 31, tap = i >> 7;
    cp16(wsm + ((tap * 4 + kg) * 32 + co) * 16, (const uint4*)(W + ((size_t)tap * 32 + co) * 32) + kg);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *(volatile uint32_t*)tslot;
  const int64_t ntiles = (int64_t)n0 * n1 * n2 / 128;
  const int64_t nq = 3 * ((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // this block's rounds
  auto tile_of = [&](int64_t q) { return (int64_t)blockIdx.x + (q / 3) * gridDim.x; };
  // copies of round q (tile, source layer z + r - 1) into buffer q & 1
  auto stage = [&](int64_t q) {
    const int64_t tile = tile_of(q);
    const int r = (int)(q % 3);
    unsigned char* buf = asmem;
    const int row0 = (int)(tile * 128 / n2);
    const int z = row0 / n1, y0 = row0 - z * n1;
    const int zz = wrapi(z + r - 1, n0);
    // copy c holds the voxels shifted by c - 1; staged row j = source row y0 + j - 1
    for (int i = tid; i < 3 * 4 * nrow * n2; i += 128) {
      const int x = i & (n2 - 1);
      int rest = i / n2;
      const int j = rest % nrow;
      rest /= nrow;
      const int cg = rest & 3, c = rest >> 2;
      const int yy = wrapi(y0 + j - 1, n1), xsrc = wrapi(x + c - 1, n2);
      cp16(buf + (((c * 4 + cg) * nrow + j) * n2 + x) * 16, (const uint4*)(in + ((size_t)(zz * n1 + yy) * n2 + xsrc) * 32) + cg);
    }
    cp_commit();
  };
  // the 18 products of round q (one thread), then their commit to the mbarrier (phase q)
  auto issue = [&](int64_t q) {
    const int r = (int)(q % 3), sz = r - 1;
    const uint32_t base = smem_u32(asmem);
    for (int sy = -1; sy <= 1; ++sy)
      for (int sx = -1; sx <= 1; ++sx) {
        const int tap = neg ? (1 - sz) * 9 + (1 - sy) * 3 + (1 - sx) : (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
        const uint32_t lbo = (uint32_t)(nrow * n2 * 16);
        const uint32_t a0 = base + (uint32_t)((((sx + 1) * 4) * nrow + (sy + 1)) * n2 * 16);
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ad = sdesc(a0 + 2u * ks * lbo, lbo, 128u);
          const uint64_t bd = sdesc(smem_u32(wsm) + (uint32_t)(((tap * 4 + 2 * ks) * 32) * 16), 512u, 128u);
          mma_bf16(tmem, ad, bd, (r > 0 || sy > -1 || sx > -1 || ks > 0) ? 1u : 0u);
        }
      }
    mma_commit(smem_u32(bar));
  };
  // the finished accumulator of a tile -> bias, activation, store
  auto epilogue = [&](int64_t tile, bool ok) {
    float acc[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
    if (!ok) {
      atomicExch(&g_timeout, 1);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = __int_as_float(0x7fc00000);
    }
    const int64_t v = tile * 128 + warp * 32 + lane;
    if (out_mode == 0) {
      uint4 pk[4];
      __nv_bfloat16* hb = (__nv_bfloat16*)pk;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float t = acc[i] + bias[i];
        hb[i] = __float2bfloat16(t > 0.f ? t : leak * t);
      }
      uint4* dst = (uint4*)((__nv_bfloat16*)out + v * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = pk[q];
    } else {
      float4* dst = (float4*)((float*)out + v * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
  };
  bool ok = true;
  for (int64_t q = 0; q < nq; ++q) {   // stage, multiply, wait: one round after another
    stage(q);                          // (the first copy group also holds the weights)
    cp_wait_group<0>();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue(q);
    }
    if (!mbar_wait(smem_u32(bar), (uint32_t)(q & 1))) ok = false;
    if (q % 3 == 2) {
      tc_fence_after();
      epilogue(tile_of(q), ok);
      ok = true;
    }
    tc_fence_before();   // the buffer and the accumulator are free for the next round
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace tc05

namespace tc05 {

// Rows of 128 voxels with a sliding window.  A work item is R consecutive rows (y0 .. y0 + R - 1) of one z
// layer; a block walks its items' rows in order and keeps, per source layer dz, a ring of 4 staged rows
// (slot = row mod 4): tile y needs rows y - 1, y, y + 1, and the copies of row y + 2 (for tile y + 1) run
// while the tensor cores work on tile y -- 3 new rows per tile instead of 9.  Two accumulators of 32 TMEM
// columns alternate, so the epilogue of tile y - 1 overlaps the products of tile y.
//   staged row (dz layer d, slot s): [d][cg][s][x (n2 + 2: periodic halo)] x 16 bytes
//   tap (dz, dy, dx): A = row slot((y + dy) mod 4) of layer d, start + (dx + 1) 16 bytes, LBO = 4 (n2 + 2) 16
constexpr int kRingRows = 16;   // R: rows per work item (1024 items at 128^3: 6.7 per block)
__host__ __device__ inline size_t ring_smem_bytes(int n2) {
  return (size_t)kWBytes + (size_t)3 * 4 * 4 * (n2 + 2) * 16 + 16;
}

__global__ void __launch_bounds__(128) conv3_tc05_ring_kernel(const __nv_bfloat16* __restrict__ in,
                                                              const __nv_bfloat16* __restrict__ W,
                                                              const float* __restrict__ bias, void* out, int n0,
                                                              int n1, int n2, int out_mode, int neg, float leak) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int xlen = n2 + 2;
  unsigned char* wsm = smem;
  unsigned char* rsm = smem + kWBytes;
  const int rbytes = 3 * 4 * 4 * xlen * 16;
  uint64_t* bar = (uint64_t*)(rsm + rbytes);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int R = n1 < kRingRows ? n1 : kRingRows;
  const int nchunk = n1 / R;
  const int64_t nitems = (int64_t)n0 * nchunk;

  for (int i = tid; i < 27 * 32 * 4; i += 128) {
    const int kg = i & 3, co = (i >> 2) & 31, tap = i >> 7;
    cp16(wsm + ((tap * 4 + kg) * 32 + co) * 16, (const uint4*)(W + ((size_t)tap * 32 + co) * 32) + kg);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *(volatile uint32_t*)tslot;

  // the copies of source row y (wrapped) of layer z + d - 1 into its ring slot, all three layers
  auto stage_row = [&](int z, int y) {
    const int yy = wrapi(y, n1), s = y & 3;
    for (int i = tid; i < 3 * 4 * xlen; i += 128) {
      const int xv = i % xlen, rest = i / xlen, cg = rest & 3, d = rest >> 2;
      const int zz = wrapi(z + d - 1, n0), xsrc = wrapi(xv - 1, n2);
      cp16(rsm + (((d * 4 + cg) * 4 + s) * xlen + xv) * 16, (const uint4*)(in + ((size_t)(zz * n1 + yy) * n2 + xsrc) * 32) + cg);
    }
  };
  // the 54 products of tile (z, y) into accumulator a, then their commit
  auto issue = [&](int y, int a) {
    const uint32_t base = smem_u32(rsm), lbo = (uint32_t)(4 * xlen * 16);
    bool first = true;
    for (int sz = -1; sz <= 1; ++sz)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          const int tap = neg ? (1 - sz) * 9 + (1 - sy) * 3 + (1 - sx) : (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
          const uint32_t a0 = base + (uint32_t)(((((sz + 1) * 4) * 4 + ((y + sy) & 3)) * xlen + (sx + 1)) * 16);
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ad = sdesc(a0 + 2u * ks * lbo, lbo, 128u);
            const uint64_t bd = sdesc(smem_u32(wsm) + (uint32_t)(((tap * 4 + 2 * ks) * 32) * 16), 512u, 128u);
            mma_bf16(tmem + (uint32_t)(a * kTmemCols), ad, bd, first ? 0u : 1u);
            first = false;
          }
        }
    mma_commit(smem_u32(bar));
  };
  auto epilogue = [&](int64_t vrow, int a, bool ok) {   // vrow: first voxel of the tile's row
    float acc[32];
    tmem_ld32(tmem + (uint32_t)(a * kTmemCols) + ((uint32_t)(warp * 32) << 16), acc);
    if (!ok) {
      atomicExch(&g_timeout, 1);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = __int_as_float(0x7fc00000);
    }
    const int64_t v = vrow + warp * 32 + lane;
    if (out_mode == 0) {
      uint4 pk[4];
      __nv_bfloat16* hb = (__nv_bfloat16*)pk;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float t = acc[i] + bias[i];
        hb[i] = __float2bfloat16(t > 0.f ? t : leak * t);
      }
      uint4* dst = (uint4*)((__nv_bfloat16*)out + v * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = pk[q];
    } else {
      float4* dst = (float4*)((float*)out + v * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
  };

  int64_t t = 0;                // tiles issued by this block: tile t completes mbarrier phase t
  int64_t pend_v = -1;          // the issued tile still waiting for its epilogue (first voxel), and its
  int pend_a = 0;               // accumulator
  bool ok = true;
  auto finish_pending = [&]() {
    if (pend_v < 0) return;
    if (!mbar_wait(smem_u32(bar), (uint32_t)((t - 1) & 1))) ok = false;
    tc_fence_after();
    epilogue(pend_v, pend_a, ok);
    ok = true;
    pend_v = -1;
    tc_fence_before();
  };
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int z = (int)(w / nchunk), yb = (int)(w % nchunk) * R;
    // the previous item's last tile reads ring slots this item's first rows go to: finish it first
    finish_pending();
    __syncthreads();
    stage_row(z, yb - 1);
    stage_row(z, yb);
    stage_row(z, yb + 1);
    cp_commit();
    for (int i = 0; i < R; ++i, ++t) {
      const int y = yb + i;
      finish_pending();   // tile t - 1: its products are done, so ring slot (y + 2) mod 4 is free
      if (i + 1 < R) {
        stage_row(z, y + 2);
        cp_commit();
        cp_wait_group<1>();   // this thread's copies of rows y - 1 .. y + 1 have landed
      } else {
        cp_wait_group<0>();
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue(y, (int)(t & 1));
      }
      pend_v = ((int64_t)z * n1 + y) * n2;
      pend_a = (int)(t & 1);
    }
  }
  finish_pending();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
}

}  // namespace tc05
