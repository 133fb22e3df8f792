// gather.cu -- subsampling and rearrangement of fields between patterns (Sec. 2.1 subpatterns,
// Sec. 2.2 pattern-congruent matrices, Sec. 5.2): out[f][s] = in[f][map[s]] with the map of
// lattice_gather_map.  A plain HBM-bound copy through an index table.
#include <stdint.h>

#include <string>

#include "internal.h"

namespace {

// each thread: 4 points per step, map entries loaded once for all planes, every load of a step issued
// before its stores (the map load and the dependent source load would otherwise serialize)
template <typename T>
__global__ void gather_kernel(const T* __restrict__ in, T* __restrict__ out, const int32_t* __restrict__ map,
                              int64_t n, int n_fields, int64_t in_plane, int64_t out_plane) {
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * U) {
    int32_t src[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      src[u] = i < n ? __ldg(map + i) : -1;
    }
    for (int f = 0; f < n_fields; ++f) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (src[u] >= 0) v[u] = in[(int64_t)f * in_plane + src[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (src[u] >= 0) out[(int64_t)f * out_plane + i0 + u * stride] = v[u];
    }
  }
}

template <typename T>
void launch(const void* in, void* out, const int32_t* map, int64_t n, int n_fields, int64_t in_plane,
            int64_t out_plane, cudaStream_t st) {
  int64_t nb = (n + 1023) / 1024;
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb < 1) nb = 1;
  gather_kernel<T><<<(unsigned)nb, 256, 0, st>>>((const T*)in, (T*)out, map, n, n_fields, in_plane, out_plane);
}

}  // namespace

extern "C" int lattice_gather(const void* in, void* out, const int32_t* map, int64_t n_out, int elem_bytes,
                              int n_fields, int64_t in_plane, int64_t out_plane, void* stream) {
  if (!in || !out || !map || n_out < 0 || n_fields < 1 || n_fields > 65535)
    return lat_fail(LAT_ERR_ARG, "lattice_gather: bad argument");
  if (n_out == 0) return LAT_OK;
  if (((uintptr_t)in | (uintptr_t)out) % (uintptr_t)(elem_bytes > 0 ? elem_bytes : 1) != 0)
    return lat_fail(LAT_ERR_ARG, "lattice_gather: buffers not aligned to the element size");
  cudaStream_t st = (cudaStream_t)stream;
  switch (elem_bytes) {
    case 1: launch<uint8_t>(in, out, map, n_out, n_fields, in_plane, out_plane, st); break;
    case 2: launch<uint16_t>(in, out, map, n_out, n_fields, in_plane, out_plane, st); break;
    case 4: launch<uint32_t>(in, out, map, n_out, n_fields, in_plane, out_plane, st); break;
    case 8: launch<uint64_t>(in, out, map, n_out, n_fields, in_plane, out_plane, st); break;
    case 16: launch<uint4>(in, out, map, n_out, n_fields, in_plane, out_plane, st); break;
    default: return lat_fail(LAT_ERR_ARG, "lattice_gather: elem_bytes must be 1, 2, 4, 8 or 16");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lat_fail(LAT_ERR_CUDA, std::string("lattice_gather: ") + cudaGetErrorString(e));
  return LAT_OK;
}
