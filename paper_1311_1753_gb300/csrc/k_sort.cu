// k_sort.cu -- data layout step of the 1D path: events sorted ascending by the observable
// of the first Voigtian leaf, so that each thread's contiguous share of the events spans
// a short interval of z and the event kernel can expand w(z) once per chunk of events
// (k_1d.cu).  Sorting is a one-time permutation of the data set; the NLL is a sum over
// events and does not depend on their order, and per-event outputs are scattered back
// through the stored permutation.
#include <cub/device/device_radix_sort.cuh>

#include "gf_internal.h"
#include "launch.h"

namespace gfi {

__global__ void k_iota(int32_t* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

__global__ void k_gather(const double* __restrict__ in, const int32_t* __restrict__ perm,
                         double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}

static int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

cudaError_t sort_by_key_f64(const double* key_in, double* key_out, int32_t* perm_tmp,
                            int32_t* perm_out, int64_t n, void* temp, size_t* temp_bytes,
                            cudaStream_t st) {
  if (!temp) {  // size query only
    return cub::DeviceRadixSort::SortPairs(nullptr, *temp_bytes, key_in, key_out, perm_tmp,
                                           perm_out, n, 0, 64, st);
  }
  k_iota<<<grid_of(n), 256, 0, st>>>(perm_tmp, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cub::DeviceRadixSort::SortPairs(temp, *temp_bytes, key_in, key_out, perm_tmp, perm_out,
                                         n, 0, 64, st);
}

cudaError_t launch_gather(const double* in, const int32_t* perm, double* out, int64_t n,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (!in || !perm || !out) return cudaErrorInvalidValue;
  k_gather<<<grid_of(n), 256, 0, st>>>(in, perm, out, n);
  return cudaGetLastError();
}

}  // namespace gfi
