// lbcg_field_moments_noalloc: the observables reduction of lbcg_obs.cu for callers that
// cannot allocate device memory, e.g. code running under a fixed memory budget or a custom
// allocator that forbids cudaMalloc, or a host thread that must not take the driver's
// allocation locks.  The per-block partial sums live in a file-scope device array instead of
// memory owned by a handle; the caller provides the input fields and the output buffer.  The
// reduction itself is the one lbcg_observables runs (lbcg_obs_reduce.cuh), on a dense
// [ny][nx] layout.
//
// The scratch is shared by every call on a device and keeps the last call's contents.  Each
// call's first kernel overwrites all kObsBlocks rows before its second kernel reads them,
// so nothing has to be cleared between calls.  Calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on the scratch and must be serialised by the caller.
#include "../../include/lbcg.h"
#include "lbcg_obs_reduce.cuh"

namespace {

using lbcg::kObsBlocks;
using lbcg::kObsQ;

// 304 x 17 doubles = 41,344 bytes, resident on every GPU that loads the library until exit.
static __device__ __align__(256) double g_noalloc_scratch[kObsBlocks * kObsQ];

__global__ void __launch_bounds__(256) k_noalloc_partial(const double* __restrict__ fields,
                                                         const uint8_t* __restrict__ mask, int nx, int ny,
                                                         double* __restrict__ partials) {
  const long long nn = (long long)nx * ny;
  lbcg::obs_block_partials(fields, fields + nn, fields + 2 * nn, fields + 3 * nn, mask, nx, ny, nx, partials);
}

__global__ void __launch_bounds__(32) k_noalloc_final(const double* __restrict__ partials, double* __restrict__ out) {
  lbcg::obs_final(partials, kObsBlocks, out);
}

lbcg_status noalloc_fail(lbcg_status s, const char* msg) {
  lbcg::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" lbcg_status lbcg_field_moments_noalloc(const double* fields, const uint8_t* mask, int32_t nx, int32_t ny,
                                                  void* stream, double* out) {
  lbcg::set_last_error("");
  if (!fields || !mask || !out) return noalloc_fail(LBCG_E_ARG, "lbcg_field_moments_noalloc: NULL pointer");
  if (nx < 1 || ny < 1 || (long long)nx * ny > LBCG_NOALLOC_MAX_NODES)
    return noalloc_fail(LBCG_E_ARG,
                        "lbcg_field_moments_noalloc: lattice must have 1 <= nx*ny <= 2147483647 nodes");
  // an error left by earlier work is reported as such, not as a failure of these launches
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return noalloc_fail(LBCG_E_CUDA, "lbcg_field_moments_noalloc: a CUDA error from earlier work is pending");
  // The array's name is a host-side stand-in, not a device address: ask the runtime for the
  // address in the current context on every call (no allocation; a cached address could
  // belong to a context that no longer exists)
  void* scratch = nullptr;
  e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess) return noalloc_fail(LBCG_E_CUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_partial<<<kObsBlocks, 256, 0, st>>>(fields, mask, nx, ny, static_cast<double*>(scratch));
  k_noalloc_final<<<1, 32, 0, st>>>(static_cast<const double*>(scratch), out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(LBCG_E_CUDA, cudaGetErrorString(e));
  return LBCG_OK;
}
