// lbcg_field_moments_noalloc: the observables reduction of lbcg_obs.cu for callers that
// cannot allocate device memory, e.g. code running under a fixed memory budget or a custom
// allocator that forbids cudaMalloc, or a host thread that must not take the driver's
// allocation locks.  The per-block partial sums live in a file-scope device array instead of
// memory owned by a handle; the caller provides the input fields and the output buffer.
//
// The scratch is shared by every call on a device and keeps the last call's contents.  Each
// call's first kernel overwrites all kNoallocBlocks rows before its second kernel reads them,
// so nothing has to be cleared between calls.  Calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on the scratch and must be serialised by the caller.
#include <cstdio>
#include <mutex>

#include "../../include/lbcg.h"
#include "lbcg_internal.h"

namespace {

constexpr int kNoallocBlocks = 304;  // 2 x 152 SMs; blocks stride over the whole lattice
constexpr int kNoallocQ = 17;        // reduced quantities, see include/lbcg.h
constexpr int kMaxDevices = 64;

// 304 x 17 doubles = 41,344 bytes, resident on every GPU that loads the library until exit.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocBlocks * kNoallocQ];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double na_rn(double r, double b) { return (r - b) / (r + b); }
__device__ __forceinline__ bool na_max_slot(int q) { return q == 2 || q == 16; }

__global__ void __launch_bounds__(256) k_noalloc_partial(const double* __restrict__ fields,
                                                         const uint8_t* __restrict__ mask, int nx, int ny,
                                                         double* __restrict__ partials) {
  const long long nn = (long long)nx * ny;
  const double* rR = fields;
  const double* rB = fields + nn;
  const double* uX = fields + 2 * nn;
  const double* uY = fields + 3 * nn;
  double q[kNoallocQ];
#pragma unroll
  for (int i = 0; i < kNoallocQ; ++i) q[i] = 0.0;
  const double hx = 0.5 * nx, hy = 0.5 * ny;
  auto add_point = [&](double x, double y) {
    const double z = x * x + y * y;
    q[3] += 1.0;
    q[4] += x;
    q[5] += y;
    q[6] += x * x;
    q[7] += y * y;
    q[8] += x * y;
    q[9] += z * x;
    q[10] += z * y;
    q[11] += z;
  };
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
    const uint8_t m = mask[i];
    if (m & LBCG_MASK_SOLID) continue;
    const double r = rR[i], b = rB[i];
    q[0] += r;
    q[1] += b;
    q[2] = fmax(q[2], sqrt(uX[i] * uX[i] + uY[i] * uY[i]));
    const double rho = r + b;
    if (!isfinite(rho)) q[16] = 1.0;
    const double rn = na_rn(r, b);
    if (rn > 0.9) {
      q[12] += rho / 3.0;
      q[13] += 1.0;
    } else if (rn < -0.9) {
      q[14] += rho / 3.0;
      q[15] += 1.0;
    }
    if (m & LBCG_MASK_NO_FIT) continue;
    if (x + 1 < nx && !(mask[i + 1] & (LBCG_MASK_SOLID | LBCG_MASK_NO_FIT))) {
      const double b2 = na_rn(rR[i + 1], rB[i + 1]);
      if ((rn >= 0) != (b2 >= 0)) add_point(x + rn / (rn - b2) - hx, y - hy);
    }
    if (y + 1 < ny && !(mask[i + nx] & (LBCG_MASK_SOLID | LBCG_MASK_NO_FIT))) {
      const double b2 = na_rn(rR[i + nx], rB[i + nx]);
      if ((rn >= 0) != (b2 >= 0)) add_point(x - hx, y + rn / (rn - b2) - hy);
    }
  }
  __shared__ double sh[kNoallocQ][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNoallocQ; ++k) {
    double v = q[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = na_max_slot(k) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNoallocQ) {
    const int k = threadIdx.x;
    double v = sh[k][0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) v = na_max_slot(k) ? fmax(v, sh[k][w]) : v + sh[k][w];
    partials[blockIdx.x * kNoallocQ + k] = v;
  }
}

__global__ void __launch_bounds__(32) k_noalloc_final(const double* __restrict__ partials, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kNoallocQ) return;
  double v = partials[k];
  for (int b = 1; b < kNoallocBlocks; ++b) {
    const double w = partials[b * kNoallocQ + k];
    v = na_max_slot(k) ? fmax(v, w) : v + w;
  }
  out[k] = v;
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(LBCG_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBCG_E_UNSUPPORTED, "lbcg_field_moments_noalloc: device index >= 64");
  double* scratch = nullptr;
  {
    // set-up once per device, with that device current: the host-side name of the array
    // is not a device address, so ask the runtime for the address on this device
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(LBCG_E_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_partial<<<kNoallocBlocks, 256, 0, st>>>(fields, mask, nx, ny, scratch);
  k_noalloc_final<<<1, 32, 0, st>>>(scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(LBCG_E_CUDA, cudaGetErrorString(e));
  return LBCG_OK;
}
