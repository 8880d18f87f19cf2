// The observable sums of one lattice's macroscopic fields (Sec. III: the masses of Eq. 16
// summed, |u|max of Eq. 46, the moments of the rho^N = 0 crossings for the circle fit of the
// contact angle, the Laplace pressure sums, a non-finite flag), in FP64: a grid-stride pass
// with warp-shuffle and shared-memory reductions into one row of partials per block, then a
// one-block pass over the rows in a fixed order (deterministic results).
//
// Shared by lbcg_observables (the handle's pitched node arrays) and
// lbcg_field_moments_noalloc (a caller's dense [ny][nx] fields), so both reduce identically.
#pragma once

#include "lbcg_internal.h"

namespace lbcg {

// the public mask bits of lbcg_field_moments_noalloc are the node flags of the handle
static_assert(F_SOLID == LBCG_MASK_SOLID && F_NEAR == LBCG_MASK_NO_FIT, "mask bits must match the node flags");

__device__ __forceinline__ double obs_rn(double r, double b) { return (r - b) / (r + b); }
// slots reduced by maximum (|u|max, the non-finite flag); the others are sums
__device__ __forceinline__ bool obs_max_slot(int q) { return q == 2 || q == 16; }

// Partial sums over the nodes this block visits, written to partials[blockIdx.x * kObsQ + q]:
//   q0, q1   sum of rho_R, rho_B over fluid nodes
//   q2       max |u|
//   q3..q11  n, Sx, Sy, Sxx, Syy, Sxy, Szx, Szy, Sz of the interface points: rho^N = 0
//            crossings, linearly interpolated on the links (x,y)-(x+1,y) and (x,y)-(x,y+1)
//            between fluid nodes not flagged F_NEAR, relative to (nx/2, ny/2), z = x^2 + y^2
//   q12..q15 sum and count of rho/3 over rho^N > 0.9, and over rho^N < -0.9
//   q16      1 if some fluid density is not finite
// Fields and flags of node (x, y) sit at index y * pitch + x.  Launch with 256 threads.
__device__ __forceinline__ void obs_block_partials(const double* __restrict__ rR, const double* __restrict__ rB,
                                                   const double* __restrict__ uX, const double* __restrict__ uY,
                                                   const uint8_t* __restrict__ fl, int nx, int ny, long long pitch,
                                                   double* __restrict__ partials) {
  const long long nn = (long long)nx * ny;
  double q[kObsQ];
#pragma unroll
  for (int i = 0; i < kObsQ; ++i) q[i] = 0.0;
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
    const long long k = (long long)y * pitch + x;
    const uint8_t f = fl[k];
    if (f & F_SOLID) continue;
    const double r = rR[k], b = rB[k];
    q[0] += r;
    q[1] += b;
    q[2] = fmax(q[2], sqrt(uX[k] * uX[k] + uY[k] * uY[k]));
    const double rho = r + b;
    if (!isfinite(rho)) q[16] = 1.0;
    const double rn = obs_rn(r, b);
    if (rn > 0.9) {
      q[12] += rho / 3.0;
      q[13] += 1.0;
    } else if (rn < -0.9) {
      q[14] += rho / 3.0;
      q[15] += 1.0;
    }
    if (f & F_NEAR) continue;
    if (x + 1 < nx && !(fl[k + 1] & (F_SOLID | F_NEAR))) {
      const double b2 = obs_rn(rR[k + 1], rB[k + 1]);
      if ((rn >= 0) != (b2 >= 0)) add_point(x + rn / (rn - b2) - hx, y - hy);
    }
    if (y + 1 < ny && !(fl[k + pitch] & (F_SOLID | F_NEAR))) {
      const double b2 = obs_rn(rR[k + pitch], rB[k + pitch]);
      if ((rn >= 0) != (b2 >= 0)) add_point(x - hx, y + rn / (rn - b2) - hy);
    }
  }
  __shared__ double sh[kObsQ][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kObsQ; ++k) {
    double v = q[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = obs_max_slot(k) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kObsQ) {
    const int k = threadIdx.x;
    double v = sh[k][0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) v = obs_max_slot(k) ? fmax(v, sh[k][w]) : v + sh[k][w];
    partials[blockIdx.x * kObsQ + k] = v;
  }
}

// out[q] = the rows of `partials` combined in block order (thread q of one block)
__device__ __forceinline__ void obs_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kObsQ) return;
  double v = partials[k];
  for (int b = 1; b < nblocks; ++b) {
    const double w = partials[b * kObsQ + k];
    v = obs_max_slot(k) ? fmax(v, w) : v + w;
  }
  out[k] = v;
}

}  // namespace lbcg
