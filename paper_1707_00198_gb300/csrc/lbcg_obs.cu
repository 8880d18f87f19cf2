// Observable reductions (Sec. III: Eq. 46, the contact angle of Tables I and III, the finger
// length and contact-line displacement of Sec. III.D) over one lattice's macroscopic fields
// rho_R, rho_B, u_x, u_y, in FP64: warp-shuffle, then shared-memory, then a one-block pass
// over the per-block partials (a fixed order, so the result is deterministic).
#include "lbcg_obs_reduce.cuh"

namespace lbcg {

size_t obs_partials_doubles() { return size_t(kObsBlocks) * kObsQ; }

__global__ void __launch_bounds__(256) k_obs_partial(const LatDev* __restrict__ lats, int lat,
                                                     const double* __restrict__ macro, long long node_total,
                                                     const uint8_t* __restrict__ flags, double* __restrict__ partials) {
  const LatDev& L = lats[lat];
  obs_block_partials(macro + L.node_off, macro + node_total + L.node_off, macro + 2 * node_total + L.node_off,
                     macro + 3 * node_total + L.node_off, flags + L.node_off, L.nx, L.ny, L.pitch, partials);
}

__global__ void __launch_bounds__(32) k_obs_final(const double* __restrict__ partials, int nblocks,
                                                  double* __restrict__ out) {
  obs_final(partials, nblocks, out);
}

// First rho^N >= 0 -> rho^N < 0 change along a row (block 0: mean of rows r0, r1 -> the finger
// tip; blocks 1, 2: rows c0, c1 -> the contact line); -1 if none.
__global__ void __launch_bounds__(256) k_obs_rows(const LatDev* __restrict__ lats, int lat,
                                                  const double* __restrict__ macro, long long node_total,
                                                  const uint8_t* __restrict__ flags, int r0, int r1, int c0, int c1,
                                                  double* __restrict__ out) {
  const LatDev& L = lats[lat];
  const int ra = blockIdx.x == 0 ? r0 : (blockIdx.x == 1 ? c0 : c1);
  const int rb = blockIdx.x == 0 ? r1 : ra;
  const bool valid = ra >= 0 && ra < L.ny && rb >= 0 && rb < L.ny;
  const uint8_t* fl = flags + L.node_off;
  const double* rR = macro + L.node_off;
  const double* rB = macro + node_total + L.node_off;
  auto rn_at = [&](int x, int y) {
    const long long k = (long long)y * L.pitch + x;
    return (fl[k] & F_SOLID) ? 0.0 : obs_rn(rR[k], rB[k]);
  };
  auto prof = [&](int x) { return 0.5 * (rn_at(x, ra) + rn_at(x, rb)); };
  int best = 0x7fffffff;
  if (valid) {
    for (int x = threadIdx.x; x + 1 < L.nx; x += blockDim.x) {
      if (prof(x) >= 0 && prof(x + 1) < 0) {
        best = x;
        break;
      }
    }
  }
  __shared__ int sb[8];
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = sb[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = min(m, sb[w]);
    double res = -1.0;
    if (m != 0x7fffffff) {
      const double a = prof(m), b = prof(m + 1);
      res = m + a / (a - b);
    }
    out[kObsQ + blockIdx.x] = res;
  }
}

cudaError_t launch_observables(const LatDev* lats, int lat, int nx, int ny, const double* macro,
                               long long node_total, const uint8_t* flags, int tip0, int tip1, int cl0, int cl1,
                               double* partials, double* out, cudaStream_t st) {
  (void)nx;
  (void)ny;
  k_obs_partial<<<kObsBlocks, 256, 0, st>>>(lats, lat, macro, node_total, flags, partials);
  k_obs_final<<<1, 32, 0, st>>>(partials, kObsBlocks, out);
  k_obs_rows<<<kObsRows, 256, 0, st>>>(lats, lat, macro, node_total, flags, tip0, tip1, cl0, cl1, out);
  return cudaGetLastError();
}

}  // namespace lbcg

// ------------------------------------------------------------------ steady-state diagnostics
// Eq. 45 and the masses of Eq. 47 in one pass over one lattice's macroscopic fields:
// q0, q1 = max |u_x - u_x'|, max |u_y - u_y'| against the stored velocity (when there is one),
// which each thread then replaces by the current velocity of its nodes; q2..q5 = rho_R and
// rho_B summed inside / outside the circle C (node (x, y) inside when (x-cx)^2 + (y-cy)^2 < r^2).
namespace lbcg {

namespace {

constexpr int kDiagQ = 6;
__device__ __forceinline__ bool diag_max_slot(int q) { return q < 2; }

__global__ void __launch_bounds__(256) k_diag_partial(const LatDev* __restrict__ lats, int lat,
                                                      const double* __restrict__ macro, long long node_total,
                                                      const uint8_t* __restrict__ flags, double* __restrict__ usnap,
                                                      int have_snap, double cx, double cy, double r2,
                                                      double* __restrict__ partials) {
  const LatDev& L = lats[lat];
  const int nx = L.nx, ny = L.ny;
  const long long nn = (long long)nx * ny;
  const uint8_t* fl = flags + L.node_off;
  const double* rR = macro + L.node_off;
  const double* rB = macro + node_total + L.node_off;
  const double* uX = macro + 2 * node_total + L.node_off;
  const double* uY = macro + 3 * node_total + L.node_off;
  double* sX = usnap + L.node_off;
  double* sY = usnap + node_total + L.node_off;
  double q[kDiagQ];
#pragma unroll
  for (int k = 0; k < kDiagQ; ++k) q[k] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
    const long long k = (long long)y * L.pitch + x;
    if (fl[k] & F_SOLID) continue;
    const double ux = uX[k], uy = uY[k];
    if (have_snap) {
      q[0] = fmax(q[0], fabs(ux - sX[k]));
      q[1] = fmax(q[1], fabs(uy - sY[k]));
    }
    sX[k] = ux;
    sY[k] = uy;
    const double dx = x - cx, dy = y - cy;
    const bool in = dx * dx + dy * dy < r2;
    q[in ? 2 : 3] += rR[k];
    q[in ? 4 : 5] += rB[k];
  }
  __shared__ double sh[kDiagQ][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kDiagQ; ++j) {
    double v = q[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = diag_max_slot(j) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[j][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagQ) {
    const int j = threadIdx.x;
    double v = sh[j][0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) v = diag_max_slot(j) ? fmax(v, sh[j][w]) : v + sh[j][w];
    partials[blockIdx.x * kDiagQ + j] = v;
  }
}

__global__ void __launch_bounds__(32) k_diag_final(const double* __restrict__ partials, int nblocks,
                                                   double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= kDiagQ) return;
  double v = partials[j];
  for (int b = 1; b < nblocks; ++b) {
    const double w = partials[b * kDiagQ + j];
    v = diag_max_slot(j) ? fmax(v, w) : v + w;
  }
  out[j] = v;
}

}  // namespace

cudaError_t launch_diagnostics(const LatDev* lats, int lat, const double* macro, long long node_total,
                               const uint8_t* flags, double* usnap, bool have_snap, double cx, double cy, double r,
                               double* partials, double* out, cudaStream_t st) {
  k_diag_partial<<<kObsBlocks, 256, 0, st>>>(lats, lat, macro, node_total, flags, usnap, have_snap ? 1 : 0, cx, cy,
                                             r * r, partials);
  k_diag_final<<<1, 32, 0, st>>>(partials, kObsBlocks, out);
  return cudaGetLastError();
}

}  // namespace lbcg
