// Device-side building blocks of the colour-gradient LBM step (arXiv 1707.00198, Sec. II).
//
// Layout in HBM (one "pool" per kind, lattices of a batch packed one after another):
//   populations : 18 stored values per node in the storage type S, laid out in blocks of
//                 32 nodes along x: [y][x/32][a][x%32][k] (direction a = 0..8, k = 0, 1).
//                 k = 0 holds the first stored quantity of direction a, k = 1 the second,
//                 so a direction's pair is one vector access; a node's nine pairs sit at
//                 fixed distances from one address, and a 32-node row segment is one
//                 contiguous chunk of 18 x 32 values.
//                 Direct storage (double, float): (f_{a,R}, f_{a,B}).
//                 Deviation storage (half, bfloat16): (d_a = f_a - w_a rho0,
//                 g_a = f_{a,R} - f_{a,B}), an exact linear transform of the pair.
//                 The stored state is the post-streaming state at each node: a step loads
//                 a node's own values and pushes its post-collision values to the
//                 neighbours (half-way bounce-back: back into the node's own opposite slot;
//                 across an open edge: dropped).
//   node arrays : [y][pitch] per lattice: flags (uint8), the solid-neighbour mask (uint8),
//                 and in the compute type T the corrected gradient / normal of the outermost
//                 fluid nodes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "lbcg_geom.h"

namespace lbcg {

enum { BC_PERIODIC = 0, BC_CLOSED = 1, BC_INOUT = 2 };

// threads of a k_sweep block; its strip has kSweepThreads - 4 interior columns
constexpr int kSweepThreads = 128;
__host__ __device__ constexpr int sweep_width(bool /*fp64*/) { return kSweepThreads - 4; }
// resident k_sweepf blocks per SM it is compiled for (registers <= 65536 / (128 * this)),
// FP32 storage and 16-bit storage
constexpr int kSweepFMinBlocks = 5;
constexpr int kSweepFMinBlocks16 = 7;
// set in a strip's lattice index (int4 .x): k_sweepf walks that segment from its top row down
// (its results are the same either way; neighbouring segments of a strip alternate, so both
// reach their shared boundary rows at about the same time and the second read hits L2)
constexpr int kStripDown = 1 << 30;

// ------------------------------------------------------------------ device error word
// Bits of a handle's device error word: a sweep block's wait for a staged row ran out; its
// outstanding copies could not be drained; a range check of the checked build failed.
enum : int { ERR_TIMEOUT = 1, ERR_DRAIN = 2, ERR_BOUNDS = 4 };

// Debug build (-DLBCG_BOUNDS_CHECK): the step kernels check every population, node-array and
// staged-row access against the extent of its buffer; a failed check sets ERR_BOUNDS in the
// error word and the access is skipped.  In the normal build checked() is constant true and
// the range expressions are dead code the compiler removes.
#ifdef LBCG_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
// an access of `len` consecutive elements starting at i lies inside [0, n)
__host__ __device__ __forceinline__ bool in_extent(long long i, long long len, long long n) {
  return i >= 0 && i + len <= n;
}
__device__ __forceinline__ bool checked(bool ok, int* err) {
  if constexpr (kBoundsCheck) {
    if (!ok) atomicOr(err, ERR_BOUNDS);
    return ok;
  } else {
    (void)err;
    return true;
  }
}

// Per-lattice constants, resident in global memory, one entry per lattice of a handle.
struct LatDev {
  int nx, ny, pitch, bcx, bcy, in_prof;   // in_prof: 1 = Poiseuille inlet profile
  long long pop_off;   // element offset of this lattice's block in the population pool
  long long plane;     // elements of one node-array plane of this lattice (pitch * ny)
  long long node_off;  // element offset of node (0,0) in the node arrays
  double nu_R, nu_B, sigma, beta, s_e, s_eps, s_q, rho0, u_in, rho_out, grad_eps;
  double h_inv_nuR, h_inv_nuB;  // 1/(2 nu_R), 1/(2 nu_B): the two weights of Eq. 18
  double in_y0, in_w;           // inlet profile: s = (y - in_y0) / in_w across the channel
  int wetting, pad2_;           // 0: improved scheme (a); 1: scheme (b), Eq. 48; 2: surface energy
  double cos_theta;             // cos(theta) of the surface-energy variant
};

// Inlet velocity of row y (Sec. III.D): uniform u_in, or the Poiseuille profile
// 4 u_in s (1 - s) whose maximum is u_in.
template <typename T>
__device__ __forceinline__ T inlet_u(const LatDev& L, int y) {
  if (!L.in_prof) return T(L.u_in);
  const double s = (y - L.in_y0) / L.in_w;
  return T(4.0 * L.u_in * s * (1.0 - s));
}

// D2Q9 velocity set (Sec. II.A), as constant-folding functions of the direction index.
__host__ __device__ constexpr int ex(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int a) {
  return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}
template <typename T>
__host__ __device__ constexpr T wgt(int a) {
  return a == 0 ? T(4.0 / 9.0) : (a <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

// ------------------------------------------------------------------ storage traits
template <typename S> struct Store;
template <> struct Store<double> {
  using T = double;
  static constexpr bool kDeviation = false;
  __device__ static void ldp(const double* p, double& lo, double& hi) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    lo = v.x;
    hi = v.y;
  }
  __device__ static void stp(double* p, double lo, double hi) {
    *reinterpret_cast<double2*>(p) = make_double2(lo, hi);
  }
};
template <> struct Store<float> {
  using T = float;
  static constexpr bool kDeviation = false;
  __device__ static void ldp(const float* p, float& lo, float& hi) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    lo = v.x;
    hi = v.y;
  }
  __device__ static void stp(float* p, float lo, float hi) { *reinterpret_cast<float2*>(p) = make_float2(lo, hi); }
};
// ------------------------------------------------------------------ stochastic rounding
// The 16-bit forms round each stored value up or down at random with the probability of its
// distance to the two neighbouring representable values, so that the stored value is exact in
// expectation: per-step changes of a population smaller than half a unit in the last place
// then accumulate instead of being rounded away every step (round-to-nearest stagnation).
// The random bits come from a counter-based hash of (node, step); the hash is
// C. Wellons' "lowbias32" integer hash.
__host__ __device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
// Two floats to a packed 16-bit pair (lo in the low half) with stochastic rounding by the
// conversion itself (cvt.rs): the random bits of the high value are r[31:16], those of the low
// value r[15:0] (FP16 uses the low 13 bits of each half, the bits below its 10-bit mantissa;
// BF16 all 16).  That is exactly "add the random bits below the kept bits of the FP32
// pattern, then truncate", in one instruction per pair.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float lo, float hi, uint32_t r) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
  return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float lo, float hi, uint32_t r) {
  uint32_t d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
  return d;
}
// key of one step of one lattice: epoch counts graph replays (device counter), step the
// launch within them (or the absolute step of a direct launch)
__device__ __forceinline__ uint32_t sr_key(const uint32_t* epoch, uint32_t step, long long pop_off) {
  return hash32(hash32(*epoch ^ 0x9E3779B9u) + step) + uint32_t(pop_off);
}

// FP16 keeps d and g scaled by 2^10: an exact power of two that leaves the rounding of
// normal values unchanged and moves FP16's subnormal range (below 2^-14) down to deviations
// under 2^-24, so that small deviations keep their relative precision.
template <> struct Store<__half> {
  using T = float;
  static constexpr bool kDeviation = true;
  static constexpr float kScale = 1024.0f;
  __device__ static void ldp(const __half* p, float& lo, float& hi) {
    const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
    lo = v.x;
    hi = v.y;
  }
  __device__ static void stp(__half* p, float lo, float hi) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(lo, hi);
  }
  // stochastic rounding: 13 random bits below the kept 10 of each FP32 mantissa, truncated
  __device__ static void stp_sr(__half* p, float lo, float hi, uint32_t r) {
    *reinterpret_cast<uint32_t*>(p) = cvt_rs_f16x2(lo, hi, r);
  }
  __device__ static void unpack(uint32_t w, float& lo, float& hi) {
    __half2 h;
    memcpy(&h, &w, 4);
    const float2 v = __half22float2(h);
    lo = v.x;
    hi = v.y;
  }
};
template <> struct Store<__nv_bfloat16> {
  using T = float;
  static constexpr bool kDeviation = true;
  static constexpr float kScale = 1.0f;
  __device__ static void ldp(const __nv_bfloat16* p, float& lo, float& hi) {
    const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
    lo = v.x;
    hi = v.y;
  }
  __device__ static void stp(__nv_bfloat16* p, float lo, float hi) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
  }
  // stochastic rounding: 16 random bits below the kept 16 bits of each FP32 pattern, truncated
  // (the magnitude rounds up with the probability of the dropped fraction)
  __device__ static void stp_sr(__nv_bfloat16* p, float lo, float hi, uint32_t r) {
    *reinterpret_cast<uint32_t*>(p) = cvt_rs_bf16x2(lo, hi, r);
  }
  __device__ static void unpack(uint32_t w, float& lo, float& hi) {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    const float2 v = __bfloat1622float2(h);
    lo = v.x;
    hi = v.y;
  }
};

// scale of the stored deviations (1 for direct storage)
template <typename S>
__host__ __device__ constexpr float store_scale() {
  if constexpr (Store<S>::kDeviation) return Store<S>::kScale;
  else return 1.0f;
}

// stored pair (lo = k 0, hi = k 1) <-> (f_R, f_B)
template <typename S, typename T>
__device__ __forceinline__ void decode(T lo, T hi, T wr0, T& fr, T& fb) {
  if constexpr (Store<S>::kDeviation) {
    constexpr float inv = 1.0f / Store<S>::kScale, hinv = 0.5f / Store<S>::kScale;
    const T f = fmaf(lo, inv, wr0);
    const T hf = T(0.5) * f;
    fr = fmaf(hi, hinv, hf);
    fb = fmaf(-hi, hinv, hf);
  } else {
    fr = lo;
    fb = hi;
  }
}
template <typename S, typename T>
__device__ __forceinline__ void encode(T fr, T fb, T wr0, T& lo, T& hi) {
  if constexpr (Store<S>::kDeviation) {
    lo = ((fr + fb) - wr0) * Store<S>::kScale;
    hi = (fr - fb) * Store<S>::kScale;
  } else {
    lo = fr;
    hi = fb;
  }
}

// ------------------------------------------------------------------ rounding-exact helpers
// The wall chain (Eq. 28-36) is evaluated without contraction into fused multiply-adds and
// in a fixed order, so that exact cancellations (e.g. a gradient exactly normal to a flat
// wall, which makes D1 == D2 in Eq. 35-36 an exact tie) are reproduced exactly.
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rsqrt_(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_(float a) { return __fsqrt_rn(a); }

// ------------------------------------------------------------------ neighbour mapping
// Periodic axes wrap; other axes clamp (on an inlet/outlet axis the clamped ghost column
// copies the edge column; closed axes have solid edges, so a clamp is never used there
// for a fluid node).
__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool periodic) {
  if (periodic) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// ------------------------------------------------------------------ Zou-He open columns
// Zou-He conditions (Sec. III.D) on the populations of a node in column x of an
// inlet/outlet lattice: velocity inlet (u_in, 0) carrying red only at x = 0 (unknown f1, f5,
// f8), pressure outlet rho_out at x = nx-1 (unknown f3, f6, f7, which take the colour
// fraction of the known populations).  Applying them again to a state that already satisfies
// them changes nothing.
template <typename T>
__device__ __forceinline__ T zh_div(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fdividef(a, b);
  else return a / b;
}
template <typename T>
__device__ __forceinline__ void zou_he(int x, int nx, T u_in, T rho_out, T fr[9], T fb[9]) {
  if (x == 0) {
    T f[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = fr[a] + fb[a];
    const T u = u_in;
    const T rho = zh_div(f[0] + f[2] + f[4] + T(2) * (f[3] + f[6] + f[7]), T(1) - u);
    f[1] = f[3] + T(2.0 / 3.0) * rho * u;
    f[5] = f[7] - T(0.5) * (f[2] - f[4]) + rho * u / T(6);
    f[8] = f[6] + T(0.5) * (f[2] - f[4]) + rho * u / T(6);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      fr[a] = f[a];
      fb[a] = T(0);
    }
  } else if (x == nx - 1) {
    T f[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = fr[a] + fb[a];
    const T r = rho_out;
    const T ux = T(-1) + zh_div(f[0] + f[2] + f[4] + T(2) * (f[1] + f[5] + f[8]), r);
    const T f3 = f[1] - T(2.0 / 3.0) * r * ux;
    const T f7 = f[5] + T(0.5) * (f[2] - f[4]) - r * ux / T(6);
    const T f6 = f[8] - T(0.5) * (f[2] - f[4]) - r * ux / T(6);
    const T kR = fr[0] + fr[1] + fr[2] + fr[4] + fr[5] + fr[8];
    const T kT = f[0] + f[1] + f[2] + f[4] + f[5] + f[8];
    const T frac = kT != T(0) ? zh_div(kR, kT) : T(0);
    fr[3] = frac * f3;
    fb[3] = (T(1) - frac) * f3;
    fr[6] = frac * f6;
    fb[6] = (T(1) - frac) * f6;
    fr[7] = frac * f7;
    fb[7] = (T(1) - frac) * f7;
  }
}

// ------------------------------------------------------------------ node access
// The nine stored pairs of one node (`base` points at its direction-0 pair) decoded to
// (f_R, f_B).
template <typename S>
__device__ __forceinline__ void load_raw(const S* __restrict__ base, typename Store<S>::T r0,
                                         typename Store<S>::T fr[9], typename Store<S>::T fb[9]) {
  using T = typename Store<S>::T;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    T lo, hi;
    Store<S>::ldp(base + a * kDir, lo, hi);
    decode<S, T>(lo, hi, wgt<T>(a) * r0, fr[a], fb[a]);
  }
}

// Encode (f_R, f_B) of one direction (rest weight wr0 = w_a rho0) and store the pair at p.
template <typename S>
__device__ __forceinline__ void store_pair(S* p, typename Store<S>::T fr, typename Store<S>::T fb,
                                           typename Store<S>::T wr0) {
  using T = typename Store<S>::T;
  T lo, hi;
  encode<S, T>(fr, fb, wr0, lo, hi);
  Store<S>::stp(p, lo, hi);
}

// Random word of a node for one step (16-bit storage; key: sr_key, node: its own population
// offset); direction a of the node uses it rotated by 7a bits (sr_bits).  The directions of a
// node share the word: that correlates their roundings but leaves each one unbiased.
__device__ __forceinline__ uint32_t sr_node(uint32_t key, int node) { return hash32(uint32_t(node) + key); }
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, int a) { return __funnelshift_l(h, h, 7 * a); }

// store_pair with stochastic rounding for 16-bit storage (r: random bits, sr_bits)
template <typename S>
__device__ __forceinline__ void store_pair_sr(S* p, typename Store<S>::T fr, typename Store<S>::T fb,
                                              typename Store<S>::T wr0, uint32_t r) {
  using T = typename Store<S>::T;
  if constexpr (Store<S>::kDeviation) {
    T lo, hi;
    encode<S, T>(fr, fb, wr0, lo, hi);
    Store<S>::stp_sr(p, lo, hi, r);
  } else {
    store_pair<S>(p, fr, fb, wr0);
  }
}

// A node's nine stored pairs as loaded, before decoding: for 16-bit storage each pair is one
// 32-bit word, so a prefetched node costs nine registers instead of eighteen.
template <typename S>
struct RawNode {
  typename Store<S>::T lo[9], hi[9];
  __device__ __forceinline__ void load(const S* __restrict__ base) {
#pragma unroll
    for (int a = 0; a < 9; ++a) Store<S>::ldp(base + a * kDir, lo[a], hi[a]);
  }
  __device__ __forceinline__ void decode_to(typename Store<S>::T r0, typename Store<S>::T fr[9],
                                            typename Store<S>::T fb[9]) const {
    using T = typename Store<S>::T;
#pragma unroll
    for (int a = 0; a < 9; ++a) decode<S, T>(lo[a], hi[a], wgt<T>(a) * r0, fr[a], fb[a]);
  }
};
template <typename S>
struct RawNode16 {
  uint32_t w[9];
  __device__ __forceinline__ void load(const S* __restrict__ base) {
#pragma unroll
    for (int a = 0; a < 9; ++a) w[a] = __ldg(reinterpret_cast<const unsigned int*>(base + a * kDir));
  }
  __device__ __forceinline__ void decode_to(float r0, float fr[9], float fb[9]) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      float lo, hi;
      Store<S>::unpack(w[a], lo, hi);
      decode<S, float>(lo, hi, wgt<float>(a) * r0, fr[a], fb[a]);
    }
  }
};
template <> struct RawNode<__half> : RawNode16<__half> {};
template <> struct RawNode<__nv_bfloat16> : RawNode16<__nv_bfloat16> {};

// Post-streaming populations of fluid node (x, y), stored at the node itself (streaming and
// bounce-back happened in the previous step's push), with the Zou-He conditions applied on
// the open columns of an inlet/outlet lattice.
template <typename S>
__device__ __forceinline__ void load_node(const LatDev& L, const S* __restrict__ src, int x, int y,
                                          typename Store<S>::T fr[9], typename Store<S>::T fb[9]) {
  using T = typename Store<S>::T;
  load_raw<S>(src + L.pop_off + pop_node(x, y, L.pitch), T(L.rho0), fr, fb);
  if (L.bcx == BC_INOUT) zou_he<T>(x, L.nx, inlet_u<T>(L, y), T(L.rho_out), fr, fb);
}

// rho^N of Eq. 12 from the colour densities of Eq. 16 (sequential sums in direction order)
template <typename T>
__device__ __forceinline__ T colour_indicator(const T fr[9], const T fb[9], T& rhoR, T& rhoB) {
  T sr = fr[0], sb = fb[0];
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    sr = radd(sr, fr[a]);
    sb = radd(sb, fb[a]);
  }
  rhoR = sr;
  rhoB = sb;
  return rdiv(rsub(sr, sb), radd(sr, sb));
}

}  // namespace lbcg
