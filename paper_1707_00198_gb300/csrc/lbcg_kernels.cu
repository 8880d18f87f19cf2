// Kernels of one time step of the colour-gradient LBM with the improved wetting scheme
// (arXiv 1707.00198, Sec. II).  Per step, in stream order:
//   k_wall  : per group of outermost fluid nodes, rho^N (Eq. 12, 16) of the wall band (those
//             nodes and their fluid neighbours) from the post-streaming populations, the
//             virtual values of Eq. 29, then on each outermost fluid node the gradient of
//             Eq. 28 and the contact-angle correction of Eq. 30-36 -> corrected gradient and
//             unit normal, kept in small node arrays;
//   k_step  : the fused bulk step over 32 x TY tiles: loads of each node's own populations
//             -> rho^N on the tile plus a 2-node halo (shared memory) ->
//             n on the tile plus a 1-node halo (outermost-fluid values from k_wall, virtual
//             n on outermost solid nodes, Eq. 29) -> grad n, kappa, F (Eq. 10, 13, 28) ->
//             u, nu, MRT collision with Guo forcing (Eq. 1-9, 17, 18) -> recolouring
//             (Eq. 14) -> push of the post-collision populations to the neighbours
//             (streaming, Eq. 15) with half-way bounce-back at solid neighbours.
#include <algorithm>

#include "lbcg_device.cuh"
#include "lbcg_internal.h"

namespace lbcg {

struct StepArgs {
  const LatDev* lats;
  const int4* tiles;      // (lattice, x0, y0, -)
  const void* src;        // population pool read this step
  void* dst;              // population pool written this step
  const uint8_t* flags;   // node flags
  void* wall;             // 4 planes of node arrays: g_x, g_y, n_x, n_y (compute type)
  long long node_total;   // elements per node-array plane
  double* macro;          // 4 planes of doubles: rho_R, rho_B, u_x, u_y (macro mode)
  const uint32_t* sr_epoch;   // stochastic rounding of 16-bit stores: replay counter
  uint32_t sr_step;           // and the step within the replay (sr_key)
  int* err;                   // device error word (range checks of the checked build)
};

// ------------------------------------------------------------------ k_wall
// One block per WallGroup, three phases separated by barriers:
//   1. rho^N (Eq. 12, 16) of the group's band nodes from their post-streaming populations;
//   2. the virtual value of each outermost solid node next to the group: the weighted mean of
//      Eq. 29 over its fluid neighbours (rho^N = cos(theta) in the surface-energy variant);
//   3. on each outermost fluid node, the gradient of Eq. 28 over those values, then the
//      contact-angle correction of Eq. 30-36 -> corrected gradient and unit normal.
// The arithmetic is rounding-exact in the oracle's order (directions 1..8, products w*phi
// then sign); the host-built stencils only replace the flag lookups of that order.
// Eq. 28 on an outermost fluid node from the shared values of its 8 neighbours, then
// Eq. 30-36; writes the corrected gradient and unit normal.
template <typename T>
__device__ __forceinline__ void wall_node(const LatDev& sL, const OfbEntry& e, const WallSten& q, const T* val,
                                          T* __restrict__ wall, long long node_total) {
  T gx = T(0), gy = T(0);
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    const T tt = rmul(wgt<T>(a), val[q.i[a - 1]]);
    if (ex(a) == 1) gx = radd(gx, tt);
    if (ex(a) == -1) gx = radd(gx, -tt);
    if (ey(a) == 1) gy = radd(gy, tt);
    if (ey(a) == -1) gy = radd(gy, -tt);
  }
  const T cs2 = T(1.0 / 3.0);
  gx = rdiv(gx, cs2);
  gy = rdiv(gy, cs2);
  const T eps = T(sL.grad_eps);
  const T mag = rsqrt_(radd(rmul(gx, gx), rmul(gy, gy)));
  T cgx = gx, cgy = gy, nx = T(0), ny = T(0);
  if (mag > eps && sL.wetting == 2) {
    nx = rdiv(gx, mag);   // no geometric correction: n from the raw gradient
    ny = rdiv(gy, mag);
  } else if (mag > eps) {
    const T esx = rdiv(gx, mag), esy = rdiv(gy, mag);                 // Eq. 30
    const T nsx = T(e.nsx), nsy = T(e.nsy), c = T(e.cos_t), s = T(e.sin_t);
    const T f1x = rsub(rmul(nsx, c), rmul(nsy, s));                   // Eq. 34, +theta
    const T f1y = radd(rmul(nsx, s), rmul(nsy, c));
    const T f2x = radd(rmul(nsx, c), rmul(nsy, s));                   // Eq. 34, -theta
    const T f2y = radd(rmul(-nsx, s), rmul(nsy, c));
    const T a1 = rsub(f1x, esx), b1 = rsub(f1y, esy);
    const T a2 = rsub(f2x, esx), b2 = rsub(f2y, esy);
    const T d1 = rsqrt_(radd(rmul(a1, a1), rmul(b1, b1)));            // Eq. 35
    const T d2 = rsqrt_(radd(rmul(a2, a2), rmul(b2, b2)));
    const T nfx = d1 <= d2 ? f1x : f2x;                               // Eq. 36
    const T nfy = d1 <= d2 ? f1y : f2y;
    cgx = rmul(mag, nfx);                                             // Eq. 31
    cgy = rmul(mag, nfy);
    const T m2 = rsqrt_(radd(rmul(cgx, cgx), rmul(cgy, cgy)));
    if (m2 > eps) {
      nx = rdiv(cgx, m2);
      ny = rdiv(cgy, m2);
    }
  }
  const long long k = sL.node_off + (long long)e.y * sL.pitch + e.x;
  wall[k] = cgx;
  wall[node_total + k] = cgy;
  wall[2 * node_total + k] = nx;
  wall[3 * node_total + k] = ny;
}

// 16-byte asynchronous copy global -> shared (no register staging)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Programmatic dependent launch of the tile schedule (launch_all): on a small lattice a step's
// two kernels are short grids, each waiting for the one before it, so the gap between one
// grid's end and the next one's start is a visible part of the step.  k_wall and k_step are
// then launched with programmatic stream serialisation: the next grid may be scheduled once
// every block of the grid before it has run dep_trigger or exited, and every thread of it
// runs dep_wait -- the hardware's wait for the full completion and memory flush of that
// grid -- before it reads or writes anything the grid before it reads or writes
// (populations, the wall kernel's output); only the static lattice tables are read before
// the wait.  For a kernel launched the ordinary way both instructions do nothing.
// Where the trigger sits decides only when the next grid's blocks are scheduled, never what
// they read.  FP32 and 16-bit storage trigger at the start of each block: the next grid then
// becomes resident and stages its tables while this one runs (it is scheduled only once every
// block of this grid has started, so its waiting blocks never hold resources this grid still
// needs); measured 1200x80 FP32 13.1 -> 10.6 us per step and 2000x102 20.2 -> 17.3 against a
// trigger after the last store.  FP64 triggers after each block's last store: its blocks hold
// several times the registers, and resident waiting FP64 blocks slowed the kernels running
// beside them on another stream (the FP64 adjoint, whose recompute runs on a side stream:
// 118 -> 177 us per step with the early trigger).
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename S>
constexpr bool kEarlyTrigger = sizeof(typename Store<S>::T) == 4;

template <typename S>
__global__ void __launch_bounds__(kWallThreads, sizeof(S) == 8 ? 3 : 5) k_wall(const LatDev* __restrict__ lats,
                                                          const WallGroup* __restrict__ groups,
                                                          const int* __restrict__ band,
                                                          const WallSten* __restrict__ virt,
                                                          const WallSten* __restrict__ sten,
                                                          const OfbEntry* __restrict__ ofb, const S* __restrict__ src,
                                                          typename Store<S>::T* __restrict__ wall, long long node_total,
                                                          int* __restrict__ err) {
  using T = typename Store<S>::T;
  static_assert(sizeof(OfbEntry) % 16 == 0 && sizeof(WallSten) == 16, "16-byte table entries");
  __shared__ T val[kWallCap];
  __shared__ __align__(16) OfbEntry s_ofb[kWallMaxNodes];
  __shared__ __align__(16) WallSten s_sten[kWallMaxNodes];
  __shared__ __align__(16) WallSten s_virt[kWallVirtCap];
  __shared__ __align__(16) int s_band[kWallCap];
  __shared__ LatDev sL;
  const WallGroup G = groups[blockIdx.x];
  const int t = threadIdx.x;
  if constexpr (kEarlyTrigger<S>) dep_trigger();
  // the group's sizes against the shared tables (uniform over the block)
  if (!checked(G.nwall >= 0 && G.nwall <= kWallMaxNodes && G.nvirt >= 0 && G.nvirt <= kWallVirtCap &&
                   G.nband >= 1 && (G.nband + 3) / 4 * 4 <= kWallCap && G.nband + G.nvirt <= kWallCap,
               err)) {
    dep_wait();
    return;
  }
  // the group's tables, copied to shared memory in 16-byte pieces that are all in flight at
  // once (band0 is a multiple of 4 and the band list is padded, so the last piece is in bounds)
  {
    constexpr int kO = int(sizeof(OfbEntry) / 16);
    const int n1 = G.nwall * kO, n2 = n1 + G.nwall, n3 = n2 + G.nvirt, n4 = n3 + (G.nband + 3) / 4;
    for (int c = t; c < n4; c += kWallThreads) {
      const uint4* from;
      uint4* to;
      if (c < n1) {
        from = reinterpret_cast<const uint4*>(ofb + G.wall0) + c;
        to = reinterpret_cast<uint4*>(s_ofb) + c;
      } else if (c < n2) {
        from = reinterpret_cast<const uint4*>(sten + G.wall0) + (c - n1);
        to = reinterpret_cast<uint4*>(s_sten) + (c - n1);
      } else if (c < n3) {
        from = reinterpret_cast<const uint4*>(virt + G.virt0) + (c - n2);
        to = reinterpret_cast<uint4*>(s_virt) + (c - n2);
      } else {
        from = reinterpret_cast<const uint4*>(band + G.band0) + (c - n3);
        to = reinterpret_cast<uint4*>(s_band) + (c - n3);
      }
      cp_async16(to, from);
    }
  }
  if (t == 0) sL = lats[G.lat];
  cp_async_wait_all();
  dep_wait();   // the populations of the step before are complete from here on
  __syncthreads();
  // phase 1, UW band nodes at a time: their populations first, then the Zou-He columns and
  // rho^N (indices past the end repeat the last node, so that no load sits behind a branch)
  constexpr int UW = sizeof(S) == 8 ? 2 : 3;
  const S* __restrict__ pop = src + sL.pop_off;
  const T r0 = T(sL.rho0);
  for (int i0 = t; i0 < G.nband; i0 += UW * kWallThreads) {
    T fr[UW][9], fb[UW][9];
    int off[UW];
#pragma unroll
    for (int v = 0; v < UW; ++v) {
      off[v] = s_band[min(i0 + v * kWallThreads, G.nband - 1)];
      if (!checked(in_extent(off[v], 8 * kDir + 2, 18 * sL.plane), err)) off[v] = 0;
    }
#pragma unroll
    for (int v = 0; v < UW; ++v) load_raw<S>(pop + off[v], r0, fr[v], fb[v]);
#pragma unroll
    for (int v = 0; v < UW; ++v) {
      const int i = i0 + v * kWallThreads;
      if (i < G.nband) {
        if (sL.bcx == BC_INOUT) {
          // node of the population offset (the inverse of pop_node)
          const int seg = off[v] / kSeg, segs = sL.pitch >> 5;
          const int x = (seg % segs) * 32 + (off[v] % kSeg) / 2, y = seg / segs;
          zou_he<T>(x, sL.nx, inlet_u<T>(sL, y), T(sL.rho_out), fr[v], fb[v]);
        }
        T rR, rB;
        val[i] = colour_indicator(fr[v], fb[v], rR, rB);
      }
    }
  }
  __syncthreads();
  for (int j = t; j < G.nvirt; j += kWallThreads) {
    T v;
    if (sL.wetting == 2) {
      v = T(sL.cos_theta);   // surface-energy formulation: rho^N = cos(theta) on the solid
    } else {
      const WallSten q = s_virt[j];
      T num = T(0), den = T(0);
#pragma unroll
      for (int b = 1; b < 9; ++b)
        if (q.i[b - 1] != kWallNone && checked(q.i[b - 1] < G.nband, err)) {
          num = radd(num, rmul(wgt<T>(b), val[q.i[b - 1]]));
          den = radd(den, wgt<T>(b));
        }
      v = rdiv(num, den);
    }
    val[G.nband + j] = v;
  }
  __syncthreads();
  for (int w = t; w < G.nwall; w += kWallThreads) {
    bool ok = in_extent((long long)s_ofb[w].y * sL.pitch + s_ofb[w].x, 1, sL.plane);
#pragma unroll
    for (int a = 0; a < 8; ++a) ok = ok && s_sten[w].i[a] < G.nband + G.nvirt;
    if (checked(ok, err)) wall_node<T>(sL, s_ofb[w], s_sten[w], val, wall, node_total);
  }
  if constexpr (!kEarlyTrigger<S>) dep_trigger();
}


// Eq. 48, wetting scheme (b) (lbcg_params.wetting = 1): grad n at an outermost fluid node from
// its fluid neighbours only, d_i n = sum_a w_a (n(x + e_a) - n(x)) e_ai / sum_a w_a e_ai^2 over
// the directions a whose neighbour is fluid (bit a-1 of `solid` clear).  nxs/nys[a] hold n at
// x + e_a (a = 0: the node).  Returned divided by 3 (= c_s^2): the bulk kernels keep their
// Eq. 28 sums at that scale and apply 1/c_s^2 in the curvature.
template <typename T>
__device__ __forceinline__ void grad_n_scheme_b(const T nxs[9], const T nys[9], unsigned solid, T& dxx, T& dyx, T& dxy,
                                                T& dyy) {
  T sxx = T(0), syx = T(0), sxy = T(0), syy = T(0), wx = T(0), wy = T(0);
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if ((solid >> (a - 1)) & 1u) continue;
    const T w = wgt<T>(a), ddx = nxs[a] - nxs[0], ddy = nys[a] - nys[0];
    if (ex(a)) {
      sxx += T(ex(a)) * w * ddx;
      syx += T(ex(a)) * w * ddy;
      wx += w;
    }
    if (ey(a)) {
      sxy += T(ey(a)) * w * ddx;
      syy += T(ey(a)) * w * ddy;
      wy += w;
    }
  }
  const T third = T(1) / T(3);
  dxx = wx > T(0) ? sxx / wx * third : T(0);
  dyx = wx > T(0) ? syx / wx * third : T(0);
  dxy = wy > T(0) ? sxy / wy * third : T(0);
  dyy = wy > T(0) ? syy / wy * third : T(0);
}

// ------------------------------------------------------------------ k_step
// Arithmetic helpers: the FP64 instantiation keeps IEEE divisions and square roots (it is the
// validation path); the FP32-arithmetic instantiations use the hardware reciprocal and
// reciprocal square root.
template <typename T>
__device__ __forceinline__ T rcp_(T x) {
  if constexpr (sizeof(T) == 4) return __fdividef(1.0f, x);
  else return T(1) / x;
}

// FP32-arithmetic instantiations are held to 64 registers so that 1024 threads fit on an
// SM (they need no more); the FP64 validation instantiation keeps its registers.
template <typename S, int TY, bool MACRO>
__global__ void __launch_bounds__(32 * TY, sizeof(typename Store<S>::T) == 4 ? 1024 / (32 * TY) : 1)
    k_step(StepArgs A) {
  using T = typename Store<S>::T;
  constexpr bool kF32 = sizeof(T) == 4;
  constexpr int TX = 32;
  constexpr int NT = TX * TY;
  constexpr int W3 = TX + 6, H3 = TY + 6;   // flags: tile + 3
  constexpr int W2 = TX + 4, H2 = TY + 4;   // rho^N: tile + 2
  constexpr int W1 = TX + 2, H1 = TY + 2;   // n: tile + 1
  __shared__ uint8_t sfl[H3 * W3];
  __shared__ T srn[H2 * W2];
  __shared__ T snx[H1 * W1];
  __shared__ T sny[H1 * W1];
  __shared__ int sxm[W3];
  __shared__ int sym[H3];
  __shared__ LatDev sL;

  const int4 tl = A.tiles[blockIdx.x];
  const int x0 = tl.y, y0 = tl.z;
  const int tid = threadIdx.x;
  if constexpr (!MACRO && kEarlyTrigger<S>) dep_trigger();
  if (tid == 0) sL = A.lats[tl.x];
  __syncthreads();
  // lattice constants in registers (shared memory cannot alias the global stores below)
  const int nx = sL.nx, ny = sL.ny, pitch = sL.pitch;
  const bool px = sL.bcx == BC_PERIODIC, py = sL.bcy == BC_PERIODIC, inout = sL.bcx == BC_INOUT;
  const T r0 = T(sL.rho0), u_in = T(sL.u_in), rho_out = T(sL.rho_out), eps = T(sL.grad_eps);
  const uint8_t* __restrict__ fl = A.flags + sL.node_off;
  const S* __restrict__ src = static_cast<const S*>(A.src) + sL.pop_off;
  const T* __restrict__ wall = static_cast<const T*>(A.wall) + sL.node_off;
  const long long NTOT = A.node_total;

  // mapped lattice coordinates of every halo column / row
  for (int i = tid; i < W3; i += NT) sxm[i] = wrap_or_clamp(x0 + i - 3, nx, px);
  for (int i = tid; i < H3; i += NT) sym[i] = wrap_or_clamp(y0 + i - 3, ny, py);
  __syncthreads();
  for (int i = tid; i < H3 * W3; i += NT) {
    const int cx = i % W3, cy = i / W3;
    const long long k = (long long)sym[cy] * pitch + sxm[cx];
    sfl[i] = checked(in_extent(k, 1, sL.plane), A.err) ? fl[k] : uint8_t(F_SOLID);
  }
  dep_wait();   // the populations and the wall kernel's output are complete from here on
  __syncthreads();

  auto load = [&](int c3x, int c3y, T fr_[9], T fb_[9]) {
    const int x = sxm[c3x];
    if (!checked(in_extent(pop_node(x, sym[c3y], pitch), 8 * kDir + 2, 18 * sL.plane), A.err)) {
#pragma unroll
      for (int a = 0; a < 9; ++a) fr_[a] = fb_[a] = T(0);
      return;
    }
    load_raw<S>(src + pop_node(x, sym[c3y], pitch), r0, fr_, fb_);
    if (inout) zou_he<T>(x, nx, inlet_u<T>(sL, sym[c3y]), rho_out, fr_, fb_);
  };
  // rho^N (Eq. 12): exactly +-1 on single-colour nodes in both arithmetic paths
  auto indicator = [&](const T fr_[9], const T fb_[9], T& sr, T& sb) -> T {
    sr = fr_[0];
    sb = fb_[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      sr += fr_[a];
      sb += fb_[a];
    }
    if constexpr (kF32) {
      const T v = (sr - sb) * rcp_(sr + sb);
      return sb == T(0) ? T(1) : (sr == T(0) ? T(-1) : v);
    } else {
      return (sr - sb) / (sr + sb);
    }
  };

  // ---- phase A: rho^N on tile + 2 (own node keeps its populations in registers)
  const int lx = tid % TX, ly = tid / TX;
  T fr[9], fb[9], rhoR = T(0), rhoB = T(0), rn = T(0);
  const bool fluid = !(sfl[(ly + 3) * W3 + lx + 3] & F_SOLID);
  if (fluid) {
    load(lx + 3, ly + 3, fr, fb);
    rn = indicator(fr, fb, rhoR, rhoB);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) fr[a] = fb[a] = T(0);
  }
  srn[(ly + 2) * W2 + lx + 2] = rn;
  for (int i = tid; i < H2 * W2; i += NT) {
    const int cx = i % W2, cy = i / W2;
    if (cx >= 2 && cx < TX + 2 && cy >= 2 && cy < TY + 2) continue;
    T v = T(0);
    if (!(sfl[(cy + 1) * W3 + cx + 1] & F_SOLID)) {
      T hr[9], hb[9], a1, a2;
      load(cx + 1, cy + 1, hr, hb);
      v = indicator(hr, hb, a1, a2);
    }
    srn[i] = v;
  }
  __syncthreads();

  // ---- phase B: grad rho^N and n on tile + 1
  T gx = T(0), gy = T(0);
  for (int i = tid; i < H1 * W1 + NT; i += NT) {
    // the first NT iterations cover the own tile node, the rest the ring of tile + 1
    int cx, cy;
    const bool own = i < NT;
    if (own) {
      cx = lx + 1;
      cy = ly + 1;
    } else {
      const int j = i - NT;
      cx = j % W1;
      cy = j / W1;
      if (cx >= 1 && cx < TX + 1 && cy >= 1 && cy < TY + 1) continue;
    }
    // A slot beyond a non-periodic edge is a ghost copy of the edge node (zero normal
    // gradient): evaluate it at the slot of the node it copies, whose stencil stays inside
    // the halo.  Periodic slots already hold their wrapped node with its own neighbours.
    const int sx = px ? cx : min(max(cx + sxm[cx + 2] - (x0 + cx - 1), 0), W1 - 1);
    const int sy = py ? cy : min(max(cy + sym[cy + 2] - (y0 + cy - 1), 0), H1 - 1);
    const int c3x = sx + 2, c3y = sy + 2;
    const uint8_t f = sfl[c3y * W3 + c3x];
    const int k = sym[c3y] * pitch + sxm[c3x];
    T ax = T(0), ay = T(0), nxv = T(0), nyv = T(0);
    if (!(f & F_SOLID)) {
      if ((f & F_OFB) && checked(in_extent(k, 1, sL.plane), A.err)) {
        ax = wall[k];
        ay = wall[NTOT + k];
        nxv = wall[2 * NTOT + k];
        nyv = wall[3 * NTOT + k];
      } else {
        const int c2x = sx + 1, c2y = sy + 1;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
          const T t = wgt<T>(a) * srn[(c2y + ey(a)) * W2 + c2x + ex(a)];
          if (ex(a)) ax += T(ex(a)) * t;
          if (ey(a)) ay += T(ey(a)) * t;
        }
        ax *= T(3);
        ay *= T(3);
        const T m2 = ax * ax + ay * ay;
        if constexpr (kF32) {
          if (m2 > eps * eps) {
            const T inv = rsqrtf(m2);
            nxv = ax * inv;
            nyv = ay * inv;
          }
        } else {
          const T m = sqrt(m2);
          if (m > eps) {
            nxv = ax / m;
            nyv = ay / m;
          }
        }
      }
    } else if (f & F_OSOLID) {
      // virtual n on the outermost solid node (Eq. 29); its fluid neighbours are outermost
      // fluid nodes, whose n k_wall has stored
      T vx = T(0), vy = T(0), den = T(0);
#pragma unroll
      for (int b = 1; b < 9; ++b) {
        if (!(sfl[(c3y + ey(b)) * W3 + c3x + ex(b)] & F_SOLID)) {
          const int k2 = sym[c3y + ey(b)] * pitch + sxm[c3x + ex(b)];
          if (!checked(in_extent(k2, 1, sL.plane), A.err)) continue;
          vx += wgt<T>(b) * wall[2 * NTOT + k2];
          vy += wgt<T>(b) * wall[3 * NTOT + k2];
          den += wgt<T>(b);
        }
      }
      if (den > T(0)) {
        nxv = vx / den;
        nyv = vy / den;
      }
    }
    snx[cy * W1 + cx] = nxv;
    sny[cy * W1 + cx] = nyv;
    if (own) {
      gx = ax;
      gy = ay;
    }
  }
  __syncthreads();

  // ---- phase C: curvature, force, collision, recolouring, push (own node)
  const int xs = x0 + lx, ys = y0 + ly;
  if (!fluid || xs >= nx || ys >= ny) return;
  const int c1x = lx + 1, c1y = ly + 1;
  T dxx = T(0), dxy = T(0), dyx = T(0), dyy = T(0);  // d_x n_x, d_y n_x, d_x n_y, d_y n_y
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    const int o = (c1y + ey(a)) * W1 + c1x + ex(a);
    const T tx = wgt<T>(a) * snx[o];
    const T ty = wgt<T>(a) * sny[o];
    if (ex(a)) {
      dxx += T(ex(a)) * tx;
      dyx += T(ex(a)) * ty;
    }
    if (ey(a)) {
      dxy += T(ey(a)) * tx;
      dyy += T(ey(a)) * ty;
    }
  }
  if (sL.wetting == 1 && (sfl[(ly + 3) * W3 + lx + 3] & F_OFB)) {
    T nxs[9], nys[9];
    unsigned solid = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int o = (c1y + ey(a)) * W1 + c1x + ex(a);
      nxs[a] = snx[o];
      nys[a] = sny[o];
      if (a && (sfl[(ly + 3 + ey(a)) * W3 + lx + 3 + ex(a)] & F_SOLID)) solid |= 1u << (a - 1);
    }
    grad_n_scheme_b<T>(nxs, nys, solid, dxx, dyx, dxy, dyy);
  }
  const T nxo = snx[c1y * W1 + c1x], nyo = sny[c1y * W1 + c1x];
  // Eq. 13 (the factor 3 = 1/c_s^2 of Eq. 28 applied once) and Eq. 10
  const T kappa = T(3) * (-nxo * nxo * dyy - nyo * nyo * dxx + nxo * nyo * (dxy + dyx));
  const T hsk = T(0.5) * T(sL.sigma) * kappa;
  const T Fx = hsk * gx;
  const T Fy = hsk * gy;

  T f[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) f[a] = fr[a] + fb[a];
  const T rho = rhoR + rhoB;
  const T irho = rcp_(rho);
  const T jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const T jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const T ux = (jx + T(0.5) * Fx) * irho;                                         // Eq. 17
  const T uy = (jy + T(0.5) * Fy) * irho;
  const int kn = ys * pitch + xs;
  if constexpr (MACRO) {
    if (!checked(in_extent(kn, 1, sL.plane), A.err)) return;
    const long long k = sL.node_off + kn;
    A.macro[k] = double(rhoR);
    A.macro[NTOT + k] = double(rhoB);
    A.macro[2 * NTOT + k] = double(ux);
    A.macro[3 * NTOT + k] = double(uy);
    return;
  } else {
    // local viscosity (Eq. 18) and s_v = 1/tau_v = 1/(3 nu + 1/2) (Eq. 5)
    const T inv_nu = (T(1) + rn) * T(sL.h_inv_nuR) + (T(1) - rn) * T(sL.h_inv_nuB);
    const T sv = inv_nu * rcp_(T(3) + T(0.5) * inv_nu);
    const T se = T(sL.s_e), seps = T(sL.s_eps), sq = T(sL.s_q);
    // moments (rows of Eq. 3, the last one read as e_x e_y)
    const T s14 = f[1] + f[2] + f[3] + f[4];
    const T s58 = f[5] + f[6] + f[7] + f[8];
    const T me = T(-4) * f[0] - s14 + T(2) * s58;
    const T meps = T(4) * f[0] - T(2) * s14 + s58;
    const T qx = T(-2) * (f[1] - f[3]) + (f[5] - f[6] - f[7] + f[8]);
    const T qy = T(-2) * (f[2] - f[4]) + (f[5] + f[6] - f[7] - f[8]);
    const T pxx = f[1] - f[2] + f[3] - f[4];
    const T pxy = f[5] - f[6] + f[7] - f[8];
    const T u2 = ux * ux + uy * uy;
    const T uF = ux * Fx + uy * Fy;
    // Delta_k = s_k (m_k - m_k^eq) - (1 - s_k/2) (M F~)_k  with M F~ =
    // (0, 6 u.F, -6 u.F, Fx, -Fx, Fy, -Fy, 2(ux Fx - uy Fy), ux Fy + uy Fx)   (Eq. 8-9)
    const T De = se * (me - rho * (T(-2) + T(3) * u2)) - (T(1) - T(0.5) * se) * (T(6) * uF);
    const T Deps = seps * (meps - rho * (T(1) - T(3) * u2)) + (T(1) - T(0.5) * seps) * (T(6) * uF);
    const T Dqx = sq * (qx + rho * ux) + (T(1) - T(0.5) * sq) * Fx;
    const T Dqy = sq * (qy + rho * uy) + (T(1) - T(0.5) * sq) * Fy;
    const T Dxx = sv * (pxx - rho * (ux * ux - uy * uy)) - (T(1) - T(0.5) * sv) * (T(2) * (ux * Fx - uy * Fy));
    const T Dxy = sv * (pxy - rho * ux * uy) - (T(1) - T(0.5) * sv) * (ux * Fy + uy * Fx);
    // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4); s_rho = s_j = 1
    // (Eq. 6), so the momentum rows give Delta_j = -F: the momentum changes by exactly F
    const T ae = De * T(1.0 / 36.0), aeps = Deps * T(1.0 / 36.0);
    const T ajx = -Fx * T(1.0 / 6.0), ajy = -Fy * T(1.0 / 6.0);
    const T aqx = Dqx * T(1.0 / 12.0), aqy = Dqy * T(1.0 / 12.0);
    const T axx = Dxx * T(0.25), axy = Dxy * T(0.25);
    T fp[9];
    fp[0] = f[0] - (T(-4) * ae + T(4) * aeps);
    const T c14 = -ae - T(2) * aeps;
    fp[1] = f[1] - (c14 + ajx - T(2) * aqx + axx);
    fp[2] = f[2] - (c14 + ajy - T(2) * aqy - axx);
    fp[3] = f[3] - (c14 - ajx + T(2) * aqx + axx);
    fp[4] = f[4] - (c14 - ajy + T(2) * aqy - axx);
    const T c58 = T(2) * ae + aeps;
    fp[5] = f[5] - (c58 + ajx + aqx + ajy + aqy + axy);
    fp[6] = f[6] - (c58 - ajx - aqx + ajy + aqy - axy);
    fp[7] = f[7] - (c58 - ajx - aqx - ajy - aqy + axy);
    fp[8] = f[8] - (c58 + ajx + aqx - ajy - aqy - axy);
    // recolouring (Eq. 14; the blue line with the minus sign)
    const T cR = rhoR * irho, cB = rhoB * irho;
    const T pc = T(sL.beta) * rhoR * rhoB * irho;
    S* __restrict__ dst = static_cast<S*>(A.dst) + sL.pop_off;
    uint32_t srk = 0;
    if constexpr (Store<S>::kDeviation) srk = sr_key(A.sr_epoch, A.sr_step, sL.pop_off);
    const int c3x = lx + 3, c3y = ly + 3;
    const int pn_own = pop_node(xs, ys, pitch);
    uint32_t srh = 0;
    if constexpr (Store<S>::kDeviation) srh = sr_node(srk, pn_own);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const T en = T(ex(a)) * nxo + T(ey(a)) * nyo;
      const T pert = pc * wgt<T>(a) * en;
      const T oR = cR * fp[a] + pert;
      const T oB = cB * fp[a] - pert;
      // streaming (Eq. 15): to x + e_a if that node is fluid; half-way bounce-back into the
      // opposite slot of this node if it is solid; dropped if it lies beyond an open edge
      int k = pn_own, slot = a;
      if (a != 0) {
        const int xr = xs + ex(a), yr = ys + ey(a);
        if ((!px && (xr < 0 || xr >= nx)) || (!py && (yr < 0 || yr >= ny))) continue;
        if (sfl[(c3y + ey(a)) * W3 + c3x + ex(a)] & F_SOLID) {
          slot = opp(a);
        } else {
          k = pop_node(sxm[c3x + ex(a)], sym[c3y + ey(a)], pitch);
        }
      }
      if (checked(in_extent((long long)k + slot * kDir, 2, 18 * sL.plane), A.err))
        store_pair_sr<S>(dst + k + slot * kDir, oR, oB, wgt<T>(a) * r0, sr_bits(srh, a));
    }
    if constexpr (!kEarlyTrigger<S>) dep_trigger();
  }
}

// ------------------------------------------------------------------ pair arithmetic
// (x, y) pairs; on the FP32 path they map onto the packed two-lane FP32 instructions of
// sm_100+ (__ffma2_rn and friends), on the FP64 path onto two scalar operations.
template <typename T> struct Pair;
template <> struct Pair<float> {
  using V = float2;
  __device__ static V mk(float a, float b) { return make_float2(a, b); }
  __device__ static V add(V a, V b) { return __fadd2_rn(a, b); }
  __device__ static V sub(V a, V b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
  __device__ static V mul(V a, V b) { return __fmul2_rn(a, b); }
  __device__ static V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
};
template <> struct Pair<double> {
  using V = double2;
  __device__ static V mk(double a, double b) { return make_double2(a, b); }
  __device__ static V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
  __device__ static V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
};

// ------------------------------------------------------------------ k_sweep
// The same time step as k_step, organised as a sweep along y over column strips: a block of
// NTH threads owns NTH - 4 interior columns plus two halo columns on each side and walks up
// a range of rows.  Per row r it loads the populations of row r and forms rho^N(r); then
// n(r-1) (needs rho^N of rows r-2..r); then collides row r-2 (needs n of rows r-3..r-1) and
// pushes it.  Halo work exists only in x (NTH / (NTH-4) loads per node); each node is loaded
// once for rho^N and once more (from L2) for its collision; the rows of the stencil live in
// small shared-memory rings whose slots, like the wrapped row indices, advance by one per row.
struct SweepArgs {
  const LatDev* lats;
  const int4* strips;     // (lattice, x0 = first interior column, y_begin, y_end)
  const void* src;
  void* dst;
  const uint8_t* flags;
  const uint8_t* nbmask;  // bit a-1 set: the neighbour in direction a (1..8) is solid
  const void* wall;
  long long node_total;
  int* err;               // k_sweepf: bit 0 set by a block whose wait for a staged row ran out,
                          // bit 1 if its copies could not be drained before it returned
  const uint32_t* sr_epoch;   // stochastic rounding of 16-bit stores (sr_key)
  uint32_t sr_step;
  int poll_limit;         // k_sweepf: polls of a staged row's barrier before a wait gives up
};

template <typename S, int NTH>
__global__ void __launch_bounds__(NTH, sizeof(typename Store<S>::T) == 4 ? 1024 / NTH : 1)
    k_sweep(SweepArgs A) {
  using T = typename Store<S>::T;
  constexpr bool kF32 = sizeof(T) == 4;
  constexpr int RR = 5;   // rho^N / flags ring (rows r-4 .. r)
  constexpr int RN = 3;   // n, grad ring (rows r-3 .. r-1)
  using P = Pair<T>;
  using V = typename P::V;
  __shared__ T srn[RR][NTH];
  __shared__ uint8_t sfl[RR][NTH];
  __shared__ V sn[RN][NTH], sg[RN][NTH];   // (n_x, n_y) and (d_x rho^N, d_y rho^N)
  __shared__ LatDev sL;

  const int4 sp = A.strips[blockIdx.x];
  const int t = threadIdx.x;
  if (t == 0) sL = A.lats[sp.x & ~kStripDown];
  __syncthreads();
  const int nx = sL.nx, ny = sL.ny, pitch = sL.pitch;
  const bool px = sL.bcx == BC_PERIODIC, py = sL.bcy == BC_PERIODIC, inout = sL.bcx == BC_INOUT;
  const T r0 = T(sL.rho0), u_in = T(sL.u_in), rho_out = T(sL.rho_out), eps = T(sL.grad_eps);
  const T sigma = T(sL.sigma), beta = T(sL.beta), se = T(sL.s_e), seps = T(sL.s_eps), sq = T(sL.s_q);
  const T hR = T(sL.h_inv_nuR), hB = T(sL.h_inv_nuB);
  const uint8_t* __restrict__ fl = A.flags + sL.node_off;
  const uint8_t* __restrict__ nbm = A.nbmask + sL.node_off;
  const S* __restrict__ src = static_cast<const S*>(A.src) + sL.pop_off;
  S* __restrict__ dst = static_cast<S*>(A.dst) + sL.pop_off;
  const T* __restrict__ wall = static_cast<const T*>(A.wall) + sL.node_off;
  const long long NTOT = A.node_total;

  // this thread's column and its neighbours
  const int cx = sp.y - 2 + t;                       // raw column
  const int xm = wrap_or_clamp(cx, nx, px);
  const int xl = wrap_or_clamp(cx - 1, nx, px), xr = wrap_or_clamp(cx + 1, nx, px);
  // a column beyond a non-periodic edge is a ghost copy of the edge column: its n is
  // evaluated at the slot of the column it copies (zero normal gradient)
  const int tc = px ? t : min(max(t + xm - cx, 1), NTH - 2);
  const int kxs = wrap_or_clamp(sp.y - 2 + tc, nx, px);  // column of the stage-2 slot
  const bool interior = t >= 2 && t < NTH - 2 && cx < nx;
  const int ys = sp.z, ye = sp.w;
  // element offsets of the neighbouring columns within a row of 32-node segments
  const int colk[3] = {(xl >> 5) * kSeg + (xl & 31) * 2, (xm >> 5) * kSeg + (xm & 31) * 2,
                       (xr >> 5) * kSeg + (xr & 31) * 2};
  const int rowseg = (pitch >> 5) * kSeg;            // elements of one lattice row

  auto map_row = [&](int v) {
    if (py) {
      while (v < 0) v += ny;
      while (v >= ny) v -= ny;
      return v;
    }
    return v < 0 ? 0 : (v >= ny ? ny - 1 : v);
  };
  auto indicator = [&](const T fr_[9], const T fb_[9], T& sr, T& sb) -> T {
    sr = fr_[0];
    sb = fb_[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      sr += fr_[a];
      sb += fb_[a];
    }
    if constexpr (kF32) {
      const T v = (sr - sb) * rcp_(sr + sb);
      return sb == T(0) ? T(1) : (sr == T(0) ? T(-1) : v);
    } else {
      return (sr - sb) / (sr + sb);
    }
  };

  int ym3 = 0, ym2 = 0, ym1 = 0, ym0 = 0;       // mapped rows r-3 .. r
  int s4 = 0, s3 = 1, s2 = 2, s1 = 3, s0 = 4;   // rho^N/flag ring slots of rows r-4 .. r
  int n2 = 0, n1 = 1, n0 = 2;                   // n ring slots of rows r-3, r-2, r-1

  for (int r = ys - 2; r <= ye + 1; ++r) {
    {
      const int t4 = s4;
      s4 = s3;
      s3 = s2;
      s2 = s1;
      s1 = s0;
      s0 = t4;
      if (r == ys - 2) {
        ym3 = map_row(r - 3);
        ym2 = map_row(r - 2);
        ym1 = map_row(r - 1);
      } else {
        ym3 = ym2;
        ym2 = ym1;
        ym1 = ym0;
      }
      ym0 = map_row(r);
    }
    // the collision of row p = r - 2 (stage 3) needs that row's populations: issue their loads
    // now, so that they travel while stages 1 and 2 run
    const int p = r - 2;
    const bool collide = p >= ys && interior && !(sfl[s2][t] & F_SOLID);
    const int kn = ym2 * rowseg + colk[1];
    RawNode<S> pre;
    uint8_t mask = 0;
    const bool pre_ok = collide && checked(in_extent(kn, 8 * kDir + 2, 18 * sL.plane) &&
                                               in_extent((long long)ym2 * pitch + xm, 1, sL.plane), A.err);
    if (pre_ok) {
      pre.load(src + kn);
      mask = nbm[ym2 * pitch + xm];
    }
    // ---- stage 1: rho^N and flags of row r
    {
      const bool f_ok = checked(in_extent((long long)ym0 * pitch + xm, 1, sL.plane) &&
                                    in_extent((long long)ym0 * rowseg + colk[1], 8 * kDir + 2, 18 * sL.plane), A.err);
      const uint8_t f = f_ok ? fl[ym0 * pitch + xm] : uint8_t(F_SOLID);
      T v = T(0);
      if (!(f & F_SOLID)) {
        T hr[9], hb[9], a1, a2;
        load_raw<S>(src + ym0 * rowseg + colk[1], r0, hr, hb);
        if (inout) zou_he<T>(xm, nx, inlet_u<T>(sL, ym0), rho_out, hr, hb);
        v = indicator(hr, hb, a1, a2);
      }
      srn[s0][t] = v;
      sfl[s0][t] = f;
    }
    __syncthreads();
    // ---- stage 2: grad rho^N and n of row q = r - 1 (columns 1 .. NTH-2)
    {
      const int tn = n2;  // the slot of row r-4 is reused for row r-1
      n2 = n1;
      n1 = n0;
      n0 = tn;
    }
    if (r - 1 >= ys - 1 && t >= 1 && t < NTH - 1) {
      const uint8_t f = sfl[s1][tc];
      T ax = T(0), ay = T(0), nxv = T(0), nyv = T(0);
      if (!(f & F_SOLID)) {
        if ((f & F_OFB) && checked(in_extent((long long)ym1 * pitch + kxs, 1, sL.plane), A.err)) {
          const int k = ym1 * pitch + kxs;
          ax = wall[k];
          ay = wall[NTOT + k];
          nxv = wall[2 * NTOT + k];
          nyv = wall[3 * NTOT + k];
        } else {
          const T* rm = srn[s2];
          const T* rc = srn[s1];
          const T* rp = srn[s0];
          // Eq. 28 over the 8 neighbours
          const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
          ax = w1 * (rc[tc + 1] - rc[tc - 1]) + w2 * (rp[tc + 1] - rp[tc - 1] + rm[tc + 1] - rm[tc - 1]);
          ay = w1 * (rp[tc] - rm[tc]) + w2 * (rp[tc + 1] + rp[tc - 1] - rm[tc - 1] - rm[tc + 1]);
          ax *= T(3);
          ay *= T(3);
          const T m2 = ax * ax + ay * ay;
          if constexpr (kF32) {
            if (m2 > eps * eps) {
              const T inv = rsqrtf(m2);
              nxv = ax * inv;
              nyv = ay * inv;
            }
          } else {
            const T m = sqrt(m2);
            if (m > eps) {
              nxv = ax / m;
              nyv = ay / m;
            }
          }
        }
      } else if (f & F_OSOLID) {
        // virtual n (Eq. 29) from the stored n of the neighbouring outermost fluid nodes
        T vx = T(0), vy = T(0), den = T(0);
        const int yr[3] = {ym2, ym1, ym0};
        const int sr[3] = {s2, s1, s0};
#pragma unroll
        for (int b = 1; b < 9; ++b) {
          if (!(sfl[sr[ey(b) + 1]][tc + ex(b)] & F_SOLID)) {
            const int k2 = yr[ey(b) + 1] * pitch + wrap_or_clamp(sp.y - 2 + tc + ex(b), nx, px);
            if (!checked(in_extent(k2, 1, sL.plane), A.err)) continue;
            vx += wgt<T>(b) * wall[2 * NTOT + k2];
            vy += wgt<T>(b) * wall[3 * NTOT + k2];
            den += wgt<T>(b);
          }
        }
        if (den > T(0)) {
          nxv = vx / den;
          nyv = vy / den;
        }
      }
      sn[n0][t] = P::mk(nxv, nyv);
      sg[n0][t] = P::mk(ax, ay);
    }
    __syncthreads();
    // ---- stage 3: collide and push row p = r - 2 (flags slot s2, n rows in n2, n1, n0)
    if (!collide) continue;
    const uint8_t myf = sfl[s2][t];
    T fr[9], fb[9];
    pre.decode_to(r0, fr, fb);
    if (inout) zou_he<T>(xm, nx, inlet_u<T>(sL, ym2), rho_out, fr, fb);
    T rhoR, rhoB;
    const T rn = indicator(fr, fb, rhoR, rhoB);
    // grad n (Eq. 28) on (n_x, n_y) pairs, then the curvature (Eq. 13)
    const V* nm = sn[n2];
    const V* n0v = sn[n1];
    const V* np = sn[n0];
    const V W1 = P::mk(T(1.0 / 9.0), T(1.0 / 9.0)), W2 = P::mk(T(1.0 / 36.0), T(1.0 / 36.0));
    const V nm_l = nm[t - 1], nm_c = nm[t], nm_r = nm[t + 1];
    const V n0_l = n0v[t - 1], n0_c = n0v[t], n0_r = n0v[t + 1];
    const V np_l = np[t - 1], np_c = np[t], np_r = np[t + 1];
    // d_x (n_x, n_y) and d_y (n_x, n_y)
    const V dX = P::fma(W1, P::sub(n0_r, n0_l), P::mul(W2, P::add(P::sub(np_r, np_l), P::sub(nm_r, nm_l))));
    const V dY = P::fma(W1, P::sub(np_c, nm_c), P::mul(W2, P::sub(P::add(np_r, np_l), P::add(nm_l, nm_r))));
    T dxx = dX.x, dyx = dX.y, dxy = dY.x, dyy = dY.y;
    if (sL.wetting == 1 && (myf & F_OFB)) {
      const V* rows3[3] = {nm, n0v, np};
      T nxs[9], nys[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const V v = rows3[ey(a) + 1][t + ex(a)];
        nxs[a] = v.x;
        nys[a] = v.y;
      }
      grad_n_scheme_b<T>(nxs, nys, mask, dxx, dyx, dxy, dyy);
    }
    const T nxo = n0_c.x, nyo = n0_c.y;
    const T kappa = T(3) * (-nxo * nxo * dyy - nyo * nyo * dxx + nxo * nyo * (dxy + dyx));
    const T hsk = T(0.5) * sigma * kappa;
    const V gv = sg[n1][t];
    const T Fx = hsk * gv.x;
    const T Fy = hsk * gv.y;

    T f[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = fr[a] + fb[a];
    const T rho = rhoR + rhoB;
    const T irho = rcp_(rho);
    const T jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const T jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const T ux = (jx + T(0.5) * Fx) * irho;
    const T uy = (jy + T(0.5) * Fy) * irho;
    const T inv_nu = (T(1) + rn) * hR + (T(1) - rn) * hB;
    const T sv = inv_nu * rcp_(T(3) + T(0.5) * inv_nu);
    const T s14 = f[1] + f[2] + f[3] + f[4];
    const T s58 = f[5] + f[6] + f[7] + f[8];
    const T me = T(-4) * f[0] - s14 + T(2) * s58;
    const T meps = T(4) * f[0] - T(2) * s14 + s58;
    const T qx = T(-2) * (f[1] - f[3]) + (f[5] - f[6] - f[7] + f[8]);
    const T qy = T(-2) * (f[2] - f[4]) + (f[5] + f[6] - f[7] - f[8]);
    const T pxx = f[1] - f[2] + f[3] - f[4];
    const T pxy = f[5] - f[6] + f[7] - f[8];
    const T u2 = ux * ux + uy * uy;
    const T uF = ux * Fx + uy * Fy;
    const T De = se * (me - rho * (T(-2) + T(3) * u2)) - (T(1) - T(0.5) * se) * (T(6) * uF);
    const T Deps = seps * (meps - rho * (T(1) - T(3) * u2)) + (T(1) - T(0.5) * seps) * (T(6) * uF);
    const T Dqx = sq * (qx + rho * ux) + (T(1) - T(0.5) * sq) * Fx;
    const T Dqy = sq * (qy + rho * uy) + (T(1) - T(0.5) * sq) * Fy;
    const T Dxx = sv * (pxx - rho * (ux * ux - uy * uy)) - (T(1) - T(0.5) * sv) * (T(2) * (ux * Fx - uy * Fy));
    const T Dxy = sv * (pxy - rho * ux * uy) - (T(1) - T(0.5) * sv) * (ux * Fy + uy * Fx);
    const T ae = De * T(1.0 / 36.0), aeps = Deps * T(1.0 / 36.0);
    const T ajx = -Fx * T(1.0 / 6.0), ajy = -Fy * T(1.0 / 6.0);
    const T aqx = Dqx * T(1.0 / 12.0), aqy = Dqy * T(1.0 / 12.0);
    const T axx = Dxx * T(0.25), axy = Dxy * T(0.25);
    T fp[9];
    fp[0] = f[0] - (T(-4) * ae + T(4) * aeps);
    const T c14 = -ae - T(2) * aeps;
    fp[1] = f[1] - (c14 + ajx - T(2) * aqx + axx);
    fp[2] = f[2] - (c14 + ajy - T(2) * aqy - axx);
    fp[3] = f[3] - (c14 - ajx + T(2) * aqx + axx);
    fp[4] = f[4] - (c14 - ajy + T(2) * aqy - axx);
    const T c58 = T(2) * ae + aeps;
    fp[5] = f[5] - (c58 + ajx + aqx + ajy + aqy + axy);
    fp[6] = f[6] - (c58 - ajx - aqx + ajy + aqy - axy);
    fp[7] = f[7] - (c58 - ajx - aqx - ajy - aqy + axy);
    fp[8] = f[8] - (c58 + ajx + aqx - ajy - aqy - axy);
    const T cR = rhoR * irho;
    const T pc = beta * rhoR * rhoB * irho;
    // streaming (Eq. 15) to rows p-1, p, p+1 and columns cx-1, cx, cx+1
    const int rowk[3] = {ym3 * rowseg, ym2 * rowseg, ym1 * rowseg};
    if (mask == 0 && !(myf & F_EDGE)) {
      // bulk node: every neighbour is a fluid node of the lattice
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const T pert = pc * wgt<T>(a) * (T(ex(a)) * nxo + T(ey(a)) * nyo);
        const T oR = cR * fp[a] + pert;   // Eq. 14; the blue share is the rest of f'_a
        const long long q = (long long)rowk[ey(a) + 1] + colk[ex(a) + 1] + a * kDir;
        if (checked(in_extent(q, 2, 18 * sL.plane), A.err)) store_pair<S>(dst + q, oR, fp[a] - oR, wgt<T>(a) * r0);
      }
    } else {
      // half-way bounce-back into the opposite slot where the neighbour is solid; dropped
      // where it lies beyond an open edge
      const bool okx[3] = {px || cx - 1 >= 0, true, px || cx + 1 < nx};
      const bool oky[3] = {py || p - 1 >= 0, true, py || p + 1 < ny};
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const T pert = pc * wgt<T>(a) * (T(ex(a)) * nxo + T(ey(a)) * nyo);
        const T oR = cR * fp[a] + pert;
        const T oB = fp[a] - oR;
        int k = kn + a * kDir;
        if (a != 0) {
          if (!(okx[ex(a) + 1] && oky[ey(a) + 1])) continue;
          if (mask & (1u << (a - 1))) k = kn + opp(a) * kDir;
          else k = rowk[ey(a) + 1] + colk[ex(a) + 1] + a * kDir;
        }
        if (checked(in_extent(k, 2, 18 * sL.plane), A.err)) store_pair<S>(dst + k, oR, oB, wgt<T>(a) * r0);
      }
    }
  }
}

// ------------------------------------------------------------------ k_sweepf (FP32 arithmetic)
// The y-sweep of k_sweep for the storage forms that compute in FP32, arranged so that no
// value is fetched from memory twice and no load is waited on right after it is issued:
//  - one thread issues bulk copies (cp.async.bulk, completing on an mbarrier) of row r + 1's
//    32-node population segments and of its flag and neighbour-mask bytes into the other of
//    two shared-memory slots while row r is processed; every thread waits with a bound;
//  - stage 1 keeps what the collision of the row needs, the nine totals f_a = f_a,R + f_a,B
//    and (rho_R, rho_B), in registers until the end of the iteration and then in a two-row
//    ring in shared memory that only the owning thread reads, so the collision two rows later
//    neither reloads nor re-sums the populations; the thread's colour gradient is carried to
//    that collision in registers (42 KB of shared memory per block: 5 blocks per SM in FP32);
//  - the moment sums and the back-transform share partial sums (fewer FP32 operations);
//  - 16-bit storage takes the totals straight from the stored deviations and forms the stored
//    pairs from f' directly, with stochastic rounding (store_scale, stp_sr).
// ---- bulk asynchronous copies (global -> shared) completing on an mbarrier
__device__ __forceinline__ unsigned smem_addr(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// generic-proxy reads of a buffer are ordered before the async-proxy write that reuses it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// bounded wait for the completion of the barrier phase of the given parity: false after
// `polls` unsuccessful polls (the default bound, kMbarPolls, is about a second)
constexpr int kMbarPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int polls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// segments of a staged row: the (at most 5) contiguous ones holding the strip's columns; the
// columns a periodic strip wraps to are loaded directly
constexpr int kStageSegs = 5;
template <typename S>
constexpr int sweepf_dyn_smem() { return 2 * kStageSegs * kSeg * int(sizeof(S)); }

template <typename S>
__device__ __forceinline__ void staged_pair(const S* row, int a, float& lo, float& hi) {
  if constexpr (sizeof(S) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(row + a * kDir);
    lo = v.x;
    hi = v.y;
  } else {
    Store<S>::unpack(*reinterpret_cast<const uint32_t*>(row + a * kDir), lo, hi);
  }
}

// kSchemeB: compiled in only for batches with a scheme-(b) lattice (the branch costs registers)
template <typename S, int NTH, bool kSchemeB>
__global__ void __launch_bounds__(NTH, sizeof(S) == 4 ? kSweepFMinBlocks : kSweepFMinBlocks16) k_sweepf(SweepArgs A) {
  using T = float;
  // rho^N / flag / neighbour-mask ring of rows r-2 .. r: row r takes row r-3's slot in stage 1
  // of iteration r; row r-3's last readers were stage 2 of iteration r-1 (other threads, before
  // that iteration's barriers) and stage 3 of iteration r-1 (only the owning thread)
  constexpr int RR = 3;
  constexpr int RN = 3;   // n, grad ring (rows r-3 .. r-1)
  constexpr int RF = 2;   // f totals / (rho_R, rho_B) ring (rows r-2, r-1; row r is written last)
  using P = Pair<T>;
  using V = typename P::V;
  __shared__ T srn[RR][NTH];
  __shared__ uint8_t sfl[RR][NTH];
  __shared__ V sn[RN][NTH];
  __shared__ T sf[RF][9][NTH];
  __shared__ V srb[RF][NTH];
  __shared__ LatDev sL;
  // two staged rows of populations (dynamic shared memory): [slot][kStageSegs * kSeg]
  extern __shared__ __align__(128) unsigned char sraw_bytes[];
  S* sraw = reinterpret_cast<S*>(sraw_bytes);
  __shared__ __align__(8) uint64_t sbar[2];
  // the staged rows' flags and neighbour-solid masks ([slot][0: flags, 1: mask][byte]), and the
  // mask of rows r-2 .. r for the collision two rows later
  __shared__ __align__(16) uint8_t sfg[2][2][NTH + 32];
  __shared__ uint8_t snb[RR][NTH];

  const int4 sp = A.strips[blockIdx.x];
  const int t = threadIdx.x;
  const bool down = (sp.x & kStripDown) != 0;
  if (t == 0) sL = A.lats[sp.x & ~kStripDown];
  __syncthreads();
  const int nx = sL.nx, ny = sL.ny, pitch = sL.pitch;
  const bool px = sL.bcx == BC_PERIODIC, py = sL.bcy == BC_PERIODIC, inout = sL.bcx == BC_INOUT;
  const T r0 = T(sL.rho0), rho_out = T(sL.rho_out), eps2 = T(sL.grad_eps) * T(sL.grad_eps);
  const T hsig = T(0.5) * T(sL.sigma), beta = T(sL.beta), se = T(sL.s_e), seps = T(sL.s_eps), sq = T(sL.s_q);
  const T kDe = T(-6) * (T(1) - T(0.5) * se), kDeps = T(6) * (T(1) - T(0.5) * seps), kq = T(1) - T(0.5) * sq;
  const T hdiff = T(sL.h_inv_nuR) - T(sL.h_inv_nuB), hsum = T(sL.h_inv_nuR) + T(sL.h_inv_nuB);
  const uint8_t* __restrict__ fl = A.flags + sL.node_off;
  const uint8_t* __restrict__ nbm = A.nbmask + sL.node_off;
  const S* __restrict__ src = static_cast<const S*>(A.src) + sL.pop_off;
  S* __restrict__ dst = static_cast<S*>(A.dst) + sL.pop_off;
  uint32_t srk = 0;
  if constexpr (Store<S>::kDeviation) srk = sr_key(A.sr_epoch, A.sr_step, sL.pop_off);

  const int cx = sp.y - 2 + t;
  const int xm = wrap_or_clamp(cx, nx, px);
  const int xl = wrap_or_clamp(cx - 1, nx, px), xr = wrap_or_clamp(cx + 1, nx, px);
  const int tc = px ? t : min(max(t + xm - cx, 1), NTH - 2);
  const int kxs = wrap_or_clamp(sp.y - 2 + tc, nx, px);
  const bool interior = t >= 2 && t < NTH - 2 && cx < nx;
  const bool edge = inout && (xm == 0 || xm == nx - 1);
  const int ys = sp.z, ye = sp.w;
  // the sweep runs over rows r = ys - 2 .. ye + 1 in this order; yrow(r) is the lattice row
  // (before wrapping) that sweep row r stands for: r itself, or the mirror image in the
  // segment for a downward sweep, whose stencils then take row r - 1 of the sweep as y + 1
  const int yflip = ys + ye - 1;
  auto yrow = [&](int r) { return down ? yflip - r : r; };
  const int colk[3] = {(xl >> 5) * kSeg + (xl & 31) * 2, (xm >> 5) * kSeg + (xm & 31) * 2,
                       (xr >> 5) * kSeg + (xr & 31) * 2};
  const int rowseg = (pitch >> 5) * kSeg;
  // staged segments of this strip: [sA, sB] holds columns max(x0-2, 0) .. min(x0+125, nx-1).
  // soff: this column's offset in a staged row, -1 if its segment is not staged (a column a
  // periodic edge strip wraps to; it is then loaded directly).
  const int sA = max(sp.y - 2, 0) >> 5, sB = min(sp.y + NTH - 3, nx - 1) >> 5;
  const int soff = ((xm >> 5) >= sA && (xm >> 5) <= sB) ? ((xm >> 5) - sA) * kSeg + (xm & 31) * 2 : -1;
  const unsigned bytesA = unsigned((sB - sA + 1) * kSeg * sizeof(S));
  // flag / mask bytes of the strip's columns, from a 16-byte boundary, a multiple of 16 long
  // (the 32-aligned pitch keeps it inside the row); fo: this column's byte, -1 if outside
  const int fx0 = max(sp.y - 2, 0) & ~15;
  const unsigned fbytes = unsigned((min(sp.y + NTH - 3, nx - 1) - fx0 + 16) & ~15);
  const int fo = (xm >= fx0 && xm < fx0 + int(fbytes)) ? xm - fx0 : -1;
  // extents of this lattice's populations and node arrays (range checks of the checked build)
  const long long pop_n = 18 * sL.plane, node_n = sL.plane;
  int* const err = A.err;

  auto map_row = [&](int v) {
    if (py) {
      while (v < 0) v += ny;
      while (v >= ny) v -= ny;
      return v;
    }
    return v < 0 ? 0 : (v >= ny ? ny - 1 : v);
  };

  int ym3 = 0, ym2 = 0, ym1 = 0, ym0 = 0;
  int s2 = 0, s1 = 1, s0 = 2;   // ring slots of rows r-2, r-1, r
  int n2 = 0, n1 = 1, n0 = 2;
  int q2 = 0, q1 = 1;   // f-total slots of rows r-2 and r-1
  // thread-private values carried between rows in registers: the f totals and (rho_R, rho_B)
  // of row r until they take the slot of row r-2 at the end of the iteration, and the colour
  // gradient (stage 2, row r-1) until the collision of that row one iteration later
  T ft[9];
  V rbt = P::mk(T(0), T(0)), g_new = P::mk(T(0), T(0)), g_old = P::mk(T(0), T(0));
  bool ft_ok = false;
  unsigned phase = 0;     // bit s: parity of the next completion of slot s
  bool lost = false;      // this thread's wait for a staged row ran out
  // issue the bulk copies of (mapped) row y into staging slot `slot` (one thread)
  auto stage_row = [&](int y, int slot) {
    S* d = sraw + slot * (kStageSegs * kSeg);
    const S* g = src + (long long)y * rowseg;
    if (!checked(in_extent((long long)y * rowseg + sA * kSeg, bytesA / sizeof(S), pop_n) &&
                     bytesA <= unsigned(kStageSegs * kSeg * sizeof(S)) &&
                     in_extent((long long)y * pitch + fx0, fbytes, node_n) && fbytes <= unsigned(NTH + 32),
                 err)) {
      mbar_expect_tx(&sbar[slot], 0);   // completes the phase without data
      return;
    }
    fence_proxy_async();
    mbar_expect_tx(&sbar[slot], bytesA + 2 * fbytes);
    bulk_copy_g2s(d, g + sA * kSeg, bytesA, &sbar[slot]);
    bulk_copy_g2s(&sfg[slot][0][0], fl + (long long)y * pitch + fx0, fbytes, &sbar[slot]);
    bulk_copy_g2s(&sfg[slot][1][0], nbm + (long long)y * pitch + fx0, fbytes, &sbar[slot]);
  };
  if (t == 0) {
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (t == 0) stage_row(map_row(yrow(ys - 2)), (ys - 2) & 1);

  // one row of the sweep; false once some thread of the block lost its wait for the row
  auto body = [&](const int r) -> bool {
    {
      const int t2 = s2;
      s2 = s1;
      s1 = s0;
      s0 = t2;
      const int tq = q2;
      q2 = q1;
      q1 = tq;
      g_old = g_new;
      if (r == ys - 2) {
        ym3 = map_row(yrow(r - 3));
        ym2 = map_row(yrow(r - 2));
        ym1 = map_row(yrow(r - 1));
      } else {
        ym3 = ym2;
        ym2 = ym1;
        ym1 = ym0;
      }
      ym0 = map_row(yrow(r));
    }
    // the next row's populations (bulk copy) and flag travel while this row is processed;
    // its slot held row r - 1, whose last reader finished before the previous barriers
    if (r + 1 <= ye + 1) {
      const int y = map_row(yrow(r + 1));
      if (t == 0) stage_row(y, (r + 1) & 1);
    }
    const int p = r - 2;
    const bool collide = p >= ys && interior && !(sfl[s2][t] & F_SOLID);
    const uint8_t mask = collide ? snb[s2][t] : 0;
    // ---- stage 1: rho^N, totals and colour densities of row r
    {
      T v = T(0);
      const int slot = r & 1;
      // (after a lost wait this row's values are garbage: the block stops at the barrier below)
      if (!mbar_wait(&sbar[slot], (phase >> slot) & 1u, A.poll_limit)) lost = true;
      phase ^= 1u << slot;
      const bool fl_ok = fo >= 0 || checked(in_extent((long long)ym0 * pitch + xm, 1, node_n), err);
      const uint8_t f_r = fo >= 0 ? sfg[slot][0][fo] : (fl_ok ? fl[ym0 * pitch + xm] : uint8_t(F_SOLID));
      snb[s0][t] = fo >= 0 ? sfg[slot][1][fo] : (fl_ok ? nbm[ym0 * pitch + xm] : uint8_t(0));
      if (!(f_r & F_SOLID)) {
        T sr, sb;
        bool done = false;
        if constexpr (Store<S>::kDeviation) {
          // deviation storage, staged, not a Zou-He column: the totals f = w rho0 + d / K and
          // the colour difference sum(g) / K come straight from the stored pairs
          if (soff >= 0 && !edge) {
            constexpr float inv = 1.0f / store_scale<S>(), hinv = 0.5f / store_scale<S>();
            const S* row = sraw + slot * (kStageSegs * kSeg) + soff;
            T rho = T(0), gsum = T(0);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
              T lo, hi;
              staged_pair<S>(row, a, lo, hi);
              ft[a] = fmaf(lo, inv, wgt<T>(a) * r0);
              rho += ft[a];
              gsum += hi;
            }
            const T hr = T(0.5) * rho;
            sr = fmaf(gsum, hinv, hr);
            sb = fmaf(-gsum, hinv, hr);
            done = true;
          }
        }
        if (!done) {
        T fr[9], fb[9];
        if (soff >= 0) {
          const S* row = sraw + slot * (kStageSegs * kSeg) + soff;
#pragma unroll
          for (int a = 0; a < 9; ++a) {
            T lo, hi;
            staged_pair<S>(row, a, lo, hi);
            decode<S, T>(lo, hi, wgt<T>(a) * r0, fr[a], fb[a]);
          }
        } else if (checked(in_extent((long long)ym0 * rowseg + colk[1], 8 * kDir + 2, pop_n), err)) {
          load_raw<S>(src + ym0 * rowseg + colk[1], r0, fr, fb);
        } else {
#pragma unroll
          for (int a = 0; a < 9; ++a) fr[a] = fb[a] = T(0);
        }
        if (edge) zou_he<T>(xm, nx, inlet_u<T>(sL, ym0), rho_out, fr, fb);
        V srb_ = P::add(P::mk(fr[0], fb[0]), P::mk(fr[1], fb[1]));
#pragma unroll
        for (int a = 2; a < 9; ++a) srb_ = P::add(srb_, P::mk(fr[a], fb[a]));
#pragma unroll
        for (int a = 0; a < 9; ++a) ft[a] = fr[a] + fb[a];
        sr = srb_.x;
        sb = srb_.y;
        }
        rbt = P::mk(sr, sb);
        const T w = (sr - sb) * rcp_(sr + sb);
        v = sb == T(0) ? T(1) : (sr == T(0) ? T(-1) : w);
      }
      ft_ok = !(f_r & F_SOLID);
      srn[s0][t] = v;
      sfl[s0][t] = f_r;
    }
    // every thread has seen row r, or the block stops here (before it writes anything of
    // this row or the rows after it)
    if (__syncthreads_or(lost)) return false;
    // ---- stage 2: grad rho^N and n of row r - 1
    {
      const int tn = n2;
      n2 = n1;
      n1 = n0;
      n0 = tn;
    }
    if (r - 1 >= ys - 1 && t >= 1 && t < NTH - 1) {
      const uint8_t f = sfl[s1][tc];
      T ax = T(0), ay = T(0), nxv = T(0), nyv = T(0);
      if (!(f & F_SOLID)) {
        if ((f & F_OFB) && checked(in_extent((long long)ym1 * pitch + kxs, 1, sL.plane), A.err)) {
          const long long NTOT = A.node_total;
          const T* wall = static_cast<const T*>(A.wall) + sL.node_off;
          const int k = ym1 * pitch + kxs;
          ax = wall[k];
          ay = wall[NTOT + k];
          nxv = wall[2 * NTOT + k];
          nyv = wall[3 * NTOT + k];
        } else {
          const T* rm = srn[down ? s0 : s2];   // rows y - 1, y, y + 1
          const T* rc = srn[s1];
          const T* rp = srn[down ? s2 : s0];
          const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
          ax = w1 * (rc[tc + 1] - rc[tc - 1]) + w2 * (rp[tc + 1] - rp[tc - 1] + rm[tc + 1] - rm[tc - 1]);
          ay = w1 * (rp[tc] - rm[tc]) + w2 * (rp[tc + 1] + rp[tc - 1] - rm[tc - 1] - rm[tc + 1]);
          ax *= T(3);
          ay *= T(3);
          const T m2 = ax * ax + ay * ay;
          if (m2 > eps2) {
            const T inv = rsqrtf(m2);
            nxv = ax * inv;
            nyv = ay * inv;
          }
        }
      } else if (f & F_OSOLID) {
        const long long NTOT = A.node_total;
        const T* wall = static_cast<const T*>(A.wall) + sL.node_off;
        T vx = T(0), vy = T(0), den = T(0);
        const int yr[3] = {down ? ym0 : ym2, ym1, down ? ym2 : ym0};   // rows y - 1, y, y + 1
        const int sr[3] = {down ? s0 : s2, s1, down ? s2 : s0};
#pragma unroll
        for (int b = 1; b < 9; ++b) {
          if (!(sfl[sr[ey(b) + 1]][tc + ex(b)] & F_SOLID)) {
            const int k2 = yr[ey(b) + 1] * pitch + wrap_or_clamp(sp.y - 2 + tc + ex(b), nx, px);
            if (!checked(in_extent(k2, 1, sL.plane), A.err)) continue;
            vx += wgt<T>(b) * wall[2 * NTOT + k2];
            vy += wgt<T>(b) * wall[3 * NTOT + k2];
            den += wgt<T>(b);
          }
        }
        if (den > T(0)) {
          nxv = vx / den;
          nyv = vy / den;
        }
      }
      sn[n0][t] = P::mk(nxv, nyv);
      g_new = P::mk(ax, ay);
    }
    __syncthreads();
    // ---- stage 3: collide and push row p = r - 2; then row r's totals take row p's slot
    if (collide) {
    const uint8_t myf = sfl[s2][t];
    T f[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = sf[q2][a][t];
    const V rb = srb[q2][t];
    const T rhoR = rb.x, rhoB = rb.y, rn = srn[s2][t];
    // grad n (Eq. 28), curvature (Eq. 13), force (Eq. 10)
    const V* nm = sn[down ? n0 : n2];   // n of rows y - 1, y, y + 1
    const V* n0v = sn[n1];
    const V* np = sn[down ? n2 : n0];
    const V W1 = P::mk(T(1.0 / 9.0), T(1.0 / 9.0)), W2 = P::mk(T(1.0 / 36.0), T(1.0 / 36.0));
    const V nm_l = nm[t - 1], nm_c = nm[t], nm_r = nm[t + 1];
    const V n0_l = n0v[t - 1], n0_c = n0v[t], n0_r = n0v[t + 1];
    const V np_l = np[t - 1], np_c = np[t], np_r = np[t + 1];
    V dX = P::fma(W1, P::sub(n0_r, n0_l), P::mul(W2, P::add(P::sub(np_r, np_l), P::sub(nm_r, nm_l))));
    V dY = P::fma(W1, P::sub(np_c, nm_c), P::mul(W2, P::sub(P::add(np_r, np_l), P::add(nm_l, nm_r))));
    if constexpr (kSchemeB) {
      if (sL.wetting == 1 && (myf & F_OFB)) {
        const V* rows3[3] = {nm, n0v, np};
        T nxs[9], nys[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          const V v = rows3[ey(a) + 1][t + ex(a)];
          nxs[a] = v.x;
          nys[a] = v.y;
        }
        grad_n_scheme_b<T>(nxs, nys, mask, dX.x, dX.y, dY.x, dY.y);
      }
    }
    const T nxo = n0_c.x, nyo = n0_c.y;
    const T kappa = T(3) * (-nxo * nxo * dY.y - nyo * nyo * dX.x + nxo * nyo * (dY.x + dX.y));
    const T hsk = hsig * kappa;
    const V gv = g_old;
    const T Fx = hsk * gv.x, Fy = hsk * gv.y;
    // moments (Eq. 3) from shared partial sums
    const T p13 = f[1] + f[3], m13 = f[1] - f[3], p24 = f[2] + f[4], m24 = f[2] - f[4];
    const T p57 = f[5] + f[7], m57 = f[5] - f[7], p68 = f[6] + f[8], m68 = f[6] - f[8];
    const T s14 = p13 + p24, pxx = p13 - p24, s58 = p57 + p68, pxy = p57 - p68;
    const T Bx = m57 - m68, Dy = m57 + m68;   // f5 - f6 - f7 + f8, f5 + f6 - f7 - f8
    const T jx = m13 + Bx, jy = m24 + Dy;
    const T qx = fmaf(T(-2), m13, Bx), qy = fmaf(T(-2), m24, Dy);
    const T me = fmaf(T(-4), f[0], fmaf(T(2), s58, -s14));
    const T meps = fmaf(T(4), f[0], fmaf(T(-2), s14, s58));
    // velocity (Eq. 17), relaxation rate of the viscous moments (Eq. 5, 18)
    const T rho = rhoR + rhoB;
    const T irho = rcp_(rho);
    const T ux = fmaf(T(0.5), Fx, jx) * irho;
    const T uy = fmaf(T(0.5), Fy, jy) * irho;
    const T inv_nu = fmaf(rn, hdiff, hsum);
    const T sv = inv_nu * rcp_(fmaf(T(0.5), inv_nu, T(3)));
    // non-equilibrium moments with the Guo source (Eq. 1-9)
    const T uy2 = uy * uy, uyF = uy * Fy;
    const T u2 = fmaf(ux, ux, uy2), uF = fmaf(ux, Fx, uyF);
    const T De = fmaf(se, fmaf(-rho, fmaf(T(3), u2, T(-2)), me), kDe * uF);
    const T Deps = fmaf(seps, fmaf(-rho, fmaf(T(-3), u2, T(1)), meps), kDeps * uF);
    const T Dqx = fmaf(sq, fmaf(rho, ux, qx), kq * Fx);
    const T Dqy = fmaf(sq, fmaf(rho, uy, qy), kq * Fy);
    const T csv = fmaf(T(-0.5), sv, T(1));
    const T Dxx = fmaf(sv, fmaf(-rho, fmaf(ux, ux, -uy2), pxx), -csv * (T(2) * fmaf(ux, Fx, -uyF)));
    const T Dxy = fmaf(sv, fmaf(-rho * ux, uy, pxy), -csv * fmaf(ux, Fy, uy * Fx));
    // back to populations: f' = f - M^-1 Delta, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const T ae = De * T(1.0 / 36.0), aeps = Deps * T(1.0 / 36.0);
    const T axx = Dxx * T(0.25), axy = Dxy * T(0.25);
    const T U1 = T(-1.0 / 6.0) * (Dqx + Fx), U2 = T(-1.0 / 6.0) * (Dqy + Fy);   // a_jx - 2 a_qx, a_jy - 2 a_qy
    const T X = fmaf(T(1.0 / 12.0), Dqx, T(-1.0 / 6.0) * Fx);                     // a_jx + a_qx
    const T Y = fmaf(T(1.0 / 12.0), Dqy, T(-1.0 / 6.0) * Fy);                     // a_jy + a_qy
    const T c14 = fmaf(T(-2), aeps, -ae), c58 = fmaf(T(2), ae, aeps);
    const T T13 = c14 + axx, T24 = c14 - axx, Pp = c58 + axy, Qm = c58 - axy;
    const T XpY = X + Y, XmY = X - Y;
    T fp[9];
    fp[0] = fmaf(T(4), ae - aeps, f[0]);
    fp[1] = (f[1] - T13) - U1;
    fp[3] = (f[3] - T13) + U1;
    fp[2] = (f[2] - T24) - U2;
    fp[4] = (f[4] - T24) + U2;
    fp[5] = (f[5] - Pp) - XpY;
    fp[7] = (f[7] - Pp) + XpY;
    fp[6] = (f[6] - Qm) + XmY;
    fp[8] = (f[8] - Qm) - XmY;
    // recolouring (Eq. 14): oR = (rho_R / rho) f' + beta (rho_R rho_B / rho) w_a e_a.n, oB = f' - oR
    // 16-bit storage stores d = K (f' - w rho0) and g = K (oR - oB) = K ((2 cR - 1) f' + 2 pert),
    // formed from f' directly: the perturbation is scaled by 2K here
    constexpr float kK = store_scale<S>();
    constexpr float kP = Store<S>::kDeviation ? 2.0f * kK : 1.0f;
    const T cR = rhoR * irho;
    const T pc = beta * rhoR * (rhoB * irho);
    const T c1 = pc * T(kP / 9.0), c2 = pc * T(kP / 36.0);
    T pert[9];
    pert[0] = T(0);
    pert[1] = c1 * nxo;
    pert[2] = c1 * nyo;
    pert[3] = -pert[1];
    pert[4] = -pert[2];
    pert[5] = c2 * (nxo + nyo);
    pert[8] = c2 * (nxo - nyo);
    pert[7] = -pert[5];
    pert[6] = -pert[8];
    const int kn = ym2 * rowseg + colk[1];
    const int rowk[3] = {(down ? ym1 : ym3) * rowseg, ym2 * rowseg, (down ? ym3 : ym1) * rowseg};   // y - 1, y, y + 1
    uint32_t srh = 0;
    if constexpr (Store<S>::kDeviation) srh = sr_node(srk, kn);
    const T cg = fmaf(cR, T(2.0f * kK), T(-kK));   // K (2 cR - 1), deviation storage only
    const T nkr0 = T(-kK) * r0;
    // the stored pair of direction a at q
    auto emit = [&](S* q, int a) {
      if (!checked(in_extent(q - dst, 2, pop_n), err)) return;
      if constexpr (Store<S>::kDeviation) {
        Store<S>::stp_sr(q, fmaf(fp[a], T(kK), nkr0 * wgt<T>(a)), fmaf(cg, fp[a], pert[a]), sr_bits(srh, a));
      } else {
        const T oR = fmaf(cR, fp[a], pert[a]);
        store_pair<S>(q, oR, fp[a] - oR, wgt<T>(a) * r0);
      }
    };
    if (mask == 0 && !(myf & F_EDGE)) {
#pragma unroll
      for (int a = 0; a < 9; ++a) emit(dst + rowk[ey(a) + 1] + colk[ex(a) + 1] + a * kDir, a);
    } else {
      const bool okx[3] = {px || cx - 1 >= 0, true, px || cx + 1 < nx};
      const int yp = yrow(p);
      const bool oky[3] = {py || yp - 1 >= 0, true, py || yp + 1 < ny};
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        int k = kn + a * kDir;
        if (a != 0) {
          if (!(okx[ex(a) + 1] && oky[ey(a) + 1])) continue;
          if (mask & (1u << (a - 1))) k = kn + opp(a) * kDir;
          else k = rowk[ey(a) + 1] + colk[ex(a) + 1] + a * kDir;
        }
        emit(dst + k, a);
      }
    }
    }
    if (ft_ok) {
#pragma unroll
      for (int a = 0; a < 9; ++a) sf[q2][a][t] = ft[a];
      srb[q2][t] = rbt;
    }
    return true;
  };

  int r = ys - 2;
  while (r <= ye + 1 && body(r)) ++r;
  if (r <= ye + 1 && t == 0) {
    // Some thread lost its wait for row r: report it, issue no further copies, and do not
    // return with copies into this block's shared memory in flight.  This thread issued
    // row r + 1 into the other slot (if the sweep goes that far) and has not waited for it;
    // row r's slot is outstanding if this thread's own wait for it ran out (its parity bit
    // was flipped regardless, so flip it back).  Wait for each with the default bound.
    int e = ERR_TIMEOUT;
    const int sr = r & 1, sn = sr ^ 1;
    if (lost && !mbar_wait(&sbar[sr], ((phase >> sr) & 1u) ^ 1u, kMbarPolls)) e |= ERR_DRAIN;
    if (r + 1 <= ye + 1 && !mbar_wait(&sbar[sn], (phase >> sn) & 1u, kMbarPolls)) e |= ERR_DRAIN;
    atomicOr(A.err, e);
  }
}

// ------------------------------------------------------------------ layout conversion
// host layout: double [2][9][ny][nx] (f_R block then f_B block) <-> storage pool
template <typename S>
__global__ void k_to_storage(const LatDev* __restrict__ lats, int lat, const double* __restrict__ in,
                             const uint8_t* __restrict__ flags, S* __restrict__ pool) {
  using T = typename Store<S>::T;
  const LatDev& L = lats[lat];
  const long long nn = (long long)L.nx * L.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * nn) return;
  const int a = int(i / nn);
  const long long r = i % nn;
  const int y = int(r / L.nx), x = int(r % L.nx);
  const long long k = (long long)y * L.pitch + x;
  const bool solid = flags[L.node_off + k] & F_SOLID;
  const T fr = solid ? T(0) : T(in[i]);
  const T fb = solid ? T(0) : T(in[9 * nn + i]);
  store_pair<S>(pool + L.pop_off + pop_node(x, y, L.pitch) + a * kDir, fr, fb, solid ? T(0) : wgt<T>(a) * T(L.rho0));
}

// host layout out <- the post-streaming state as a step reads it (Zou-He applied on open edges)
template <typename S>
__global__ void k_from_storage(const LatDev* __restrict__ lats, int lat, const S* __restrict__ pool,
                               const uint8_t* __restrict__ flags, double* __restrict__ out) {
  using T = typename Store<S>::T;
  const LatDev& L = lats[lat];
  const long long nn = (long long)L.nx * L.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int y = int(i / L.nx), x = int(i % L.nx);
  const long long k = (long long)y * L.pitch + x;
  T fr[9], fb[9];
  if (flags[L.node_off + k] & F_SOLID) {
#pragma unroll
    for (int a = 0; a < 9; ++a) fr[a] = fb[a] = T(0);
  } else {
    load_node<S>(L, pool, x, y, fr, fb);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    out[a * nn + i] = double(fr[a]);
    out[(9 + a) * nn + i] = double(fb[a]);
  }
}

// ------------------------------------------------------------------ launchers
// advances the replay counter of the stochastic-rounding keys (once per replayed graph)
__global__ void k_sr_tick(uint32_t* epoch) { *epoch += 1u; }

// launches kernel k on `grid` blocks of `block` threads; with `dep` set, as a programmatic
// dependent launch of the kernel before it in the stream (the kernel's dep_wait orders it)
template <typename... P, typename... Q>
static void launch_k(void (*k)(P...), int grid, int block, cudaStream_t st, bool dep, Q... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(block));
  cfg.stream = st;
  cfg.attrs = dep ? at : nullptr;
  cfg.numAttrs = dep ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);   // errors: cudaGetLastError below
}

template <typename S>
static cudaError_t launch_all(const LaunchStep& p, cudaStream_t st) {
  using T = typename Store<S>::T;
  auto rec = [&](int i) {
    if (p.ev) cudaEventRecord(p.ev[i], st);
  };
  // the tile schedule's steps are dependent launches (not while the kernels are timed one by
  // one with events, nor for the macro-field pass); the sweep's kernels are long enough that
  // it measured no gain there
  const bool tiles = !(p.sweep && p.macro == nullptr);
  const bool dep = tiles && p.ev == nullptr && p.macro == nullptr;
  rec(0);
  if (p.ngroups > 0)
    launch_k(k_wall<S>, p.ngroups, kWallThreads, st, dep, p.lats, p.groups, p.wband, p.wvirt, p.wsten, p.ofb,
             static_cast<const S*>(p.src), static_cast<T*>(p.wall), p.node_total, p.err);
  rec(1);
  rec(2);
  if (p.sweep && p.macro == nullptr) {
    if (p.nstrips > 0) {
      SweepArgs B{p.lats, p.strips, p.src, p.dst, p.flags, p.nbmask, p.wall, p.node_total, p.err, p.sr_epoch,
                  p.sr_step, p.poll_limit};
      if constexpr (sizeof(T) == 4)
      {
        if (p.scheme_b) k_sweepf<S, kSweepThreads, true><<<p.nstrips, kSweepThreads, sweepf_dyn_smem<S>(), st>>>(B);
        else k_sweepf<S, kSweepThreads, false><<<p.nstrips, kSweepThreads, sweepf_dyn_smem<S>(), st>>>(B);
      }
      else k_sweep<S, kSweepThreads><<<p.nstrips, kSweepThreads, 0, st>>>(B);
    }
  } else if (p.ntiles > 0) {
    StepArgs A{p.lats, p.tiles, p.src, p.dst, p.flags, p.wall, p.node_total, p.macro, p.sr_epoch, p.sr_step, p.err};
    const bool macro = p.macro != nullptr;
    switch (p.ty) {
      case 4:
        if (macro) k_step<S, 4, true><<<p.ntiles, 128, 0, st>>>(A);
        else launch_k(k_step<S, 4, false>, p.ntiles, 128, st, dep, A);
        break;
      case 16:
        if (macro) k_step<S, 16, true><<<p.ntiles, 512, 0, st>>>(A);
        else launch_k(k_step<S, 16, false>, p.ntiles, 512, st, dep, A);
        break;
      default:
        if (macro) k_step<S, 8, true><<<p.ntiles, 256, 0, st>>>(A);
        else launch_k(k_step<S, 8, false>, p.ntiles, 256, st, dep, A);
        break;
    }
  }
  rec(3);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t prepare_sweepf() {
  cudaError_t e = cudaFuncSetAttribute(k_sweepf<S, kSweepThreads, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sweepf_dyn_smem<S>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweepf<S, kSweepThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sweepf_dyn_smem<S>());
  return e;
}

cudaError_t prepare_kernels(int prec) {
  switch (prec) {
    case 1: return prepare_sweepf<float>();
    case 2: return prepare_sweepf<__half>();
    case 3: return prepare_sweepf<__nv_bfloat16>();
  }
  return cudaSuccess;
}

cudaError_t launch_step(int prec, const LaunchStep& p, cudaStream_t st) {
  switch (prec) {
    case 0: return launch_all<double>(p, st);
    case 1: return launch_all<float>(p, st);
    case 2: return launch_all<__half>(p, st);
    case 3: return launch_all<__nv_bfloat16>(p, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sr_tick(uint32_t* epoch, cudaStream_t st) {
  k_sr_tick<<<1, 1, 0, st>>>(epoch);
  return cudaGetLastError();
}

cudaError_t launch_to_storage(int prec, const LatDev* lats, int lat, long long nn, const double* in,
                              const uint8_t* flags, void* pool, cudaStream_t st) {
  const long long n = 9 * nn;
  const int blocks = int((n + 255) / 256);
  switch (prec) {
    case 0: k_to_storage<double><<<blocks, 256, 0, st>>>(lats, lat, in, flags, static_cast<double*>(pool)); break;
    case 1: k_to_storage<float><<<blocks, 256, 0, st>>>(lats, lat, in, flags, static_cast<float*>(pool)); break;
    case 2: k_to_storage<__half><<<blocks, 256, 0, st>>>(lats, lat, in, flags, static_cast<__half*>(pool)); break;
    case 3:
      k_to_storage<__nv_bfloat16><<<blocks, 256, 0, st>>>(lats, lat, in, flags, static_cast<__nv_bfloat16*>(pool));
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_from_storage(int prec, const LatDev* lats, int lat, long long nn, const void* pool,
                                const uint8_t* flags, double* out, cudaStream_t st) {
  const long long n = nn;
  const int blocks = int((n + 255) / 256);
  switch (prec) {
    case 0: k_from_storage<double><<<blocks, 256, 0, st>>>(lats, lat, static_cast<const double*>(pool), flags, out); break;
    case 1: k_from_storage<float><<<blocks, 256, 0, st>>>(lats, lat, static_cast<const float*>(pool), flags, out); break;
    case 2: k_from_storage<__half><<<blocks, 256, 0, st>>>(lats, lat, static_cast<const __half*>(pool), flags, out); break;
    case 3:
      k_from_storage<__nv_bfloat16><<<blocks, 256, 0, st>>>(lats, lat, static_cast<const __nv_bfloat16*>(pool), flags,
                                                            out);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbcg
