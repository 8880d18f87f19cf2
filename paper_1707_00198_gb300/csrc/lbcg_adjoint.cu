// Discrete adjoint (reverse mode) of the colour-gradient LBM step, for gradients of an
// objective of the state at step T with respect to the contact angle (per outermost fluid
// node), the interfacial tension sigma and the two viscosities (Sec. II; Eq. 1-18, 28-36).
//
// One reverse step, from the adjoint lambda' of the stored post-streaming state after the
// step to the adjoint lambda of the state before it, has six stages:
//   fwd_local   : forward intermediates recomputed from the stored state: post-Zou-He
//                 populations, colour densities and rho^N (Eq. 12, 16); clears the scatter
//                 targets of this step;
//   fwd_grad    : raw gradient (Eq. 28, Eq. 29 virtual values evaluated on the fly), the
//                 wetting correction (Eq. 30-36) and n;
//   fwd_dn      : grad n (Eq. 28 on n with Eq. 29 virtual values);
//   adj_collide : transpose of streaming + bounce-back (a gather of lambda'), the
//                 hand-derived reverse of Eq. 14, 1-9, 17, 18, 10 and 13 per node, and the
//                 transpose of Eq. 28/29 applied to n (a scatter onto the n stencil);
//   adj_normal  : reverse of n = g/|g|, of Eq. 30-36 (d|g| and d theta), and the transpose of
//                 Eq. 28/29 applied to rho^N (a scatter);
//   adj_rho     : reverse of Eq. 12 and 16, then of the Zou-He columns -> lambda.
// The three forward stages of step j - 1 have the same neighbour dependencies as the three
// reverse stages of step j, so a reverse step runs as three launches, each with one reverse
// stage of step j and, in separate blocks beside it, one forward stage of step j - 1
// (double-buffered intermediates); only the first reversed step of a checkpoint segment needs
// the three forward kernels alone.
// A value that a stencil reads on a solid neighbour is that node's Eq. 29 virtual value, a
// weighted mean of its own fluid neighbours; the transpose scatters straight through that
// mean onto those fluid nodes.  The kernels are templates on their arithmetic R: double, or
// float for the FP32 reverse sweep (whose chains of dependent operations are several times
// shorter in latency than FP64's); scatters accumulate with atomics in R, the per-node
// parameter adjoints in double.  Node arrays are compact [ny][nx] (index y * nx + x).  The
// lattices are small, so blocks are small (64 threads) to spread a lattice over every SM.
#include <vector>

#include "../../include/lbcg.h"
#include "lbcg_internal.h"

namespace lbcg {

namespace {

constexpr int kAdjThreads = 64;

template <typename R>
__device__ __forceinline__ bool is_solid(const AdjDevT<R>& A, int x, int y) {
  return A.sol[y * A.L.nx + x] != 0;
}
// bit a-1 of node j's mask: its neighbour in direction a (1..8) is solid
template <typename R>
__device__ __forceinline__ bool nb_solid(const AdjDevT<R>& A, int j, int a) {
  return (A.nbm[j] >> (a - 1)) & 1u;
}
__device__ __forceinline__ bool mask_bit(unsigned m, int a) { return (m >> (a - 1)) & 1u; }
template <typename R>
__device__ __forceinline__ uint8_t flag_at(const AdjDevT<R>& A, int x, int y) {
  return A.flags[A.L.node_off + (long long)y * A.L.pitch + x];
}
template <typename R>
__device__ __forceinline__ int mapx(const AdjDevT<R>& A, int v) { return wrap_or_clamp(v, A.L.nx, A.L.bcx == BC_PERIODIC); }
template <typename R>
__device__ __forceinline__ int mapy(const AdjDevT<R>& A, int v) { return wrap_or_clamp(v, A.L.ny, A.L.bcy == BC_PERIODIC); }

// ------------------------------------------------------------------ forward intermediates
template <typename R>
__device__ __forceinline__ void fwd_local_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  // The kernels of the reverse sweep run a few warps per SM, so each memory round trip on a
  // thread's path counts: a node's loads are issued together, before its solid test (the
  // slots of a solid node are read but not used).
  const bool solid = is_solid(A, x, y);
  A.lnt_x[i] = A.lnt_y[i] = A.lrnt[i] = R(0.0);
  R fr[9], fb[9], rR, rB;
  if (A.src_fp32) {
    // FP32 forward: its post-Zou-He populations, converted to the reverse arithmetic
    float fr32[9], fb32[9];
    load_node<float>(A.L, static_cast<const float*>(A.src), x, y, fr32, fb32);
    for (int a = 0; a < 9; ++a) {
      fr[a] = R(fr32[a]);
      fb[a] = R(fb32[a]);
    }
  } else {
    double fr64[9], fb64[9];
    load_node<double>(A.L, static_cast<const double*>(A.src), x, y, fr64, fb64);
    for (int a = 0; a < 9; ++a) {
      fr[a] = R(fr64[a]);
      fb[a] = R(fb64[a]);
    }
  }
  if (solid) {
    for (int a = 0; a < 9; ++a) A.fr[a * N + i] = A.fb[a * N + i] = R(0.0);
    A.rr[i] = A.rb[i] = A.rn[i] = R(0.0);
    return;
  }
  for (int a = 0; a < 9; ++a) {
    A.fr[a * N + i] = fr[a];
    A.fb[a * N + i] = fb[a];
  }
  A.rn[i] = colour_indicator(fr, fb, rR, rB);
  A.rr[i] = rR;
  A.rb[i] = rB;
}

// Sum of the D2Q9 weights toward the fluid neighbours of a solid node (Eq. 29 denominator)
template <typename R>
__device__ R weight_sum(const AdjDevT<R>& A, int x, int y) {
  const unsigned m = A.nbm[y * A.L.nx + x];
  R den = R(0.0);
  for (int b = 1; b < 9; ++b)
    if (!((m >> (b - 1)) & 1u)) den = radd(den, wgt<R>(b));
  return den;
}

// Value of field v that a stencil reads at (x, y): v itself on a fluid node, the Eq. 29
// virtual value (the same sums in the same order as the step kernels) on a solid node
// (solid: whether (x, y) is a solid node, known from the reading node's neighbour mask)
template <typename R>
__device__ R read_field(const AdjDevT<R>& A, const R* v, int x, int y, bool solid) {
  if (!solid) return v[y * A.L.nx + x];
  const unsigned m = A.nbm[y * A.L.nx + x];
  R num = R(0.0), den = R(0.0);
  for (int b = 1; b < 9; ++b) {
    if (!((m >> (b - 1)) & 1u)) {
      const int x2 = mapx(A, x + ex(b)), y2 = mapy(A, y + ey(b));
      num = radd(num, rmul(wgt<R>(b), v[y2 * A.L.nx + x2]));
      den = radd(den, wgt<R>(b));
    }
  }
  return den > R(0.0) ? rdiv(num, den) : R(0.0);
}

// Transpose of read_field for one or two fields: add `val` to the adjoint of what was read
template <typename R>
__device__ void scatter_field(const AdjDevT<R>& A, R* acc0, R* acc1, int x, int y, bool solid, R v0, R v1) {
  if (!solid) {
    const int j = y * A.L.nx + x;
    atomicAdd(&acc0[j], v0);
    if (acc1) atomicAdd(&acc1[j], v1);
    return;
  }
  const R den = weight_sum(A, x, y);
  if (!(den > R(0.0))) return;
  const R r = R(1.0) / den;
  const unsigned m = A.nbm[y * A.L.nx + x];
  for (int b = 1; b < 9; ++b) {
    if ((m >> (b - 1)) & 1u) continue;
    const int x2 = mapx(A, x + ex(b)), y2 = mapy(A, y + ey(b));
    const int j = y2 * A.L.nx + x2;
    const R c = wgt<R>(b) * r;
    atomicAdd(&acc0[j], c * v0);
    if (acc1) atomicAdd(&acc1[j], c * v1);
  }
}

template <typename R>
__device__ __forceinline__ void fwd_grad_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  const uint8_t f = flag_at(A, x, y);
  const unsigned msk = A.nbm[i];
  const R nsx = A.nsx[i], nsy = A.nsy[i];
  const R c = A.cos_t[i], s = A.sin_t[i];
  A.pick[i] = 0;
  if (f & F_SOLID) {
    A.grx[i] = A.gry[i] = A.gcx[i] = A.gcy[i] = R(0.0);
    A.nxv[i] = A.nyv[i] = R(0.0);
    return;
  }
  R gx = R(0.0), gy = R(0.0);
  for (int a = 1; a < 9; ++a) {
    const R t = rmul(wgt<R>(a), read_field(A, A.rn, mapx(A, x + ex(a)), mapy(A, y + ey(a)), mask_bit(msk, a)));
    if (ex(a) == 1) gx = radd(gx, t);
    if (ex(a) == -1) gx = radd(gx, -t);
    if (ey(a) == 1) gy = radd(gy, t);
    if (ey(a) == -1) gy = radd(gy, -t);
  }
  gx = rdiv(gx, R(1.0 / 3.0));
  gy = rdiv(gy, R(1.0 / 3.0));
  A.grx[i] = gx;
  A.gry[i] = gy;
  R cgx = gx, cgy = gy;
  const R eps = R(A.L.grad_eps);
  const R mag = rsqrt_(radd(rmul(gx, gx), rmul(gy, gy)));
  if ((f & F_OFB) && mag > eps) {
    const R esx = rdiv(gx, mag), esy = rdiv(gy, mag);
    const R f1x = rsub(rmul(nsx, c), rmul(nsy, s)), f1y = radd(rmul(nsx, s), rmul(nsy, c));
    const R f2x = radd(rmul(nsx, c), rmul(nsy, s)), f2y = radd(rmul(-nsx, s), rmul(nsy, c));
    const R a1 = rsub(f1x, esx), b1 = rsub(f1y, esy), a2 = rsub(f2x, esx), b2 = rsub(f2y, esy);
    const R d1 = rsqrt_(radd(rmul(a1, a1), rmul(b1, b1)));
    const R d2 = rsqrt_(radd(rmul(a2, a2), rmul(b2, b2)));
    const bool one = d1 <= d2;
    A.pick[i] = one ? 1 : 2;
    cgx = rmul(mag, one ? f1x : f2x);
    cgy = rmul(mag, one ? f1y : f2y);
  }
  A.gcx[i] = cgx;
  A.gcy[i] = cgy;
  const R m2 = sqrt(cgx * cgx + cgy * cgy);
  A.nxv[i] = m2 > eps ? cgx / m2 : R(0.0);
  A.nyv[i] = m2 > eps ? cgy / m2 : R(0.0);
}

template <typename R>
__device__ __forceinline__ void fwd_dn_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  R d[4] = {0, 0, 0, 0};
  const bool solid = is_solid(A, x, y);
  const unsigned msk = A.nbm[i];
  if (!solid) {
    for (int a = 1; a < 9; ++a) {
      const int x2 = mapx(A, x + ex(a)), y2 = mapy(A, y + ey(a));
      const bool sn = mask_bit(msk, a);
      const R tx = wgt<R>(a) * read_field(A, A.nxv, x2, y2, sn);
      const R ty = wgt<R>(a) * read_field(A, A.nyv, x2, y2, sn);
      d[0] += ex(a) * tx;
      d[1] += ey(a) * tx;
      d[2] += ex(a) * ty;
      d[3] += ey(a) * ty;
    }
  }
  for (int q = 0; q < 4; ++q) A.dn[q * N + i] = R(3.0) * d[q];
}

// ------------------------------------------------------------------ reverse kernels
// Transpose of the push (Eq. 15, half-way bounce-back, open edges) and the reverse of the
// node-local part of the step.
template <typename R>
__device__ __forceinline__ void adj_collide_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  const LatDev& L = A.L;
  // the node's masks, forward intermediates and parameter adjoints so far, all in flight
  // together before the solid test
  const bool solid = is_solid(A, x, y);
  const unsigned msk = A.nbm[i];
  R fr[9], fb[9], f[9];
  for (int a = 0; a < 9; ++a) {
    fr[a] = A.fr[a * N + i];
    fb[a] = A.fb[a * N + i];
    f[a] = fr[a] + fb[a];
  }
  const R rhoR = A.rr[i], rhoB = A.rb[i], rn = A.rn[i];
  const R nxo = A.nxv[i], nyo = A.nyv[i];
  const R gx = A.gcx[i], gy = A.gcy[i];
  const R dxx = A.dn[i], dxy = A.dn[N + i], dyx = A.dn[2 * N + i], dyy = A.dn[3 * N + i];
  const double p_hR0 = A.p_hR[i], p_hB0 = A.p_hB[i], p_sigma0 = A.p_sigma[i];
  if (solid) {
    for (int a = 0; a < 9; ++a) A.lf_r[a * N + i] = A.lf_b[a * N + i] = R(0.0);
    A.ln_x[i] = A.ln_y[i] = A.lg_x[i] = A.lg_y[i] = A.lrn[i] = R(0.0);
    return;
  }
  const bool px = L.bcx == BC_PERIODIC, py = L.bcy == BC_PERIODIC;
  // adjoint of the post-collision, recoloured values (oR_a, oB_a) leaving this node
  R mR[9], mB[9];
  for (int a = 0; a < 9; ++a) {
    mR[a] = mB[a] = R(0.0);
    int j = i, slot = a;
    if (a != 0) {
      const int xr = x + ex(a), yr = y + ey(a);
      if ((!px && (xr < 0 || xr >= L.nx)) || (!py && (yr < 0 || yr >= L.ny))) continue;
      const int xd = mapx(A, xr), yd = mapy(A, yr);
      if (mask_bit(msk, a)) slot = opp(a);
      else j = yd * L.nx + xd;
    }
    mR[a] = A.lam_next[(2 * slot) * N + j];
    mB[a] = A.lam_next[(2 * slot + 1) * N + j];
  }
  // forward recomputation of the node-local quantities
  const R rho = rhoR + rhoB, ir = R(1.0) / rho;
  const R kappa = -nxo * nxo * dyy - nyo * nyo * dxx + nxo * nyo * (dxy + dyx);
  const R hsk = R(0.5) * R(L.sigma) * kappa;
  const R Fx = hsk * gx, Fy = hsk * gy;
  const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const R ux = (jx + R(0.5) * Fx) * ir, uy = (jy + R(0.5) * Fy) * ir;
  const R inv_nu = (1 + rn) * R(L.h_inv_nuR) + (1 - rn) * R(L.h_inv_nuB);
  const R den_sv = R(3.0) + R(0.5) * inv_nu;
  const R sv = inv_nu / den_sv;
  const R se = L.s_e, seps = L.s_eps, sq = L.s_q, beta = L.beta;
  const R s14 = f[1] + f[2] + f[3] + f[4], s58 = f[5] + f[6] + f[7] + f[8];
  const R me = -4 * f[0] - s14 + 2 * s58;
  const R meps = 4 * f[0] - 2 * s14 + s58;
  const R qx = -2 * (f[1] - f[3]) + (f[5] - f[6] - f[7] + f[8]);
  const R qy = -2 * (f[2] - f[4]) + (f[5] + f[6] - f[7] - f[8]);
  const R pxx = f[1] - f[2] + f[3] - f[4];
  const R pxy = f[5] - f[6] + f[7] - f[8];
  const R u2 = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
  const R De = se * (me - rho * (-2 + 3 * u2)) - (1 - R(0.5) * se) * (6 * uF);
  const R Deps = seps * (meps - rho * (1 - 3 * u2)) + (1 - R(0.5) * seps) * (6 * uF);
  const R Dqx = sq * (qx + rho * ux) + (1 - R(0.5) * sq) * Fx;
  const R Dqy = sq * (qy + rho * uy) + (1 - R(0.5) * sq) * Fy;
  const R Axx = pxx - rho * (ux * ux - uy * uy), Bxx = 2 * (ux * Fx - uy * Fy);
  const R Dxx = sv * Axx - (1 - R(0.5) * sv) * Bxx;
  const R Axy = pxy - rho * ux * uy, Bxy = ux * Fy + uy * Fx;
  const R Dxy = sv * Axy - (1 - R(0.5) * sv) * Bxy;
  constexpr R k36 = R(1.0) / 36, k12 = R(1.0) / 12, k6 = R(1.0) / 6;
  const R ae = De * k36, aeps = Deps * k36, ajx = -Fx * k6, ajy = -Fy * k6;
  const R aqx = Dqx * k12, aqy = Dqy * k12, axx = Dxx * R(0.25), axy = Dxy * R(0.25);
  R fp[9];
  fp[0] = f[0] - (-4 * ae + 4 * aeps);
  const R c14 = -ae - 2 * aeps;
  fp[1] = f[1] - (c14 + ajx - 2 * aqx + axx);
  fp[2] = f[2] - (c14 + ajy - 2 * aqy - axx);
  fp[3] = f[3] - (c14 - ajx + 2 * aqx + axx);
  fp[4] = f[4] - (c14 - ajy + 2 * aqy - axx);
  const R c58 = 2 * ae + aeps;
  fp[5] = f[5] - (c58 + ajx + aqx + ajy + aqy + axy);
  fp[6] = f[6] - (c58 - ajx - aqx + ajy + aqy - axy);
  fp[7] = f[7] - (c58 - ajx - aqx - ajy - aqy + axy);
  fp[8] = f[8] - (c58 + ajx + aqx - ajy - aqy - axy);
  const R cR = rhoR * ir;
  const R pc = beta * rhoR * rhoB * ir;
  // ---- reverse of Eq. 14: oR = cR fp + pc w (e.n), oB = fp - oR
  R lfp[9], lcR = 0, lpc = 0, lnx = 0, lny = 0;
  for (int a = 0; a < 9; ++a) {
    const R mu = mR[a] - mB[a];        // adjoint of oR through both outputs
    const R en = ex(a) * nxo + ey(a) * nyo;
    lfp[a] = mB[a] + mu * cR;
    lcR += mu * fp[a];
    lpc += mu * wgt<R>(a) * en;
    lnx += mu * pc * wgt<R>(a) * ex(a);
    lny += mu * pc * wgt<R>(a) * ey(a);
  }
  R lrhoR = (lcR + lpc * beta * rhoB) * ir;
  R lrhoB = lpc * beta * rhoR * ir;
  R lrho = -(lcR * rhoR + lpc * beta * rhoR * rhoB) * ir * ir;
  // ---- reverse of fp = f - M^T diag(...) Delta
  R lf[9];
  for (int a = 0; a < 9; ++a) lf[a] = lfp[a];
  // adjoints of the a_k: l_ak = -sum_a M[k][a] lfp[a]
  const R lae = -(-4 * lfp[0] - lfp[1] - lfp[2] - lfp[3] - lfp[4] + 2 * (lfp[5] + lfp[6] + lfp[7] + lfp[8]));
  const R laeps = -(4 * lfp[0] - 2 * (lfp[1] + lfp[2] + lfp[3] + lfp[4]) + lfp[5] + lfp[6] + lfp[7] + lfp[8]);
  const R lajx = -(lfp[1] - lfp[3] + lfp[5] - lfp[6] - lfp[7] + lfp[8]);
  const R lajy = -(lfp[2] - lfp[4] + lfp[5] + lfp[6] - lfp[7] - lfp[8]);
  const R laqx = -(-2 * lfp[1] + 2 * lfp[3] + lfp[5] - lfp[6] - lfp[7] + lfp[8]);
  const R laqy = -(-2 * lfp[2] + 2 * lfp[4] + lfp[5] + lfp[6] - lfp[7] - lfp[8]);
  const R laxx = -(lfp[1] - lfp[2] + lfp[3] - lfp[4]);
  const R laxy = -(lfp[5] - lfp[6] + lfp[7] - lfp[8]);
  const R lDe = lae * k36, lDeps = laeps * k36, lDqx = laqx * k12, lDqy = laqy * k12;
  const R lDxx = laxx * R(0.25), lDxy = laxy * R(0.25);
  R lFx = -lajx * k6, lFy = -lajy * k6;
  R lux = 0, luy = 0, lu2 = 0, luF = 0, lsv = 0;
  R lme = 0, lmeps = 0, lqx = 0, lqy = 0, lpxx = 0, lpxy = 0;
  // De
  lme += se * lDe;
  lrho += -se * (-2 + 3 * u2) * lDe;
  lu2 += -3 * se * rho * lDe;
  luF += -6 * (1 - R(0.5) * se) * lDe;
  // Deps
  lmeps += seps * lDeps;
  lrho += -seps * (1 - 3 * u2) * lDeps;
  lu2 += 3 * seps * rho * lDeps;
  luF += 6 * (1 - R(0.5) * seps) * lDeps;
  // Dqx, Dqy
  lqx += sq * lDqx;
  lrho += sq * ux * lDqx;
  lux += sq * rho * lDqx;
  lFx += (1 - R(0.5) * sq) * lDqx;
  lqy += sq * lDqy;
  lrho += sq * uy * lDqy;
  luy += sq * rho * lDqy;
  lFy += (1 - R(0.5) * sq) * lDqy;
  // Dxx = sv Axx - (1 - sv/2) Bxx
  lsv += (Axx + R(0.5) * Bxx) * lDxx;
  lpxx += sv * lDxx;
  lrho += -sv * (ux * ux - uy * uy) * lDxx;
  lux += -2 * sv * rho * ux * lDxx - (1 - R(0.5) * sv) * 2 * Fx * lDxx;
  luy += 2 * sv * rho * uy * lDxx + (1 - R(0.5) * sv) * 2 * Fy * lDxx;
  lFx += -(1 - R(0.5) * sv) * 2 * ux * lDxx;
  lFy += (1 - R(0.5) * sv) * 2 * uy * lDxx;
  // Dxy = sv Axy - (1 - sv/2) Bxy
  lsv += (Axy + R(0.5) * Bxy) * lDxy;
  lpxy += sv * lDxy;
  lrho += -sv * ux * uy * lDxy;
  lux += -sv * rho * uy * lDxy - (1 - R(0.5) * sv) * Fy * lDxy;
  luy += -sv * rho * ux * lDxy - (1 - R(0.5) * sv) * Fx * lDxy;
  lFy += -(1 - R(0.5) * sv) * ux * lDxy;
  lFx += -(1 - R(0.5) * sv) * uy * lDxy;
  // u2, uF
  lux += 2 * ux * lu2 + Fx * luF;
  luy += 2 * uy * lu2 + Fy * luF;
  lFx += ux * luF;
  lFy += uy * luF;
  // moments -> f
  for (int a = 0; a < 9; ++a) {
    const R r1 = (a == 0) ? -4 : (a <= 4 ? -1 : 2);
    const R r2 = (a == 0) ? 4 : (a <= 4 ? -2 : 1);
    const R rqx = (a == 1) ? -2 : (a == 3) ? 2 : (a >= 5 ? (R)ex(a) : R(0.0));
    const R rqy = (a == 2) ? -2 : (a == 4) ? 2 : (a >= 5 ? (R)ey(a) : R(0.0));
    const R rxx = (a == 1 || a == 3) ? 1 : (a == 2 || a == 4) ? -1 : 0;
    const R rxy = (a >= 5) ? (R)(ex(a) * ey(a)) : R(0.0);
    lf[a] += r1 * lme + r2 * lmeps + rqx * lqx + rqy * lqy + rxx * lpxx + rxy * lpxy;
  }
  // sv = inv_nu / (3 + inv_nu / 2); inv_nu = (1 + rn) hR + (1 - rn) hB
  const R linv = lsv * R(3.0) / (den_sv * den_sv);
  R lrn_loc = (R(L.h_inv_nuR) - R(L.h_inv_nuB)) * linv;
  A.p_hR[i] = p_hR0 + (1 + rn) * linv;
  A.p_hB[i] = p_hB0 + (1 - rn) * linv;
  // u = (j + F/2) / rho
  const R ljx = lux * ir, ljy = luy * ir;
  lFx += R(0.5) * ljx;
  lFy += R(0.5) * ljy;
  lrho += -(ux * lux + uy * luy) * ir;
  for (int a = 0; a < 9; ++a) lf[a] += ex(a) * ljx + ey(a) * ljy;
  // F = (sigma kappa / 2) g
  const R lhsk = gx * lFx + gy * lFy;
  const R lgx = hsk * lFx, lgy = hsk * lFy;
  A.p_sigma[i] = p_sigma0 + R(0.5) * kappa * lhsk;
  const R lk = R(0.5) * R(L.sigma) * lhsk;
  // kappa = -nx^2 dyy - ny^2 dxx + nx ny (dxy + dyx)
  lnx += (-2 * nxo * dyy + nyo * (dxy + dyx)) * lk;
  lny += (-2 * nyo * dxx + nxo * (dxy + dyx)) * lk;
  // transpose of grad n = 3 sum_a w_a e_a n~(x + e_a) (Eq. 28 on the Eq. 29-filled n)
  if (lk != R(0.0)) {
    const R lxx = -nyo * nyo * lk;   // adjoint of d_x n_x
    const R lxy = nxo * nyo * lk;    // d_y n_x
    const R lyx = nxo * nyo * lk;    // d_x n_y
    const R lyy = -nxo * nxo * lk;   // d_y n_y
    for (int a = 1; a < 9; ++a) {
      const R w = R(3.0) * wgt<R>(a);
      scatter_field(A, A.lnt_x, A.lnt_y, mapx(A, x + ex(a)), mapy(A, y + ey(a)), mask_bit(msk, a),
                    w * (ex(a) * lxx + ey(a) * lxy),
                    w * (ex(a) * lyx + ey(a) * lyy));
    }
  }
  // rho = rhoR + rhoB; f = fr + fb
  lrhoR += lrho;
  lrhoB += lrho;
  for (int a = 0; a < 9; ++a) {
    A.lf_r[a * N + i] = lf[a] + lrhoR;
    A.lf_b[a * N + i] = lf[a] + lrhoB;
  }
  A.lrn[i] = lrn_loc;
  A.ln_x[i] = lnx;
  A.ln_y[i] = lny;
  A.lg_x[i] = lgx;
  A.lg_y[i] = lgy;
}

// Reverse of n = g_c / |g_c| (zero below the guard), of Eq. 30-36 (g_c = |g_r| n_f(theta) on
// Omega_Fb, g_c = g_r elsewhere), and the transpose of the raw gradient (Eq. 28 on the
// Eq. 29-filled rho^N), scattered onto rho^N.
template <typename R>
__device__ __forceinline__ void adj_normal_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  // everything the node reads, in flight together before the solid test
  const bool solid = is_solid(A, x, y);
  const unsigned msk = A.nbm[i];
  const R lnx = A.ln_x[i] + A.lnt_x[i], lny = A.ln_y[i] + A.lnt_y[i];
  R lgx = A.lg_x[i], lgy = A.lg_y[i];
  const R gcx = A.gcx[i], gcy = A.gcy[i];
  const int pick = A.pick[i];
  const R grx = A.grx[i], gry = A.gry[i];
  const R nsx = A.nsx[i], nsy = A.nsy[i];
  const R c = A.cos_t[i], s = A.sin_t[i];
  const double p_theta0 = A.p_theta[i];
  if (solid) return;
  {
    const R gx = gcx, gy = gcy;
    const R m = sqrt(gx * gx + gy * gy);
    if (m > A.n_eps) {   // below it n is frozen in the reverse sweep (see AdjDev::n_eps)
      const R im = R(1.0) / m, nx = gx * im, ny = gy * im;
      const R dot = nx * lnx + ny * lny;
      lgx += (lnx - nx * dot) * im;
      lgy += (lny - ny * dot) * im;
    }
  }
  R lrx = lgx, lry = lgy;
  if (pick != 0) {
    const R gx = grx, gy = gry;
    const R m = sqrt(gx * gx + gy * gy);
    R nfx, nfy, dfx, dfy;
    if (pick == 1) {   // rotation by +theta; d n_f / d theta = (-n_fy, n_fx)
      nfx = nsx * c - nsy * s;
      nfy = nsx * s + nsy * c;
      dfx = -nfy;
      dfy = nfx;
    } else {           // rotation by -theta; d n_f / d theta = (n_fy, -n_fx)
      nfx = nsx * c + nsy * s;
      nfy = -nsx * s + nsy * c;
      dfx = nfy;
      dfy = -nfx;
    }
    const R proj = (nfx * lgx + nfy * lgy) / m;
    lrx = gx * proj;
    lry = gy * proj;
    A.p_theta[i] = p_theta0 + m * (dfx * lgx + dfy * lgy);
  }
  if (lrx != R(0.0) || lry != R(0.0))
    for (int a = 1; a < 9; ++a)
      scatter_field(A, A.lrnt, static_cast<R*>(nullptr), mapx(A, x + ex(a)), mapy(A, y + ey(a)), mask_bit(msk, a),
                    R(3.0) * wgt<R>(a) * (ex(a) * lrx + ey(a) * lry), R(0.0));
}

// reverse of rho^N = (rhoR - rhoB)/(rhoR + rhoB) and of the Zou-He columns
template <typename R>
__device__ __forceinline__ void adj_rho_body(const AdjDevT<R>& A, const int i) {
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  // the node's inputs, in flight together before the solid test
  const bool solid = is_solid(A, x, y);
  const R lrn = A.lrn[i] + A.lrnt[i];
  const R rR = A.rr[i], rB = A.rb[i];
  R lr[9], lb[9];
  for (int a = 0; a < 9; ++a) {
    lr[a] = A.lf_r[a * N + i];
    lb[a] = A.lf_b[a * N + i];
  }
  if (solid) {
    for (int a = 0; a < 18; ++a) A.lam[a * N + i] = R(0.0);
    return;
  }
  const R rho = rR + rB;
  const R ir2 = R(1.0) / (rho * rho);
  const R cR = 2 * rB * ir2 * lrn, cB = -2 * rR * ir2 * lrn;
  for (int a = 0; a < 9; ++a) {
    lr[a] += cR;
    lb[a] += cB;
  }
  const LatDev& L = A.L;
  R sr[9], sb[9];   // adjoint of the stored values
  if (L.bcx == BC_INOUT && x == 0) {
    // inlet: fr = f (f1, f5, f8 from Zou-He of the known totals), fb = 0
    const R u = inlet_u<R>(L, y);
    const R ck[9] = {1, 0, 1, 2, 1, 0, 2, 2, 0};
    R lt[9];
    for (int a = 0; a < 9; ++a) lt[a] = R(0.0);
    const int known[6] = {0, 2, 3, 4, 6, 7};
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      const R drho = ck[k] / (1 - u);
      R v = lr[k];
      v += lr[1] * ((k == 3 ? R(1.0) : R(0.0)) + R(2.0 / 3.0) * u * drho);
      v += lr[5] * ((k == 7 ? R(1.0) : R(0.0)) - (k == 2 ? R(0.5) : R(0.0)) + (k == 4 ? R(0.5) : R(0.0)) + u / 6 * drho);
      v += lr[8] * ((k == 6 ? R(1.0) : R(0.0)) + (k == 2 ? R(0.5) : R(0.0)) - (k == 4 ? R(0.5) : R(0.0)) + u / 6 * drho);
      lt[k] = v;
    }
    for (int a = 0; a < 9; ++a) sr[a] = sb[a] = lt[a];
  } else if (L.bcx == BC_INOUT && x == L.nx - 1) {
    // outlet: known 0,1,2,4,5,8 pass through; f3, f6, f7 from Zou-He, split by frac = kR/kT
    const R* FR = A.fr;
    const R* FB = A.fb;
    const int known[6] = {0, 1, 2, 4, 5, 8};
    R kR = 0, kT = 0;
    for (int q = 0; q < 6; ++q) {
      kR += FR[known[q] * N + i];
      kT += FR[known[q] * N + i] + FB[known[q] * N + i];
    }
    const R frac = kT != 0 ? kR / kT : R(0.0);
    R lt[9], lfrac = 0;
    for (int a = 0; a < 9; ++a) lt[a] = R(0.0);
    const int unk[3] = {3, 6, 7};
    for (int q = 0; q < 3; ++q) {
      const int uu = unk[q];
      const R fu = FR[uu * N + i] + FB[uu * N + i];
      lt[uu] = frac * lr[uu] + (1 - frac) * lb[uu];   // adjoint of the total f_u
      lfrac += fu * (lr[uu] - lb[uu]);
    }
    // f3 = f1 + 2/3 r - 2/3 S, f7 = f5 + (f2 - f4)/2 + r/6 - S/6, f6 = f8 - (f2 - f4)/2 + r/6 - S/6,
    // S = f0 + f2 + f4 + 2 (f1 + f5 + f8)
    const R cs[9] = {1, 2, 1, 0, 1, 2, 0, 0, 2};
    R ltk[9];
    for (int a = 0; a < 9; ++a) ltk[a] = R(0.0);
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      ltk[k] += lt[3] * ((k == 1 ? R(1.0) : R(0.0)) - R(2.0 / 3.0) * cs[k]);
      ltk[k] += lt[7] * ((k == 5 ? R(1.0) : R(0.0)) + (k == 2 ? R(0.5) : R(0.0)) - (k == 4 ? R(0.5) : R(0.0)) - cs[k] / 6);
      ltk[k] += lt[6] * ((k == 8 ? R(1.0) : R(0.0)) - (k == 2 ? R(0.5) : R(0.0)) + (k == 4 ? R(0.5) : R(0.0)) - cs[k] / 6);
    }
    for (int a = 0; a < 9; ++a) sr[a] = sb[a] = R(0.0);
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      const R dfr = kT != 0 ? (kT - kR) / (kT * kT) : R(0.0);   // d frac / d s_R
      const R dfb = kT != 0 ? -kR / (kT * kT) : R(0.0);         // d frac / d s_B
      sr[k] = lr[k] + ltk[k] + lfrac * dfr;
      sb[k] = lb[k] + ltk[k] + lfrac * dfb;
    }
  } else {
    for (int a = 0; a < 9; ++a) {
      sr[a] = lr[a];
      sb[a] = lb[a];
    }
  }
  for (int a = 0; a < 9; ++a) {
    A.lam[(2 * a) * N + i] = sr[a];
    A.lam[(2 * a + 1) * N + i] = sb[a];
  }
}

inline int nblk(int n) { return (n + kAdjThreads - 1) / kAdjThreads; }

// Programmatic dependent launch.  The kernels of a reverse sweep are short, latency-bound
// grids, each depending on the one before it.  A kernel launched by launch_dep may be scheduled
// once every block of the kernel before it has run its dep_trigger (placed after all of a
// block's stores) or exited; its threads wait in dep_wait (the hardware's wait for the full
// completion and memory flush of that kernel) before they read anything.  So the next grid's
// launch overlaps the tail of the last one.  For a kernel launched the ordinary way both
// instructions do nothing.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... P, typename... Q>
cudaError_t launch_dep(void (*k)(P...), int grid, cudaStream_t st, Q... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kAdjThreads);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Forward intermediates of one state (the prologue of a segment's reverse sweep).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_fwd_local(AdjDevT<R> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.N) fwd_local_body(A, i);
}
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_fwd_grad(AdjDevT<R> A) {
  dep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.N) fwd_grad_body(A, i);
  dep_trigger();
}
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_fwd_dn(AdjDevT<R> A) {
  dep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.N) fwd_dn_body(A, i);
  dep_trigger();
}

// The reverse of step j (A) in three stages, each paired in one launch with the stage of the
// forward intermediates of the state before it (B, step j - 1) that has the same dependency on
// the neighbours: (adj_collide, fwd_local), (adj_normal, fwd_grad), (adj_rho, fwd_dn).  A and B
// share the reverse arrays and parameter adjoints but have their own forward intermediates
// and scatter targets, so the two halves of a launch touch disjoint data and run in separate
// blocks side by side: blocks [0, nrev) take the reverse stage, the rest (none for the first
// step of a segment, whose previous state is not recomputed yet) the forward stage.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_rev_collide(AdjDevT<R> A, AdjDevT<R> B, int nrev) {
  const bool rev = int(blockIdx.x) < nrev;
  const int i = (rev ? blockIdx.x : blockIdx.x - nrev) * blockDim.x + threadIdx.x;
  dep_wait();
  if (i < A.N) {
    if (rev) adj_collide_body(A, i);
    else fwd_local_body(B, i);
  }
  dep_trigger();
}
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_rev_normal(AdjDevT<R> A, AdjDevT<R> B, int nrev) {
  const bool rev = int(blockIdx.x) < nrev;
  const int i = (rev ? blockIdx.x : blockIdx.x - nrev) * blockDim.x + threadIdx.x;
  dep_wait();
  if (i < A.N) {
    if (rev) adj_normal_body(A, i);
    else fwd_grad_body(B, i);
  }
  dep_trigger();
}
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_rev_rho(AdjDevT<R> A, AdjDevT<R> B, int nrev) {
  const bool rev = int(blockIdx.x) < nrev;
  const int i = (rev ? blockIdx.x : blockIdx.x - nrev) * blockDim.x + threadIdx.x;
  dep_wait();
  if (i < A.N) {
    if (rev) adj_rho_body(A, i);
    else fwd_dn_body(B, i);
  }
  dep_trigger();
}
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_rho(AdjDevT<R> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.N) adj_rho_body(A, i);
}

// Seed for an objective J = sum_x c(x) rho^N(x) of the stored state: lam = dJ/d(state).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_seed_weighted(AdjDevT<R> A, const R* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int N = A.N;
  for (int a = 0; a < 9; ++a) A.lf_r[a * N + i] = A.lf_b[a * N + i] = R(0.0);
  const int x = i % A.L.nx, y = i / A.L.nx;
  A.lrn[i] = is_solid(A, x, y) ? R(0.0) : c[i];
}

// Seed for J = sum over fluid nodes of rho_R = sum_a f_a,R (the red mass) of the stored state.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_seed_red_mass(AdjDevT<R> A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int N = A.N;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const R one = is_solid(A, x, y) ? R(0.0) : R(1.0);
  for (int a = 0; a < 9; ++a) {
    A.lf_r[a * N + i] = one;
    A.lf_b[a * N + i] = R(0.0);
  }
  A.lrn[i] = R(0.0);
}

}  // namespace

// Forward intermediates of the state A.src (three kernels: the prologue of a segment).
template <typename R>
cudaError_t adjoint_forward(const AdjDevT<R>& A, cudaStream_t st) {
  const int b = nblk(A.N);
  k_fwd_local<R><<<b, kAdjThreads, 0, st>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_dep(k_fwd_grad<R>, b, st, A);
  if (e == cudaSuccess) e = launch_dep(k_fwd_dn<R>, b, st, A);
  return e;
}

// One reverse step: lam <- (d step / d state)^T lam_next, parameter adjoints accumulated,
// from the forward intermediates of A's state (computed by the previous call, or by
// adjoint_forward); with B non-null the same three kernels compute B's intermediates.
template <typename R>
cudaError_t adjoint_step(const AdjDevT<R>& A, const AdjDevT<R>* B, cudaStream_t st) {
  const int b = nblk(A.N);
  const AdjDevT<R>& Bv = B ? *B : A;
  const int g = B ? 2 * b : b;
  cudaError_t e = launch_dep(k_rev_collide<R>, g, st, A, Bv, b);
  if (e == cudaSuccess) e = launch_dep(k_rev_normal<R>, g, st, A, Bv, b);
  if (e == cudaSuccess) e = launch_dep(k_rev_rho<R>, g, st, A, Bv, b);
  return e;
}

template <typename R>
cudaError_t adjoint_seed(const AdjDevT<R>& A, const R* c, bool red_mass, cudaStream_t st) {
  const int b = nblk(A.N);
  k_fwd_local<R><<<b, kAdjThreads, 0, st>>>(A);   // also clears lrnt
  if (red_mass) k_seed_red_mass<R><<<b, kAdjThreads, 0, st>>>(A);
  else k_seed_weighted<R><<<b, kAdjThreads, 0, st>>>(A, c);
  k_adj_rho<R><<<b, kAdjThreads, 0, st>>>(A);
  return cudaGetLastError();
}

template cudaError_t adjoint_forward<double>(const AdjDevT<double>&, cudaStream_t);
template cudaError_t adjoint_forward<float>(const AdjDevT<float>&, cudaStream_t);
template cudaError_t adjoint_step<double>(const AdjDevT<double>&, const AdjDevT<double>*, cudaStream_t);
template cudaError_t adjoint_step<float>(const AdjDevT<float>&, const AdjDevT<float>*, cudaStream_t);
template cudaError_t adjoint_seed<double>(const AdjDevT<double>&, const double*, bool, cudaStream_t);
template cudaError_t adjoint_seed<float>(const AdjDevT<float>&, const float*, bool, cudaStream_t);

}  // namespace lbcg
