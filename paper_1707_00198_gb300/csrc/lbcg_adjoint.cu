// Discrete adjoint (reverse mode) of the colour-gradient LBM step, for gradients of an
// objective of the state at step T with respect to the contact angle (per outermost fluid
// node), the interfacial tension sigma and the two viscosities (Sec. II; Eq. 1-18, 28-36).
//
// One reverse step, from the adjoint lambda' of the stored post-streaming state after the
// step to the adjoint lambda of the state before it, runs these kernels in order:
//   forward intermediates, recomputed from the stored state (fwd_*): post-Zou-He
//     populations, colour densities and rho^N, Eq. 29 virtual rho^N, raw and corrected
//     gradient (Eq. 28, 30-36), n, Eq. 29 virtual n, grad n;
//   adj_collide   : transpose of streaming + bounce-back (a gather of lambda'), then the
//                   hand-derived reverse of Eq. 17, 18, 5, 1-9, 13, 10 and 14 per node;
//   adj_dn        : transpose of Eq. 28 applied to n (a scatter onto the n stencil);
//   adj_vn        : transpose of Eq. 29 for n on outermost solid nodes;
//   adj_n         : reverse of n = g / |g| (zero below the guard);
//   adj_wet       : reverse of Eq. 30-36 on outermost fluid nodes (d|g| and d theta);
//   adj_grad      : transpose of Eq. 28 applied to rho^N;
//   adj_vrn       : transpose of Eq. 29 for rho^N;
//   adj_rho       : reverse of Eq. 12 and 16, then of the Zou-He columns -> lambda.
// Scatters accumulate with FP64 atomics.  Everything is FP64; node arrays are compact
// [ny][nx] (index y * nx + x).
#include <vector>

#include "../../include/lbcg.h"
#include "lbcg_internal.h"

namespace lbcg {

namespace {

__device__ __forceinline__ bool is_solid(const AdjDev& A, int x, int y) {
  return (A.flags[A.L.node_off + (long long)y * A.L.pitch + x] & F_SOLID) != 0;
}
__device__ __forceinline__ uint8_t flag_at(const AdjDev& A, int x, int y) {
  return A.flags[A.L.node_off + (long long)y * A.L.pitch + x];
}
__device__ __forceinline__ int mapx(const AdjDev& A, int v) { return wrap_or_clamp(v, A.L.nx, A.L.bcx == BC_PERIODIC); }
__device__ __forceinline__ int mapy(const AdjDev& A, int v) { return wrap_or_clamp(v, A.L.ny, A.L.bcy == BC_PERIODIC); }

// ------------------------------------------------------------------ forward intermediates
__global__ void fwd_local(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  if (is_solid(A, x, y)) {
    for (int a = 0; a < 9; ++a) A.fr[a * N + i] = A.fb[a * N + i] = 0.0;
    A.rr[i] = A.rb[i] = A.rn[i] = 0.0;
    return;
  }
  double fr[9], fb[9], rR, rB;
  load_node<double>(A.L, A.src, x, y, fr, fb);
  for (int a = 0; a < 9; ++a) {
    A.fr[a * N + i] = fr[a];
    A.fb[a * N + i] = fb[a];
  }
  A.rn[i] = colour_indicator(fr, fb, rR, rB);
  A.rr[i] = rR;
  A.rb[i] = rB;
}

// Eq. 29 on outermost solid nodes for a field v (fluid values already in v)
__device__ double virtual_value(const AdjDev& A, const double* v, int x, int y) {
  double num = 0.0, den = 0.0;
  for (int b = 1; b < 9; ++b) {
    const int x2 = mapx(A, x + ex(b)), y2 = mapy(A, y + ey(b));
    if (!is_solid(A, x2, y2)) {
      num = radd(num, rmul(wgt<double>(b), v[y2 * A.L.nx + x2]));
      den = radd(den, wgt<double>(b));
    }
  }
  return den > 0.0 ? rdiv(num, den) : 0.0;
}
__device__ double weight_sum(const AdjDev& A, int x, int y) {
  double den = 0.0;
  for (int b = 1; b < 9; ++b)
    if (!is_solid(A, mapx(A, x + ex(b)), mapy(A, y + ey(b)))) den = radd(den, wgt<double>(b));
  return den;
}

__global__ void fwd_virtual(AdjDev A, double* v0, double* v1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (!(flag_at(A, x, y) & F_OSOLID)) return;
  // reads fluid entries only, writes solid entries only: no race
  v0[i] = virtual_value(A, v0, x, y);
  if (v1) v1[i] = virtual_value(A, v1, x, y);
}

__global__ void fwd_grad(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const uint8_t f = flag_at(A, x, y);
  A.pick[i] = 0;
  if (f & F_SOLID) {
    A.grx[i] = A.gry[i] = A.gcx[i] = A.gcy[i] = 0.0;
    A.nxv[i] = A.nyv[i] = 0.0;
    return;
  }
  double gx = 0.0, gy = 0.0;
  for (int a = 1; a < 9; ++a) {
    const double t = rmul(wgt<double>(a), A.rn[mapy(A, y + ey(a)) * A.L.nx + mapx(A, x + ex(a))]);
    if (ex(a) == 1) gx = radd(gx, t);
    if (ex(a) == -1) gx = radd(gx, -t);
    if (ey(a) == 1) gy = radd(gy, t);
    if (ey(a) == -1) gy = radd(gy, -t);
  }
  gx = rdiv(gx, 1.0 / 3.0);
  gy = rdiv(gy, 1.0 / 3.0);
  A.grx[i] = gx;
  A.gry[i] = gy;
  double cgx = gx, cgy = gy;
  const double eps = A.L.grad_eps;
  const double mag = rsqrt_(radd(rmul(gx, gx), rmul(gy, gy)));
  if ((f & F_OFB) && mag > eps) {
    const double esx = rdiv(gx, mag), esy = rdiv(gy, mag);
    const double nsx = A.nsx[i], nsy = A.nsy[i];
    const double c = A.cos_t[i], s = A.sin_t[i];
    const double f1x = rsub(rmul(nsx, c), rmul(nsy, s)), f1y = radd(rmul(nsx, s), rmul(nsy, c));
    const double f2x = radd(rmul(nsx, c), rmul(nsy, s)), f2y = radd(rmul(-nsx, s), rmul(nsy, c));
    const double a1 = rsub(f1x, esx), b1 = rsub(f1y, esy), a2 = rsub(f2x, esx), b2 = rsub(f2y, esy);
    const double d1 = rsqrt_(radd(rmul(a1, a1), rmul(b1, b1)));
    const double d2 = rsqrt_(radd(rmul(a2, a2), rmul(b2, b2)));
    const bool one = d1 <= d2;
    A.pick[i] = one ? 1 : 2;
    cgx = rmul(mag, one ? f1x : f2x);
    cgy = rmul(mag, one ? f1y : f2y);
  }
  A.gcx[i] = cgx;
  A.gcy[i] = cgy;
  const double m2 = sqrt(cgx * cgx + cgy * cgy);
  A.nxv[i] = m2 > eps ? cgx / m2 : 0.0;
  A.nyv[i] = m2 > eps ? cgy / m2 : 0.0;
}

__global__ void fwd_dn(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  double d[4] = {0, 0, 0, 0};
  if (!is_solid(A, x, y)) {
    for (int a = 1; a < 9; ++a) {
      const int j = mapy(A, y + ey(a)) * A.L.nx + mapx(A, x + ex(a));
      const double tx = wgt<double>(a) * A.nxv[j], ty = wgt<double>(a) * A.nyv[j];
      d[0] += ex(a) * tx;
      d[1] += ey(a) * tx;
      d[2] += ex(a) * ty;
      d[3] += ey(a) * ty;
    }
  }
  for (int q = 0; q < 4; ++q) A.dn[q * N + i] = 3.0 * d[q];
}

// ------------------------------------------------------------------ reverse kernels
// Transpose of the push (Eq. 15, half-way bounce-back, open edges) and the reverse of the
// node-local part of the step.
__global__ void adj_collide(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  const LatDev& L = A.L;
  for (int a = 0; a < 9; ++a) A.lf_r[a * N + i] = A.lf_b[a * N + i] = 0.0;
  A.ln_x[i] = A.ln_y[i] = A.lg_x[i] = A.lg_y[i] = A.lrn[i] = 0.0;
  for (int q = 0; q < 4; ++q) A.ldn[q * N + i] = 0.0;
  if (is_solid(A, x, y)) return;
  const bool px = L.bcx == BC_PERIODIC, py = L.bcy == BC_PERIODIC;
  // adjoint of the post-collision, recoloured values (oR_a, oB_a) leaving this node
  double mR[9], mB[9];
  for (int a = 0; a < 9; ++a) {
    mR[a] = mB[a] = 0.0;
    int j = i, slot = a;
    if (a != 0) {
      const int xr = x + ex(a), yr = y + ey(a);
      if ((!px && (xr < 0 || xr >= L.nx)) || (!py && (yr < 0 || yr >= L.ny))) continue;
      const int xd = mapx(A, xr), yd = mapy(A, yr);
      if (is_solid(A, xd, yd)) slot = opp(a);
      else j = yd * L.nx + xd;
    }
    mR[a] = A.lam_next[(2 * slot) * N + j];
    mB[a] = A.lam_next[(2 * slot + 1) * N + j];
  }
  // forward recomputation of the node-local quantities
  double fr[9], fb[9], f[9];
  for (int a = 0; a < 9; ++a) {
    fr[a] = A.fr[a * N + i];
    fb[a] = A.fb[a * N + i];
    f[a] = fr[a] + fb[a];
  }
  const double rhoR = A.rr[i], rhoB = A.rb[i], rn = A.rn[i];
  const double rho = rhoR + rhoB;
  const double nxo = A.nxv[i], nyo = A.nyv[i];
  const double gx = A.gcx[i], gy = A.gcy[i];
  const double dxx = A.dn[i], dxy = A.dn[N + i], dyx = A.dn[2 * N + i], dyy = A.dn[3 * N + i];
  const double kappa = -nxo * nxo * dyy - nyo * nyo * dxx + nxo * nyo * (dxy + dyx);
  const double hsk = 0.5 * L.sigma * kappa;
  const double Fx = hsk * gx, Fy = hsk * gy;
  const double jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const double jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
  const double inv_nu = (1 + rn) * L.h_inv_nuR + (1 - rn) * L.h_inv_nuB;
  const double den_sv = 3.0 + 0.5 * inv_nu;
  const double sv = inv_nu / den_sv;
  const double se = L.s_e, seps = L.s_eps, sq = L.s_q, beta = L.beta;
  const double s14 = f[1] + f[2] + f[3] + f[4], s58 = f[5] + f[6] + f[7] + f[8];
  const double me = -4 * f[0] - s14 + 2 * s58;
  const double meps = 4 * f[0] - 2 * s14 + s58;
  const double qx = -2 * (f[1] - f[3]) + (f[5] - f[6] - f[7] + f[8]);
  const double qy = -2 * (f[2] - f[4]) + (f[5] + f[6] - f[7] - f[8]);
  const double pxx = f[1] - f[2] + f[3] - f[4];
  const double pxy = f[5] - f[6] + f[7] - f[8];
  const double u2 = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
  const double De = se * (me - rho * (-2 + 3 * u2)) - (1 - 0.5 * se) * (6 * uF);
  const double Deps = seps * (meps - rho * (1 - 3 * u2)) + (1 - 0.5 * seps) * (6 * uF);
  const double Dqx = sq * (qx + rho * ux) + (1 - 0.5 * sq) * Fx;
  const double Dqy = sq * (qy + rho * uy) + (1 - 0.5 * sq) * Fy;
  const double Axx = pxx - rho * (ux * ux - uy * uy), Bxx = 2 * (ux * Fx - uy * Fy);
  const double Dxx = sv * Axx - (1 - 0.5 * sv) * Bxx;
  const double Axy = pxy - rho * ux * uy, Bxy = ux * Fy + uy * Fx;
  const double Dxy = sv * Axy - (1 - 0.5 * sv) * Bxy;
  const double ae = De / 36, aeps = Deps / 36, ajx = -Fx / 6, ajy = -Fy / 6;
  const double aqx = Dqx / 12, aqy = Dqy / 12, axx = Dxx / 4, axy = Dxy / 4;
  double fp[9];
  fp[0] = f[0] - (-4 * ae + 4 * aeps);
  const double c14 = -ae - 2 * aeps;
  fp[1] = f[1] - (c14 + ajx - 2 * aqx + axx);
  fp[2] = f[2] - (c14 + ajy - 2 * aqy - axx);
  fp[3] = f[3] - (c14 - ajx + 2 * aqx + axx);
  fp[4] = f[4] - (c14 - ajy + 2 * aqy - axx);
  const double c58 = 2 * ae + aeps;
  fp[5] = f[5] - (c58 + ajx + aqx + ajy + aqy + axy);
  fp[6] = f[6] - (c58 - ajx - aqx + ajy + aqy - axy);
  fp[7] = f[7] - (c58 - ajx - aqx - ajy - aqy + axy);
  fp[8] = f[8] - (c58 + ajx + aqx - ajy - aqy - axy);
  const double cR = rhoR / rho;
  const double pc = beta * rhoR * rhoB / rho;
  // ---- reverse of Eq. 14: oR = cR fp + pc w (e.n), oB = fp - oR
  double lfp[9], lcR = 0, lpc = 0, lnx = 0, lny = 0;
  for (int a = 0; a < 9; ++a) {
    const double mu = mR[a] - mB[a];        // adjoint of oR through both outputs
    const double en = ex(a) * nxo + ey(a) * nyo;
    lfp[a] = mB[a] + mu * cR;
    lcR += mu * fp[a];
    lpc += mu * wgt<double>(a) * en;
    lnx += mu * pc * wgt<double>(a) * ex(a);
    lny += mu * pc * wgt<double>(a) * ey(a);
  }
  double lrhoR = lcR / rho + lpc * beta * rhoB / rho;
  double lrhoB = lpc * beta * rhoR / rho;
  double lrho = -lcR * rhoR / (rho * rho) - lpc * beta * rhoR * rhoB / (rho * rho);
  // ---- reverse of fp = f - M^T diag(...) Delta
  double lf[9];
  for (int a = 0; a < 9; ++a) lf[a] = lfp[a];
  // adjoints of the a_k: l_ak = -sum_a M[k][a] lfp[a]
  const double lae = -(-4 * lfp[0] - lfp[1] - lfp[2] - lfp[3] - lfp[4] + 2 * (lfp[5] + lfp[6] + lfp[7] + lfp[8]));
  const double laeps = -(4 * lfp[0] - 2 * (lfp[1] + lfp[2] + lfp[3] + lfp[4]) + lfp[5] + lfp[6] + lfp[7] + lfp[8]);
  const double lajx = -(lfp[1] - lfp[3] + lfp[5] - lfp[6] - lfp[7] + lfp[8]);
  const double lajy = -(lfp[2] - lfp[4] + lfp[5] + lfp[6] - lfp[7] - lfp[8]);
  const double laqx = -(-2 * lfp[1] + 2 * lfp[3] + lfp[5] - lfp[6] - lfp[7] + lfp[8]);
  const double laqy = -(-2 * lfp[2] + 2 * lfp[4] + lfp[5] + lfp[6] - lfp[7] - lfp[8]);
  const double laxx = -(lfp[1] - lfp[2] + lfp[3] - lfp[4]);
  const double laxy = -(lfp[5] - lfp[6] + lfp[7] - lfp[8]);
  const double lDe = lae / 36, lDeps = laeps / 36, lDqx = laqx / 12, lDqy = laqy / 12;
  const double lDxx = laxx / 4, lDxy = laxy / 4;
  double lFx = -lajx / 6, lFy = -lajy / 6;
  double lux = 0, luy = 0, lu2 = 0, luF = 0, lsv = 0;
  double lme = 0, lmeps = 0, lqx = 0, lqy = 0, lpxx = 0, lpxy = 0;
  // De
  lme += se * lDe;
  lrho += -se * (-2 + 3 * u2) * lDe;
  lu2 += -3 * se * rho * lDe;
  luF += -6 * (1 - 0.5 * se) * lDe;
  // Deps
  lmeps += seps * lDeps;
  lrho += -seps * (1 - 3 * u2) * lDeps;
  lu2 += 3 * seps * rho * lDeps;
  luF += 6 * (1 - 0.5 * seps) * lDeps;
  // Dqx, Dqy
  lqx += sq * lDqx;
  lrho += sq * ux * lDqx;
  lux += sq * rho * lDqx;
  lFx += (1 - 0.5 * sq) * lDqx;
  lqy += sq * lDqy;
  lrho += sq * uy * lDqy;
  luy += sq * rho * lDqy;
  lFy += (1 - 0.5 * sq) * lDqy;
  // Dxx = sv Axx - (1 - sv/2) Bxx
  lsv += (Axx + 0.5 * Bxx) * lDxx;
  lpxx += sv * lDxx;
  lrho += -sv * (ux * ux - uy * uy) * lDxx;
  lux += -2 * sv * rho * ux * lDxx - (1 - 0.5 * sv) * 2 * Fx * lDxx;
  luy += 2 * sv * rho * uy * lDxx + (1 - 0.5 * sv) * 2 * Fy * lDxx;
  lFx += -(1 - 0.5 * sv) * 2 * ux * lDxx;
  lFy += (1 - 0.5 * sv) * 2 * uy * lDxx;
  // Dxy = sv Axy - (1 - sv/2) Bxy
  lsv += (Axy + 0.5 * Bxy) * lDxy;
  lpxy += sv * lDxy;
  lrho += -sv * ux * uy * lDxy;
  lux += -sv * rho * uy * lDxy - (1 - 0.5 * sv) * Fy * lDxy;
  luy += -sv * rho * ux * lDxy - (1 - 0.5 * sv) * Fx * lDxy;
  lFy += -(1 - 0.5 * sv) * ux * lDxy;
  lFx += -(1 - 0.5 * sv) * uy * lDxy;
  // u2, uF
  lux += 2 * ux * lu2 + Fx * luF;
  luy += 2 * uy * lu2 + Fy * luF;
  lFx += ux * luF;
  lFy += uy * luF;
  // moments -> f
  for (int a = 0; a < 9; ++a) {
    const double r1 = (a == 0) ? -4 : (a <= 4 ? -1 : 2);
    const double r2 = (a == 0) ? 4 : (a <= 4 ? -2 : 1);
    const double rqx = (a == 1) ? -2 : (a == 3) ? 2 : (a >= 5 ? (double)ex(a) : 0.0);
    const double rqy = (a == 2) ? -2 : (a == 4) ? 2 : (a >= 5 ? (double)ey(a) : 0.0);
    const double rxx = (a == 1 || a == 3) ? 1 : (a == 2 || a == 4) ? -1 : 0;
    const double rxy = (a >= 5) ? (double)(ex(a) * ey(a)) : 0.0;
    lf[a] += r1 * lme + r2 * lmeps + rqx * lqx + rqy * lqy + rxx * lpxx + rxy * lpxy;
  }
  // sv = inv_nu / (3 + inv_nu / 2); inv_nu = (1 + rn) hR + (1 - rn) hB
  const double linv = lsv * 3.0 / (den_sv * den_sv);
  double lrn_loc = (L.h_inv_nuR - L.h_inv_nuB) * linv;
  A.p_hR[i] += (1 + rn) * linv;
  A.p_hB[i] += (1 - rn) * linv;
  // u = (j + F/2) / rho
  const double ljx = lux / rho, ljy = luy / rho;
  lFx += 0.5 * lux / rho;
  lFy += 0.5 * luy / rho;
  lrho += -(ux * lux + uy * luy) / rho;
  for (int a = 0; a < 9; ++a) lf[a] += ex(a) * ljx + ey(a) * ljy;
  // F = (sigma kappa / 2) g
  const double lhsk = gx * lFx + gy * lFy;
  const double lgx = hsk * lFx, lgy = hsk * lFy;
  A.p_sigma[i] += 0.5 * kappa * lhsk;
  const double lk = 0.5 * L.sigma * lhsk;
  // kappa = -nx^2 dyy - ny^2 dxx + nx ny (dxy + dyx)
  lnx += (-2 * nxo * dyy + nyo * (dxy + dyx)) * lk;
  lny += (-2 * nyo * dxx + nxo * (dxy + dyx)) * lk;
  A.ldn[i] = -nyo * nyo * lk;             // d_x n_x
  A.ldn[N + i] = nxo * nyo * lk;          // d_y n_x
  A.ldn[2 * N + i] = nxo * nyo * lk;      // d_x n_y
  A.ldn[3 * N + i] = -nxo * nxo * lk;     // d_y n_y
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

// transpose of grad n = 3 sum_a w_a e_a n~(x + e_a): scatter onto the virtual-filled n
__global__ void adj_dn(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (is_solid(A, x, y)) return;
  const int N = A.N;
  const double lxx = A.ldn[i], lxy = A.ldn[N + i], lyx = A.ldn[2 * N + i], lyy = A.ldn[3 * N + i];
  for (int a = 1; a < 9; ++a) {
    const int j = mapy(A, y + ey(a)) * A.L.nx + mapx(A, x + ex(a));
    const double w = 3.0 * wgt<double>(a);
    atomicAdd(&A.lnt_x[j], w * (ex(a) * lxx + ey(a) * lxy));
    atomicAdd(&A.lnt_y[j], w * (ex(a) * lyx + ey(a) * lyy));
  }
}

// transpose of Eq. 29 (virtual value of an outermost solid node from its fluid neighbours)
__global__ void adj_virtual(AdjDev A, double* t0, double* t1, double* d0, double* d1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (!(flag_at(A, x, y) & F_OSOLID)) return;
  const double den = weight_sum(A, x, y);
  if (!(den > 0.0)) return;
  for (int b = 1; b < 9; ++b) {
    const int x2 = mapx(A, x + ex(b)), y2 = mapy(A, y + ey(b));
    if (is_solid(A, x2, y2)) continue;
    const int j = y2 * A.L.nx + x2;
    const double c = wgt<double>(b) / den;
    atomicAdd(&d0[j], c * t0[i]);
    if (t1) atomicAdd(&d1[j], c * t1[i]);
  }
}

// reverse of n = g / |g| on fluid nodes
__global__ void adj_n(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (is_solid(A, x, y)) return;
  const double lnx = A.ln_x[i] + A.lnt_x[i], lny = A.ln_y[i] + A.lnt_y[i];
  const double gx = A.gcx[i], gy = A.gcy[i];
  const double m = sqrt(gx * gx + gy * gy);
  if (!(m > A.L.grad_eps)) return;
  const double nx = gx / m, ny = gy / m;
  const double dot = nx * lnx + ny * lny;
  A.lg_x[i] += (lnx - nx * dot) / m;
  A.lg_y[i] += (lny - ny * dot) / m;
}

// reverse of Eq. 30-36: g_c = |g_r| n_f(theta) on Omega_Fb, the identity elsewhere
__global__ void adj_wet(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (is_solid(A, x, y)) return;
  const double lgx = A.lg_x[i], lgy = A.lg_y[i];
  if (A.pick[i] == 0) {
    A.lgr_x[i] = lgx;
    A.lgr_y[i] = lgy;
    return;
  }
  const double gx = A.grx[i], gy = A.gry[i];
  const double m = sqrt(gx * gx + gy * gy);
  const double nsx = A.nsx[i], nsy = A.nsy[i];
  const double c = A.cos_t[i], s = A.sin_t[i];
  double nfx, nfy, dfx, dfy;
  if (A.pick[i] == 1) {   // rotation by +theta
    nfx = nsx * c - nsy * s;
    nfy = nsx * s + nsy * c;
    dfx = -nfy;
    dfy = nfx;
  } else {                // rotation by -theta
    nfx = nsx * c + nsy * s;
    nfy = -nsx * s + nsy * c;
    dfx = nfy;
    dfy = -nfx;
  }
  const double proj = nfx * lgx + nfy * lgy;
  A.lgr_x[i] = gx / m * proj;
  A.lgr_y[i] = gy / m * proj;
  A.p_theta[i] += m * (dfx * lgx + dfy * lgy);
}

// transpose of the raw gradient (Eq. 28 on the virtual-filled rho^N): scatter
__global__ void adj_grad(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (is_solid(A, x, y)) return;
  const double lx = A.lgr_x[i], ly = A.lgr_y[i];
  for (int a = 1; a < 9; ++a) {
    const int j = mapy(A, y + ey(a)) * A.L.nx + mapx(A, x + ex(a));
    atomicAdd(&A.lrnt[j], 3.0 * wgt<double>(a) * (ex(a) * lx + ey(a) * ly));
  }
}

// reverse of rho^N = (rhoR - rhoB)/(rhoR + rhoB) and of the Zou-He columns
__global__ void adj_rho(AdjDev A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int x = i % A.L.nx, y = i / A.L.nx;
  const int N = A.N;
  for (int a = 0; a < 18; ++a) A.lam[a * N + i] = 0.0;
  if (is_solid(A, x, y)) return;
  const double lrn = A.lrn[i] + A.lrnt[i];
  const double rR = A.rr[i], rB = A.rb[i], rho = rR + rB;
  const double cR = 2 * rB / (rho * rho) * lrn, cB = -2 * rR / (rho * rho) * lrn;
  double lr[9], lb[9];
  for (int a = 0; a < 9; ++a) {
    lr[a] = A.lf_r[a * N + i] + cR;
    lb[a] = A.lf_b[a * N + i] + cB;
  }
  const LatDev& L = A.L;
  double sr[9], sb[9];   // adjoint of the stored values
  if (L.bcx == BC_INOUT && x == 0) {
    // inlet: fr = f (f1, f5, f8 from Zou-He of the known totals), fb = 0
    const double u = L.u_in;
    const double ck[9] = {1, 0, 1, 2, 1, 0, 2, 2, 0};
    double lt[9];
    for (int a = 0; a < 9; ++a) lt[a] = 0.0;
    const int known[6] = {0, 2, 3, 4, 6, 7};
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      const double drho = ck[k] / (1 - u);
      double v = lr[k];
      v += lr[1] * ((k == 3 ? 1.0 : 0.0) + 2.0 / 3.0 * u * drho);
      v += lr[5] * ((k == 7 ? 1.0 : 0.0) - (k == 2 ? 0.5 : 0.0) + (k == 4 ? 0.5 : 0.0) + u / 6 * drho);
      v += lr[8] * ((k == 6 ? 1.0 : 0.0) + (k == 2 ? 0.5 : 0.0) - (k == 4 ? 0.5 : 0.0) + u / 6 * drho);
      lt[k] = v;
    }
    for (int a = 0; a < 9; ++a) sr[a] = sb[a] = lt[a];
  } else if (L.bcx == BC_INOUT && x == L.nx - 1) {
    // outlet: known 0,1,2,4,5,8 pass through; f3, f6, f7 from Zou-He, split by frac = kR/kT
    const double* FR = A.fr;
    const double* FB = A.fb;
    const int known[6] = {0, 1, 2, 4, 5, 8};
    double kR = 0, kT = 0;
    for (int q = 0; q < 6; ++q) {
      kR += FR[known[q] * N + i];
      kT += FR[known[q] * N + i] + FB[known[q] * N + i];
    }
    const double frac = kT != 0 ? kR / kT : 0.0;
    double lt[9], lfrac = 0;
    for (int a = 0; a < 9; ++a) lt[a] = 0.0;
    const int unk[3] = {3, 6, 7};
    for (int q = 0; q < 3; ++q) {
      const int uu = unk[q];
      const double fu = FR[uu * N + i] + FB[uu * N + i];
      lt[uu] = frac * lr[uu] + (1 - frac) * lb[uu];   // adjoint of the total f_u
      lfrac += fu * (lr[uu] - lb[uu]);
    }
    // f3 = f1 + 2/3 r - 2/3 S, f7 = f5 + (f2 - f4)/2 + r/6 - S/6, f6 = f8 - (f2 - f4)/2 + r/6 - S/6,
    // S = f0 + f2 + f4 + 2 (f1 + f5 + f8)
    const double cs[9] = {1, 2, 1, 0, 1, 2, 0, 0, 2};
    double ltk[9];
    for (int a = 0; a < 9; ++a) ltk[a] = 0.0;
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      ltk[k] += lt[3] * ((k == 1 ? 1.0 : 0.0) - 2.0 / 3.0 * cs[k]);
      ltk[k] += lt[7] * ((k == 5 ? 1.0 : 0.0) + (k == 2 ? 0.5 : 0.0) - (k == 4 ? 0.5 : 0.0) - cs[k] / 6);
      ltk[k] += lt[6] * ((k == 8 ? 1.0 : 0.0) - (k == 2 ? 0.5 : 0.0) + (k == 4 ? 0.5 : 0.0) - cs[k] / 6);
    }
    for (int a = 0; a < 9; ++a) sr[a] = sb[a] = 0.0;
    for (int q = 0; q < 6; ++q) {
      const int k = known[q];
      const double dfr = kT != 0 ? (kT - kR) / (kT * kT) : 0.0;   // d frac / d s_R
      const double dfb = kT != 0 ? -kR / (kT * kT) : 0.0;         // d frac / d s_B
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

inline int nblk(int n) { return (n + 255) / 256; }

}  // namespace

// One reverse step: lam <- (d step / d state)^T lam_next, parameter adjoints accumulated.
// `A` carries device pointers; the forward intermediates are recomputed from A.src.
cudaError_t adjoint_step(const AdjDev& A, cudaStream_t st) {
  const int b = nblk(A.N);
  fwd_local<<<b, 256, 0, st>>>(A);
  fwd_virtual<<<b, 256, 0, st>>>(A, A.rn, nullptr);
  fwd_grad<<<b, 256, 0, st>>>(A);
  fwd_virtual<<<b, 256, 0, st>>>(A, A.nxv, A.nyv);
  fwd_dn<<<b, 256, 0, st>>>(A);
  cudaMemsetAsync(A.lnt_x, 0, A.N * sizeof(double), st);
  cudaMemsetAsync(A.lnt_y, 0, A.N * sizeof(double), st);
  cudaMemsetAsync(A.lrnt, 0, A.N * sizeof(double), st);
  adj_collide<<<b, 256, 0, st>>>(A);
  adj_dn<<<b, 256, 0, st>>>(A);
  // lnt on outermost solid nodes goes to their fluid neighbours' n
  adj_virtual<<<b, 256, 0, st>>>(A, A.lnt_x, A.lnt_y, A.ln_x, A.ln_y);
  adj_n<<<b, 256, 0, st>>>(A);
  adj_wet<<<b, 256, 0, st>>>(A);
  adj_grad<<<b, 256, 0, st>>>(A);
  adj_virtual<<<b, 256, 0, st>>>(A, A.lrnt, nullptr, A.lrn, nullptr);
  adj_rho<<<b, 256, 0, st>>>(A);
  return cudaGetLastError();
}

// Seed for an objective J = sum_x c(x) rho^N(x) of the stored state: lam = dJ/d(state).
__global__ void k_seed_weighted(AdjDev A, const double* c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.N) return;
  const int N = A.N;
  for (int a = 0; a < 9; ++a) A.lf_r[a * N + i] = A.lf_b[a * N + i] = 0.0;
  A.lrn[i] = 0.0;
  A.lrnt[i] = 0.0;
  const int x = i % A.L.nx, y = i / A.L.nx;
  if (!is_solid(A, x, y)) A.lrn[i] = c[i];
}

cudaError_t adjoint_seed(const AdjDev& A, const double* c, cudaStream_t st) {
  const int b = nblk(A.N);
  fwd_local<<<b, 256, 0, st>>>(A);
  k_seed_weighted<<<b, 256, 0, st>>>(A, c);
  adj_rho<<<b, 256, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace lbcg
