/*
 * Plain C (OpenMP) implementation of one time step of the two-colour D2Q9 MRT colour-gradient
 * lattice Boltzmann method with the improved geometric wetting scheme (Yu, Liu, Zhang & Liang,
 * arXiv 1707.00198, Sec. II), in FP64, node by node.
 *
 * THIS IS TEST INFRASTRUCTURE, like the PyTorch oracle beside it: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.  It shares no code with the
 * CUDA library or with the PyTorch oracle; the tests check it against the PyTorch oracle, so
 * two independent CPU implementations of the paper pin each other, and bench.py times it on
 * the host cores as the CPU baseline.
 *
 * Readings (the same as the oracle's): the last row of M (Eq. 3) is e_x e_y; the blue line of
 * Eq. 14 carries a minus sign and its perturbation is w_a (e_a . n); each colour streams
 * itself (Eq. 15); tau_v = 3 nu + 1/2 with the harmonic nu of Eq. 18 per node; u of Eq. 17
 * feeds Eq. 7 and 9; n = 0 where |grad rho^N| <= grad_eps; Omega_Fb = fluid nodes with a solid
 * D2Q9 neighbour, outermost solid nodes = solid nodes with a fluid neighbour (Eq. 29); the
 * corrected gradient of Eq. 31 replaces the raw one downstream; n_s of Eq. 32 points into
 * the solid, theta is measured through red, Eq. 34 rotates n_s by +theta for candidate 1 and
 * the tie of Eq. 36 goes to candidate 1; the E8 stencil (Eq. 32-33) wraps on periodic axes,
 * sees solid beyond closed edges and copies the edge column on the inlet/outlet axis;
 * Zou-He velocity inlet carrying red at x = 0 and pressure outlet at x = nx-1 (Sec. III.D),
 * whose unknown populations take the red fraction of the known ones.
 *
 * Layout: populations [9][ny][nx] per colour, row-major, x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { BCX_PERIODIC = 0, BCX_CLOSED = 1, BCX_INOUT = 2 };
enum { BCY_PERIODIC = 0, BCY_CLOSED = 1 };

static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

typedef struct {
  double nu_R, nu_B, sigma, beta, s_e, s_eps, s_q, rho0, u_in, rho_out, grad_eps;
  int inlet_profile, wetting;
} cpu_params;

/* Lattice: geometry, classification and the work arrays of one step (allocated by setup). */
typedef struct {
  int nx, ny, bcx, bcy;
  cpu_params p;
  uint8_t *solid, *ofb, *osolid;
  double *nsx, *nsy, *cth, *sth;   /* solid normal at Omega_Fb nodes; cos, sin of theta */
  double Minv[81];                 /* inverse of M (Eq. 3), by Gauss-Jordan elimination */
  double in_y0, in_w;              /* Poiseuille inlet: s = (y - in_y0) / in_w */
  /* work */
  double *rR, *rB, *rN, *gx, *gy, *nX, *nY, *fill, *Fx, *Fy, *pR, *pB;
} cpu_lattice;

static const double M[81] = {
    1, 1, 1, 1, 1, 1, 1, 1, 1,            /* rho */
    -4, -1, -1, -1, -1, 2, 2, 2, 2,       /* e */
    4, -2, -2, -2, -2, 1, 1, 1, 1,        /* epsilon */
    0, 1, 0, -1, 0, 1, -1, -1, 1,         /* j_x */
    0, -2, 0, 2, 0, 1, -1, -1, 1,         /* q_x */
    0, 0, 1, 0, -1, 1, 1, -1, -1,         /* j_y */
    0, 0, -2, 0, 2, 1, 1, -1, -1,         /* q_y */
    0, 1, -1, 1, -1, 0, 0, 0, 0,          /* p_xx */
    0, 0, 0, 0, 0, 1, -1, 1, -1};         /* p_xy = e_x e_y (the printed row is garbled) */

/* index of x + dx along an axis: periodic wrap, else clamp (the ghost copies the edge node) */
static int nb_index(int v, int n, int periodic) {
  if (periodic) return ((v % n) + n) % n;
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

static int idx(const cpu_lattice* L, int x, int y) { return y * L->nx + x; }

static int neighbour(const cpu_lattice* L, int x, int y, int dx, int dy) {
  return idx(L, nb_index(x + dx, L->nx, L->bcx == BCX_PERIODIC), nb_index(y + dy, L->ny, L->bcy == BCY_PERIODIC));
}

static void invert9(const double* A, double* out) {
  double a[9][18];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 18; ++j) a[i][j] = j < 9 ? A[i * 9 + j] : (j - 9 == i ? 1.0 : 0.0);
  for (int c = 0; c < 9; ++c) {
    int piv = c;
    for (int r = c + 1; r < 9; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    for (int j = 0; j < 18; ++j) {
      double t = a[c][j];
      a[c][j] = a[piv][j];
      a[piv][j] = t;
    }
    const double d = a[c][c];
    for (int j = 0; j < 18; ++j) a[c][j] /= d;
    for (int r = 0; r < 9; ++r)
      if (r != c) {
        const double f = a[r][c];
        for (int j = 0; j < 18; ++j) a[r][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) out[i * 9 + j] = a[i][j + 9];
}

/* E8 stencil value of the solid indicator beyond the array (Eq. 32 edge rule) */
static double e8_solid(const cpu_lattice* L, int x, int y) {
  if (x < 0 || x >= L->nx) {
    if (L->bcx == BCX_PERIODIC) x = nb_index(x, L->nx, 1);
    else if (L->bcx == BCX_CLOSED) return 1.0;
    else x = x < 0 ? 0 : L->nx - 1;
  }
  if (y < 0 || y >= L->ny) {
    if (L->bcy == BCY_PERIODIC) y = nb_index(y, L->ny, 1);
    else return 1.0;
  }
  return L->solid[idx(L, x, y)] ? 1.0 : 0.0;
}

void lbcg_cpu_destroy(cpu_lattice* L) {
  if (!L) return;
  void* ptrs[] = {L->solid, L->ofb, L->osolid, L->nsx, L->nsy, L->cth, L->sth, L->rR, L->rB, L->rN, L->gx,
                  L->gy, L->nX, L->nY, L->fill, L->Fx, L->Fy, L->pR, L->pB};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
  free(L);
}

/* Set up a lattice: classification (Sec. II.C), solid normals (given, else Eq. 32-33) and
 * contact angles (per node, else the global theta).  normal: [2][ny][nx] or NULL; theta_node:
 * [ny][nx] or NULL.  Returns NULL if memory runs out. */
cpu_lattice* lbcg_cpu_create(int nx, int ny, int bcx, int bcy, const uint8_t* solid, const double* normal,
                             const double* theta_node, double theta, const cpu_params* p) {
  cpu_lattice* L = (cpu_lattice*)calloc(1, sizeof(cpu_lattice));
  if (!L) return NULL;
  const size_t n = (size_t)nx * ny;
  L->nx = nx;
  L->ny = ny;
  L->bcx = bcx;
  L->bcy = bcy;
  L->p = *p;
  L->solid = (uint8_t*)malloc(n);
  L->ofb = (uint8_t*)calloc(n, 1);
  L->osolid = (uint8_t*)calloc(n, 1);
  double** arrs[] = {&L->nsx, &L->nsy, &L->cth, &L->sth, &L->rR, &L->rB, &L->rN, &L->gx, &L->gy,
                     &L->nX, &L->nY, &L->fill, &L->Fx, &L->Fy};
  int ok = L->solid && L->ofb && L->osolid;
  for (size_t i = 0; i < sizeof(arrs) / sizeof(arrs[0]); ++i) {
    *arrs[i] = (double*)calloc(n, sizeof(double));
    ok = ok && *arrs[i];
  }
  L->pR = (double*)calloc(9 * n, sizeof(double));
  L->pB = (double*)calloc(9 * n, sizeof(double));
  if (!ok || !L->pR || !L->pB) {
    lbcg_cpu_destroy(L);
    return NULL;
  }
  for (size_t i = 0; i < n; ++i) L->solid[i] = solid[i] != 0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      int any_fluid = 0, any_solid = 0;
      for (int a = 1; a < 9; ++a) {
        const int j = neighbour(L, x, y, EX[a], EY[a]);
        if (L->solid[j]) any_solid = 1;
        else any_fluid = 1;
      }
      L->osolid[i] = L->solid[i] && any_fluid;
      L->ofb[i] = !L->solid[i] && any_solid;
      const double th = theta_node ? theta_node[i] : theta;
      L->cth[i] = cos(th);
      L->sth[i] = sin(th);
    }
  /* solid normal at Omega_Fb nodes: analytic, or Eq. 32 with the Eq. 33 weights in units of
   * 1/5040 (960, 448, 84, 32, 1 for |c|^2 = 1, 2, 4, 5, 8), which the normalisation cancels */
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      if (!L->ofb[i]) continue;
      if (normal) {
        L->nsx[i] = normal[i];
        L->nsy[i] = normal[n + i];
        continue;
      }
      double vx = 0, vy = 0;
      for (int cy = -2; cy <= 2; ++cy)
        for (int cx = -2; cx <= 2; ++cx) {
          const int c2 = cx * cx + cy * cy;
          double k = 0;
          if (c2 == 1) k = 960;
          else if (c2 == 2) k = 448;
          else if (c2 == 4) k = 84;
          else if (c2 == 5) k = 32;
          else if (c2 == 8) k = 1;
          if (k == 0) continue;
          const double s = e8_solid(L, x + cx, y + cy);
          vx += k * s * cx;
          vy += k * s * cy;
        }
      const double m = sqrt(vx * vx + vy * vy);
      if (m > 0) {
        L->nsx[i] = vx / m;
        L->nsy[i] = vy / m;
      }
    }
  invert9(M, L->Minv);
  /* Poiseuille inlet: the fluid rows of column 0, walls half a node beyond */
  int lo = -1, hi = -1;
  for (int y = 0; y < ny; ++y)
    if (!L->solid[idx(L, 0, y)]) {
      if (lo < 0) lo = y;
      hi = y;
    }
  L->in_y0 = lo < 0 ? 0.0 : lo - 0.5;
  L->in_w = lo < 0 ? 1.0 : (double)(hi - lo + 1);
  return L;
}

/* Eq. 29: the w-weighted mean of phi over the D2Q9 fluid neighbours of outermost solid node i */
static double virtual_value(const cpu_lattice* L, const double* phi, int x, int y) {
  double num = 0, den = 0;
  for (int a = 1; a < 9; ++a) {
    const int j = neighbour(L, x, y, EX[a], EY[a]);
    if (!L->solid[j]) {
      num += W[a] * phi[j];
      den += W[a];
    }
  }
  return num / den;
}

/* Eq. 28 of field `fill` at node (x, y): (1/c_s^2) sum_a w_a fill(x + e_a) e_a */
static void iso_gradient(const cpu_lattice* L, const double* fill, int x, int y, double* gx, double* gy) {
  double sx = 0, sy = 0;
  for (int a = 1; a < 9; ++a) {
    const double v = fill[neighbour(L, x, y, EX[a], EY[a])];
    sx += W[a] * v * EX[a];
    sy += W[a] * v * EY[a];
  }
  *gx = sx * 3.0;
  *gy = sy * 3.0;
}

/* Eq. 48 (scheme (b)), each component normalised by sum_a w_a e_ai^2 over fluid directions */
static void one_sided_gradient(const cpu_lattice* L, const double* phi, int x, int y, double* gx, double* gy) {
  double sx = 0, sy = 0, wx = 0, wy = 0;
  const double c = phi[idx(L, x, y)];
  for (int a = 1; a < 9; ++a) {
    const int j = neighbour(L, x, y, EX[a], EY[a]);
    if (L->solid[j]) continue;
    const double d = phi[j] - c;
    sx += W[a] * d * EX[a];
    sy += W[a] * d * EY[a];
    wx += W[a] * EX[a] * EX[a];
    wy += W[a] * EY[a] * EY[a];
  }
  *gx = wx > 0 ? sx / wx : 0.0;
  *gy = wy > 0 ? sy / wy : 0.0;
}

/* One time step: (fR, fB) -> (oR, oB), [9][ny][nx] each; nthreads <= 0 uses OpenMP's default. */
void lbcg_cpu_step(cpu_lattice* L, const double* fR, const double* fB, double* oR, double* oB, int nthreads) {
  const int nx = L->nx, ny = L->ny;
  const int n = nx * ny;
  const cpu_params* p = &L->p;
  const double eps = p->grad_eps;
#ifdef _OPENMP
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();  /* per loop: no global setting */
#else
  (void)nthreads;
#endif
  /* 1. colour densities and rho^N (Eq. 16, 12) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int i = 0; i < n; ++i) {
    double r = 0, b = 0;
    if (!L->solid[i])
      for (int a = 0; a < 9; ++a) {
        r += fR[a * n + i];
        b += fB[a * n + i];
      }
    L->rR[i] = r;
    L->rB[i] = b;
    L->rN[i] = L->solid[i] ? 0.0 : (r - b) / (r + b);
  }
  /* 2. rho^N on the outermost solid nodes: Eq. 29, or cos(theta) (surface-energy variant) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      if (!L->solid[i]) L->fill[i] = L->rN[i];
      else if (!L->osolid[i]) L->fill[i] = 0.0;
      else L->fill[i] = p->wetting == 2 ? L->cth[i] : virtual_value(L, L->rN, x, y);
    }
  /* 3. grad rho^N (Eq. 28), wetting correction on Omega_Fb (Eq. 30-36), n (Eq. 11) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      double gx = 0, gy = 0, nxv = 0, nyv = 0;
      if (!L->solid[i]) {
        iso_gradient(L, L->fill, x, y, &gx, &gy);
        const double mag = sqrt(gx * gx + gy * gy);
        if (L->ofb[i] && p->wetting != 2 && mag > eps) {
          const double esx = gx / mag, esy = gy / mag;                          /* Eq. 30 */
          const double nsx = L->nsx[i], nsy = L->nsy[i], c = L->cth[i], s = L->sth[i];
          const double f1x = nsx * c - nsy * s, f1y = nsx * s + nsy * c;       /* Eq. 34, +theta */
          const double f2x = nsx * c + nsy * s, f2y = -nsx * s + nsy * c;      /* Eq. 34, -theta */
          const double d1 = sqrt((f1x - esx) * (f1x - esx) + (f1y - esy) * (f1y - esy));  /* Eq. 35 */
          const double d2 = sqrt((f2x - esx) * (f2x - esx) + (f2y - esy) * (f2y - esy));
          gx = mag * (d1 <= d2 ? f1x : f2x);                                    /* Eq. 36, 31 */
          gy = mag * (d1 <= d2 ? f1y : f2y);
        }
        const double m2 = sqrt(gx * gx + gy * gy);
        if (m2 > eps) {
          nxv = gx / m2;
          nyv = gy / m2;
        }
      }
      L->gx[i] = gx;
      L->gy[i] = gy;
      L->nX[i] = nxv;
      L->nY[i] = nyv;
    }
  /* 4. grad n (Eq. 28 with the virtual n of Eq. 29; Eq. 48 on Omega_Fb in scheme (b)),
   *    curvature (Eq. 13), force (Eq. 10) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      double Fx = 0, Fy = 0;
      if (!L->solid[i]) {
        double nfx[9], nfy[9];
        for (int a = 1; a < 9; ++a) {
          const int j = neighbour(L, x, y, EX[a], EY[a]);
          const int jx = nb_index(x + EX[a], nx, L->bcx == BCX_PERIODIC);
          const int jy = nb_index(y + EY[a], ny, L->bcy == BCY_PERIODIC);
          if (!L->solid[j]) {
            nfx[a] = L->nX[j];
            nfy[a] = L->nY[j];
          } else if (L->osolid[j]) {
            nfx[a] = virtual_value(L, L->nX, jx, jy);
            nfy[a] = virtual_value(L, L->nY, jx, jy);
          } else {
            nfx[a] = nfy[a] = 0.0;
          }
        }
        double dxx = 0, dxy = 0, dyx = 0, dyy = 0;   /* d_x n_x, d_y n_x, d_x n_y, d_y n_y */
        for (int a = 1; a < 9; ++a) {
          dxx += W[a] * nfx[a] * EX[a];
          dxy += W[a] * nfx[a] * EY[a];
          dyx += W[a] * nfy[a] * EX[a];
          dyy += W[a] * nfy[a] * EY[a];
        }
        dxx *= 3.0;
        dxy *= 3.0;
        dyx *= 3.0;
        dyy *= 3.0;
        if (p->wetting == 1 && L->ofb[i]) {
          one_sided_gradient(L, L->nX, x, y, &dxx, &dxy);
          one_sided_gradient(L, L->nY, x, y, &dyx, &dyy);
        }
        const double nxv = L->nX[i], nyv = L->nY[i];
        const double kappa = -nxv * nxv * dyy - nyv * nyv * dxx + nxv * nyv * (dxy + dyx);
        Fx = 0.5 * p->sigma * kappa * L->gx[i];
        Fy = 0.5 * p->sigma * kappa * L->gy[i];
      }
      L->Fx[i] = Fx;
      L->Fy[i] = Fy;
    }
  /* 5. velocity (Eq. 17), viscosity (Eq. 18), MRT collision with Guo forcing (Eq. 1-9),
   *    recolouring (Eq. 14) -> post-collision populations pR, pB */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int i = 0; i < n; ++i) {
    if (L->solid[i]) {
      for (int a = 0; a < 9; ++a) L->pR[a * n + i] = L->pB[a * n + i] = 0.0;
      continue;
    }
    double f[9], feq[9], src[9], mneq[9], mF[9], S[9];
    const double rhoR = L->rR[i], rhoB = L->rB[i], rho = rhoR + rhoB;
    double jx = 0, jy = 0;
    for (int a = 0; a < 9; ++a) {
      f[a] = fR[a * n + i] + fB[a * n + i];
      jx += f[a] * EX[a];
      jy += f[a] * EY[a];
    }
    const double Fx = L->Fx[i], Fy = L->Fy[i];
    const double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    const double usq = ux * ux + uy * uy;
    for (int a = 0; a < 9; ++a) {
      const double eu = EX[a] * ux + EY[a] * uy;
      feq[a] = rho * W[a] * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * usq);                         /* Eq. 7 */
      src[a] = W[a] * (((EX[a] - ux) * 3 + eu * EX[a] * 9) * Fx + ((EY[a] - uy) * 3 + eu * EY[a] * 9) * Fy); /* Eq. 9 */
    }
    const double rn = L->rN[i];
    const double inv_nu = (1 + rn) / (2 * p->nu_R) + (1 - rn) / (2 * p->nu_B);
    const double sv = 1.0 / (3.0 / inv_nu + 0.5);
    S[0] = 1;
    S[1] = p->s_e;
    S[2] = p->s_eps;
    S[3] = 1;
    S[4] = p->s_q;
    S[5] = 1;
    S[6] = p->s_q;
    S[7] = sv;
    S[8] = sv;
    for (int k = 0; k < 9; ++k) {
      double a1 = 0, a2 = 0;
      for (int a = 0; a < 9; ++a) {
        a1 += M[k * 9 + a] * (f[a] - feq[a]);
        a2 += M[k * 9 + a] * src[a];
      }
      mneq[k] = S[k] * a1;
      mF[k] = (1 - 0.5 * S[k]) * a2;
    }
    const double nxv = L->nX[i], nyv = L->nY[i];
    for (int a = 0; a < 9; ++a) {
      double om = 0, fb = 0;
      for (int k = 0; k < 9; ++k) {
        om += L->Minv[a * 9 + k] * mneq[k];
        fb += L->Minv[a * 9 + k] * mF[k];
      }
      const double fp = f[a] - om + fb;                                                        /* Eq. 1, 8 */
      const double pert = p->beta * rhoR * rhoB / rho * W[a] * (EX[a] * nxv + EY[a] * nyv);
      L->pR[a * n + i] = rhoR / rho * fp + pert;                                               /* Eq. 14 */
      L->pB[a * n + i] = rhoB / rho * fp - pert;
    }
  }
  /* 6. streaming (Eq. 15) by push: f''_a(x) goes to x + e_a if that is a fluid node of the
   *    lattice, back into the opposite slot of x if it is solid (half-way bounce-back), and
   *    nowhere if it lies beyond an open edge */
  memset(oR, 0, sizeof(double) * 9 * (size_t)n);
  memset(oB, 0, sizeof(double) * 9 * (size_t)n);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int i = idx(L, x, y);
      if (L->solid[i]) continue;
      for (int a = 0; a < 9; ++a) {
        int tx = x + EX[a], ty = y + EY[a];
        const int out_x = (tx < 0 || tx >= nx) && L->bcx != BCX_PERIODIC;
        const int out_y = (ty < 0 || ty >= ny) && L->bcy != BCY_PERIODIC;
        int j, slot;
        if (out_x || out_y) {
          /* beyond an edge: dropped at an open edge; closed edges are solid, so a fluid node
           * never reaches them.  The ghost of an open column copies the edge node, whose
           * solidity decides a bounce-back there. */
          const int gj = neighbour(L, x, y, EX[a], EY[a]);
          if (L->solid[gj]) {
            j = i;
            slot = OPP[a];
          } else {
            continue;
          }
        } else {
          tx = nb_index(tx, nx, 1);
          ty = nb_index(ty, ny, 1);
          j = idx(L, tx, ty);
          slot = a;
          if (L->solid[j]) {
            j = i;
            slot = OPP[a];
          }
        }
        /* each slot receives exactly one population (pushes never collide) */
        oR[slot * n + j] = L->pR[a * n + i];
        oB[slot * n + j] = L->pB[a * n + i];
      }
    }
  if (L->bcx != BCX_INOUT) return;
  /* 7. Zou-He columns (Sec. III.D): inlet x = 0 (velocity, red only; unknown 1, 5, 8),
   *    outlet x = nx-1 (density rho_out; unknown 3, 6, 7 with the known red fraction) */
  for (int y = 0; y < ny; ++y) {
    int i = idx(L, 0, y);
    if (!L->solid[i]) {
      double f[9];
      for (int a = 0; a < 9; ++a) f[a] = oR[a * n + i] + oB[a * n + i];
      double u = p->u_in;
      if (p->inlet_profile) {
        const double s = (y - L->in_y0) / L->in_w;
        u = 4 * p->u_in * s * (1 - s);
      }
      const double rho = (f[0] + f[2] + f[4] + 2 * (f[3] + f[6] + f[7])) / (1 - u);
      f[1] = f[3] + 2.0 / 3.0 * rho * u;
      f[5] = f[7] - 0.5 * (f[2] - f[4]) + rho * u / 6.0;
      f[8] = f[6] + 0.5 * (f[2] - f[4]) + rho * u / 6.0;
      for (int a = 0; a < 9; ++a) {
        oR[a * n + i] = f[a];
        oB[a * n + i] = 0.0;
      }
    }
    i = idx(L, nx - 1, y);
    if (!L->solid[i]) {
      double fr[9], f[9];
      for (int a = 0; a < 9; ++a) {
        fr[a] = oR[a * n + i];
        f[a] = fr[a] + oB[a * n + i];
      }
      const double r = p->rho_out;
      const double ux = -1 + (f[0] + f[2] + f[4] + 2 * (f[1] + f[5] + f[8])) / r;
      const double u3 = f[1] - 2.0 / 3.0 * r * ux;
      const double u7 = f[5] + 0.5 * (f[2] - f[4]) - r * ux / 6.0;
      const double u6 = f[8] - 0.5 * (f[2] - f[4]) - r * ux / 6.0;
      const double kR = fr[0] + fr[1] + fr[2] + fr[4] + fr[5] + fr[8];
      const double kT = f[0] + f[1] + f[2] + f[4] + f[5] + f[8];
      const double frac = kT != 0 ? kR / kT : 0.0;
      const int un[3] = {3, 6, 7};
      const double uv[3] = {u3, u6, u7};
      for (int q = 0; q < 3; ++q) {
        oR[un[q] * n + i] = frac * uv[q];
        oB[un[q] * n + i] = (1 - frac) * uv[q];
      }
    }
  }
}

/* The open columns of a post-streaming state (Sec. III.D) applied in place: the initial state
 * of an inlet/outlet lattice satisfies them too.  Implemented as a step's column pass. */
void lbcg_cpu_open_columns(cpu_lattice* L, double* fR, double* fB) {
  const int nx = L->nx, ny = L->ny, n = nx * ny;
  const cpu_params* p = &L->p;
  if (L->bcx != BCX_INOUT) return;
  for (int y = 0; y < ny; ++y) {
    int i = idx(L, 0, y);
    if (!L->solid[i]) {
      double f[9];
      for (int a = 0; a < 9; ++a) f[a] = fR[a * n + i] + fB[a * n + i];
      double u = p->u_in;
      if (p->inlet_profile) {
        const double s = (y - L->in_y0) / L->in_w;
        u = 4 * p->u_in * s * (1 - s);
      }
      const double rho = (f[0] + f[2] + f[4] + 2 * (f[3] + f[6] + f[7])) / (1 - u);
      f[1] = f[3] + 2.0 / 3.0 * rho * u;
      f[5] = f[7] - 0.5 * (f[2] - f[4]) + rho * u / 6.0;
      f[8] = f[6] + 0.5 * (f[2] - f[4]) + rho * u / 6.0;
      for (int a = 0; a < 9; ++a) {
        fR[a * n + i] = f[a];
        fB[a * n + i] = 0.0;
      }
    }
    i = idx(L, nx - 1, y);
    if (!L->solid[i]) {
      double fr[9], f[9];
      for (int a = 0; a < 9; ++a) {
        fr[a] = fR[a * n + i];
        f[a] = fr[a] + fB[a * n + i];
      }
      const double r = p->rho_out;
      const double ux = -1 + (f[0] + f[2] + f[4] + 2 * (f[1] + f[5] + f[8])) / r;
      const double u3 = f[1] - 2.0 / 3.0 * r * ux;
      const double u7 = f[5] + 0.5 * (f[2] - f[4]) - r * ux / 6.0;
      const double u6 = f[8] - 0.5 * (f[2] - f[4]) - r * ux / 6.0;
      const double kR = fr[0] + fr[1] + fr[2] + fr[4] + fr[5] + fr[8];
      const double kT = f[0] + f[1] + f[2] + f[4] + f[5] + f[8];
      const double frac = kT != 0 ? kR / kT : 0.0;
      const int un[3] = {3, 6, 7};
      const double uv[3] = {u3, u6, u7};
      for (int q = 0; q < 3; ++q) {
        fR[un[q] * n + i] = frac * uv[q];
        fB[un[q] * n + i] = (1 - frac) * uv[q];
      }
    }
  }
}

/* Threads a step may use: OpenMP's default team size, or 1 without OpenMP. */
int lbcg_cpu_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int lbcg_cpu_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}
