// Internal interface between the host runtime (lbcg_host.cu) and the kernel launchers
// (lbcg_kernels.cu, lbcg_obs.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbcg_device.cuh"

namespace lbcg {

// Everything one launch of the step kernels needs (device pointers).
struct LaunchStep {
  const LatDev* lats;
  const WallGroup* groups;   // wall kernel work units
  int ngroups;
  const int* wband;          // band nodes of the groups (population offset in their lattice)
  const WallSten* wvirt;     // virtual (outermost solid) nodes of the groups
  const WallSten* wsten;     // per outermost fluid node: its 8 neighbours' local indices
  const OfbEntry* ofb;       // outermost fluid list
  const int4* tiles;      // tile list (lattice, x0, y0, -)
  int ntiles;
  int ty;                 // tile height (tiles are 32 wide)
  const void* src;
  void* dst;
  const uint8_t* flags;
  const uint8_t* nbmask;  // per node: bit a-1 set if the neighbour in direction a is solid
  void* wall;
  long long node_total;
  const int4* strips;     // sweep schedule: (lattice, x0, y_begin, y_end)
  int nstrips;
  int sweep;              // 1: k_sweep over strips, 0: k_step over tiles
  int scheme_b;           // 1: some lattice of the batch uses wetting scheme (b)
  double* macro;          // non-null: write macroscopic fields instead of stepping (tiles)
  cudaEvent_t* ev;        // non-null: 4 events recorded around k_wall and the step kernel
  int* err;               // device error word: a sweep block's bounded wait ran out
  int poll_limit;         // polls before a sweep block's wait for a staged row gives up
  const uint32_t* sr_epoch;   // 16-bit storage: stochastic-rounding replay counter (device)
  uint32_t sr_step;           // and the step within the replay / the absolute step
};

cudaError_t launch_step(int prec, const LaunchStep& p, cudaStream_t st);
// the number of kernels launch_step launches for p (the wall kernel, the bulk kernel)
inline int step_kernels(const LaunchStep& p) {
  return (p.ngroups > 0 ? 1 : 0) + ((p.sweep && p.macro == nullptr) ? (p.nstrips > 0 ? 1 : 0) : (p.ntiles > 0 ? 1 : 0));
}
// Advances the stochastic-rounding replay counter (one single-thread launch).
cudaError_t launch_sr_tick(uint32_t* epoch, cudaStream_t st);
// One-time kernel attributes for a precision (the sweep's dynamic shared memory); called
// before any launch or graph capture of that precision.
cudaError_t prepare_kernels(int prec);
cudaError_t launch_to_storage(int prec, const LatDev* lats, int lat, long long nn, const double* in,
                              const uint8_t* flags, void* pool, cudaStream_t st);
cudaError_t launch_from_storage(int prec, const LatDev* lats, int lat, long long nn, const void* pool,
                                const uint8_t* flags, double* out, cudaStream_t st);

// Observable reductions over one lattice's macroscopic fields (lbcg_obs.cu).
// `partials` must hold obs_partials_doubles(nx*ny) doubles; `out` receives kObsOut doubles.
constexpr int kObsQ = 17;     // reduced quantities
constexpr int kObsRows = 3;   // row-crossing results
constexpr int kObsOut = kObsQ + kObsRows;
constexpr int kObsBlocks = 304;  // 2 x 152 SMs
size_t obs_partials_doubles();
// Steady-state diagnostics (lbcg_obs.cu): 6 doubles into `out` -- max |du_x|, max |du_y|
// against usnap ([2][node_total], overwritten with the current velocity), rho_R inside / outside
// the circle, rho_B inside / outside.  `partials` holds kObsBlocks * 6 doubles.
cudaError_t launch_diagnostics(const LatDev* lats, int lat, const double* macro, long long node_total,
                               const uint8_t* flags, double* usnap, bool have_snap, double cx, double cy, double r,
                               double* partials, double* out, cudaStream_t st);
cudaError_t launch_observables(const LatDev* lats, int lat, int nx, int ny, const double* macro,
                               long long node_total, const uint8_t* flags, int tip0, int tip1, int cl0, int cl1,
                               double* partials, double* out, cudaStream_t st);

// Device pointers of one reverse step of the adjoint (lbcg_adjoint.cu); node arrays are
// compact [ny][nx], FP64.
template <typename R>
struct AdjDevT {
  LatDev L;
  int N;
  const void* src;       // stored state (population pool of the lattice), FP64 or FP32
  int src_fp32;          // 1: the state is stored in FP32 (an FP32 forward)
  // |grad rho^N| at or below which the reverse sweep takes n = g/|g| as constant.  FP64
  // states: the forward's own guard.  FP32 states: 1e-5 -- their pure phases carry rounding
  // noise |grad rho^N| ~ 1e-7 whose normals the forward only ever multiplies by ~0, but whose
  // 1/|g| ~ 1e8 would give the linearised map a spurious growing mode.
  double n_eps;
  const uint8_t* flags;  // node flags (pitch layout)
  const uint8_t* sol;    // compact [ny][nx]: 1 on solid nodes
  const uint8_t* nbm;    // compact [ny][nx], every node: bit a-1 set if its neighbour in
                         // direction a (periodic wrap, else clamp) is solid
  const R* nsx;     // solid normal at outermost fluid nodes (compact, 0 elsewhere)
  const R* nsy;
  const R* cos_t;   // cos and sin of the contact angle per node (compact)
  const R* sin_t;
  // forward intermediates (compact)
  R *fr, *fb;       // [9][N] post-streaming populations after the Zou-He columns
  R *rr, *rb, *rn;  // colour densities, rho^N (fluid nodes; 0 on solid nodes)
  R *grx, *gry;     // raw gradient (Eq. 28)
  R *gcx, *gcy;     // corrected gradient (Eq. 31; = raw off Omega_Fb)
  R *nxv, *nyv;     // n on fluid nodes (0 on solid nodes)
  R *dn;            // [4][N] d_x n_x, d_y n_x, d_x n_y, d_y n_y
  int *pick;             // 1 or 2: the candidate Eq. 36 chose (0 off Omega_Fb / below guard)
  // adjoints
  const R* lam_next;  // [18][N] adjoint of the stored state after the step: (fr, fb) pairs
  R* lam;             // [18][N] adjoint of the stored state before the step
  R *lf_r, *lf_b;     // [9][N] adjoint of the post-Zou-He populations
  R *ln_x, *ln_y;     // adjoint of n (local part)
  R *lnt_x, *lnt_y;   // adjoint of n through the neighbours' grad n (scatter target)
  R *lg_x, *lg_y;     // adjoint of the corrected gradient (force path)
  R *lrn, *lrnt;      // adjoint of rho^N: local part, and through the neighbours' gradient
  double *p_sigma, *p_hR, *p_hB, *p_theta;  // per-node parameter adjoints (accumulated)
};

// R: the arithmetic of the reverse kernels (double, or float for the FP32 reverse sweep);
// the per-node parameter adjoints accumulate in double either way.
// adjoint_forward: the forward intermediates of state A.src into A's intermediate arrays.
// adjoint_step: the reverse of the step from A.src (lam <- J^T lam_next), using A's
// intermediates; with B non-null it also computes B's (the state before A's), which must use
// other intermediate and scatter-target arrays than A (the reverse arrays may be shared).
template <typename R>
cudaError_t adjoint_forward(const AdjDevT<R>& A, cudaStream_t st);
template <typename R>
cudaError_t adjoint_step(const AdjDevT<R>& A, const AdjDevT<R>* B, cudaStream_t st);
// seed lam = dJ/d(state): J = sum weight * rho^N (red_mass false) or the red mass (true)
template <typename R>
cudaError_t adjoint_seed(const AdjDevT<R>& A, const R* weight, bool red_mass, cudaStream_t st);

// Sets the calling thread's message returned by lbcg_last_error() (lbcg_host.cu).
void set_last_error(const char* msg);

}  // namespace lbcg
