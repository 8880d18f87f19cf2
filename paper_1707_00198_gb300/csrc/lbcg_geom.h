// Host-side geometry of a lattice (Sec. II.C): node flags and neighbour-solid masks, the list
// of outermost fluid nodes with their solid normals (the E8 estimate of Eq. 32-33, or given) and
// contact angles, and the work units of the wall kernel.  Plain C++ (no CUDA types): the
// runtime and the kernels share these layouts, and the host tests build them without a GPU.
#pragma once

#include <stdint.h>

#include <vector>

#include "lbcg.h"

#if defined(__CUDACC__)
#define LBCG_HD __host__ __device__
#else
#define LBCG_HD
#endif

namespace lbcg {

// node flags
enum : uint8_t {
  F_SOLID = 1,    // solid node (indicator s = 1 of Eq. 32)
  F_OFB = 2,      // outermost fluid node (fluid with a solid D2Q9 neighbour), Omega_Fb
  F_OSOLID = 4,   // outermost solid node (solid with a fluid D2Q9 neighbour), Eq. 29
  F_NEAR = 8,     // within Chebyshev distance 3 of a solid node (excluded from the fit)
  F_EDGE = 16,    // fluid node in an open (inlet/outlet) column: some pushes leave the lattice
};

// Entry of the outermost-fluid list: node, its solid normal and contact angle.
struct OfbEntry {
  int lat, x, y, pad_;
  double nsx, nsy, cos_t, sin_t;
};

// Work unit of the wall kernel (one block): consecutive outermost-fluid entries [wall0,
// wall0 + nwall) of lattice `lat`, the fluid nodes [band0, band0 + nband) of the band list
// (each as the offset of its populations in the lattice's pool, pop_node) whose rho^N they
// need, and the outermost solid nodes [virt0, virt0 + nvirt) of the virtual list next to them
// (Eq. 29).  The kernel keeps rho^N of the band nodes in shared memory at
// local indices 0 .. nband-1 and the virtual values at nband .. nband+nvirt-1.
struct WallGroup {
  int lat, wall0, nwall, band0, nband, virt0, nvirt, pad_;
};
// Local indices into that shared array, one per direction a = 1..8 (element a-1): for an
// outermost fluid node, the value at x + e_a (band node or virtual solid node); for a virtual
// node, the band node at x + e_a, or kWallNone if that neighbour is solid.
struct WallSten {
  uint16_t i[8];
};
constexpr uint16_t kWallNone = 0xFFFF;
constexpr int kWallThreads = 128;   // block size
constexpr int kWallMaxNodes = 256;  // outermost fluid nodes per group, at most
constexpr int kWallCap = 1024;      // shared values per group (band + virtual), at most
constexpr int kWallVirtCap = 512;   // virtual nodes per group, at most

// Element offset of the direction-0 pair of node (x, y) within its lattice's population block
// (pitch is a multiple of 32); the pair of direction a is kDir * a further.
constexpr int kDir = 64;          // elements between the pairs of consecutive directions
constexpr int kSeg = 9 * kDir;    // elements of a 32-node row segment
LBCG_HD inline int pop_node(int x, int y, int pitch) {
  return (y * (pitch >> 5) + (x >> 5)) * kSeg + (x & 31) * 2;
}

// D2Q9 directions on the host (the same order as ex()/ey() on the device)
extern const int EXH[9];
extern const int EYH[9];
// periodic wrap, else clamp to [0, n - 1]
int wrap_clamp(int v, int n, bool periodic);

// What the wall groups need of a lattice: its size, row pitch of the node arrays, boundary
// codes and solid indicator ([ny][nx], nonzero = solid).
struct LatGeom {
  int nx, ny, pitch, bcx, bcy;
  const uint8_t* solid;
};

// Flags and neighbour masks ([ny][nx]) of one lattice, and its outermost fluid nodes appended
// to `ofb` (lattice index `lat`, row-major order).
void classify(const lbcg_geometry* g, const lbcg_params* p, int lat, std::vector<uint8_t>& flags,
              std::vector<uint8_t>& mask, std::vector<OfbEntry>& ofb);

// Work units of the wall kernel over the whole `ofb` list (see WallGroup), at most gmax outermost
// fluid nodes each (gmax <= kWallMaxNodes).
void build_wall_groups(const std::vector<LatGeom>& lats, const std::vector<OfbEntry>& ofb, int gmax,
                       std::vector<WallGroup>& groups, std::vector<int>& band, std::vector<WallSten>& virt,
                       std::vector<WallSten>& sten);

}  // namespace lbcg
