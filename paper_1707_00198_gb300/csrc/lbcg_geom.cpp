// Host-side geometry of a lattice: classification of its nodes, the outermost-fluid list with
// the solid normals, and the work units of the wall kernel (declarations in lbcg_geom.h).
#include "lbcg_geom.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace lbcg {

int wrap_clamp(int v, int n, bool periodic) {
  if (periodic) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

const int EXH[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int EYH[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Classification of one lattice (Sec. II.C): flags, neighbour masks, outermost-fluid entries.
void classify(const lbcg_geometry* g, const lbcg_params* p, int lat, std::vector<uint8_t>& flags_local,
              std::vector<uint8_t>& mask_local, std::vector<OfbEntry>& ofb) {
  const int nx = g->nx, ny = g->ny;
  const bool px = g->bc_x == LBCG_BCX_PERIODIC, py = g->bc_y == LBCG_BCY_PERIODIC;
  auto S = [&](int x, int y) { return g->solid[(size_t)y * nx + x] != 0; };
  flags_local.assign((size_t)nx * ny, 0);
  mask_local.assign((size_t)nx * ny, 0);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      uint8_t f = 0;
      const bool s = S(x, y);
      bool any_s = false, any_f = false;
      uint8_t m = 0;
      for (int a = 1; a < 9; ++a) {
        const bool sn = S(wrap_clamp(x + EXH[a], nx, px), wrap_clamp(y + EYH[a], ny, py));
        any_s |= sn;
        any_f |= !sn;
        if (sn) m |= uint8_t(1u << (a - 1));
      }
      if (!s) mask_local[(size_t)y * nx + x] = m;
      if (!s && g->bc_x == LBCG_BCX_INOUT && (x == 0 || x == nx - 1)) f |= F_EDGE;
      if (s) {
        f |= F_SOLID;
        if (any_f) f |= F_OSOLID;
      } else if (any_s) {
        f |= F_OFB;
      }
      bool near = false;
      for (int dy = -3; dy <= 3 && !near; ++dy)
        for (int dx = -3; dx <= 3 && !near; ++dx)
          near = S(wrap_clamp(x + dx, nx, px), wrap_clamp(y + dy, ny, py));
      if (near) f |= F_NEAR;
      flags_local[(size_t)y * nx + x] = f;
    }
  // E8 stencil (Eq. 33): the weights are k/5040 with integer k = 960, 448, 84, 32, 1 for
  // |c|^2 = 1, 2, 4, 5, 8; the sums are taken exactly over the integers k
  struct C8 {
    int cx, cy, k;
  };
  std::vector<C8> st;
  for (int cy = -2; cy <= 2; ++cy)
    for (int cx = -2; cx <= 2; ++cx) {
      const int c2 = cx * cx + cy * cy;
      const int k = c2 == 1 ? 960 : c2 == 2 ? 448 : c2 == 4 ? 84 : c2 == 5 ? 32 : c2 == 8 ? 1 : 0;
      if (k) st.push_back({cx, cy, k});
    }
  auto s_e8 = [&](int x, int y) -> int {
    // edge rule: periodic wrap; closed -> solid; inlet/outlet x -> copy of the edge column
    if (x < 0 || x >= nx) {
      if (px) x = wrap_clamp(x, nx, true);
      else if (g->bc_x == LBCG_BCX_CLOSED) return 1;
      else x = wrap_clamp(x, nx, false);
    }
    if (y < 0 || y >= ny) {
      if (py) y = wrap_clamp(y, ny, true);
      else return 1;
    }
    return S(x, y) ? 1 : 0;
  };
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (!(flags_local[(size_t)y * nx + x] & F_OFB)) continue;
      OfbEntry e{};
      e.lat = lat;
      e.x = x;
      e.y = y;
      const size_t i = (size_t)y * nx + x;
      if (g->normal) {
        e.nsx = g->normal[i];
        e.nsy = g->normal[(size_t)nx * ny + i];
      } else {
        long long vx = 0, vy = 0;
        for (const C8& c : st) {
          const int s = s_e8(x + c.cx, y + c.cy);
          vx += (long long)c.k * s * c.cx;
          vy += (long long)c.k * s * c.cy;
        }
        const double dx = double(vx), dy = double(vy);
        const double m = std::sqrt(dx * dx + dy * dy);
        e.nsx = m > 0 ? dx / m : 0.0;
        e.nsy = m > 0 ? dy / m : 0.0;
      }
      const double th = g->theta_node ? g->theta_node[i] : p->theta;
      e.cos_t = std::cos(th);
      e.sin_t = std::sin(th);
      ofb.push_back(e);
    }
}

// Work units of the wall kernel: runs of consecutive outermost fluid entries of one lattice,
// at most gmax entries and kWallCap shared values (band + virtual nodes) per unit.  Each unit
// lists the fluid nodes whose rho^N its entries read (their fluid neighbours and the fluid
// neighbours of their solid neighbours, Eq. 28-29) and the solid neighbours (virtual nodes),
// and every entry gets the local index of the value at each of its 8 neighbours.  Nodes next
// to two units appear in both.  Each unit's band run starts on a multiple of 4 entries and the
// list ends with 4 padding entries: the kernel copies the runs in 16-byte pieces.
void build_wall_groups(const std::vector<LatGeom>& lats, const std::vector<OfbEntry>& ofb, int gmax,
                       std::vector<WallGroup>& groups, std::vector<int>& band, std::vector<WallSten>& virt,
                       std::vector<WallSten>& sten) {
  groups.clear();
  band.clear();
  virt.clear();
  sten.assign(ofb.size(), WallSten{});
  size_t i = 0;
  while (i < ofb.size()) {
    const int l = ofb[i].lat;
    const LatGeom& L = lats[l];
    const int nx = L.nx, ny = L.ny;
    const bool px = L.bcx == LBCG_BCX_PERIODIC, py = L.bcy == LBCG_BCY_PERIODIC;
    auto solid = [&](long long k) { return L.solid[k] != 0; };
    auto nbr = [&](long long k, int a) {
      const int x = int(k % nx), y = int(k / nx);
      return (long long)wrap_clamp(y + EYH[a], ny, py) * nx + wrap_clamp(x + EXH[a], nx, px);
    };
    std::unordered_map<long long, int> bmap, vmap;
    std::vector<long long> gb, gv, nb, nv;
    size_t j = i;
    while (j < ofb.size() && ofb[j].lat == l && j - i < (size_t)gmax) {
      nb.clear();
      nv.clear();
      auto want_band = [&](long long k) {
        if (!bmap.count(k) && std::find(nb.begin(), nb.end(), k) == nb.end()) nb.push_back(k);
      };
      const long long k0 = (long long)ofb[j].y * nx + ofb[j].x;
      for (int a = 1; a < 9; ++a) {
        const long long k = nbr(k0, a);
        if (!solid(k)) {
          want_band(k);
        } else if (!vmap.count(k) && std::find(nv.begin(), nv.end(), k) == nv.end()) {
          nv.push_back(k);
          for (int b = 1; b < 9; ++b) {
            const long long k2 = nbr(k, b);
            if (!solid(k2)) want_band(k2);
          }
        }
      }
      if (j > i && (gb.size() + gv.size() + nb.size() + nv.size() > (size_t)kWallCap ||
                    gv.size() + nv.size() > (size_t)kWallVirtCap))
        break;
      for (long long k : nb) {
        bmap[k] = int(gb.size());
        gb.push_back(k);
      }
      for (long long k : nv) {
        vmap[k] = int(gv.size());
        gv.push_back(k);
      }
      ++j;
    }
    // row-major order, so that neighbouring threads load neighbouring nodes
    std::sort(gb.begin(), gb.end());
    std::sort(gv.begin(), gv.end());
    for (size_t m = 0; m < gb.size(); ++m) bmap[gb[m]] = int(m);
    for (size_t m = 0; m < gv.size(); ++m) vmap[gv[m]] = int(m);
    while (band.size() % 4) band.push_back(0);   // each group's band run starts on 16 bytes
    WallGroup G{};
    G.lat = l;
    G.wall0 = int(i);
    G.nwall = int(j - i);
    G.band0 = int(band.size());
    G.nband = int(gb.size());
    G.virt0 = int(virt.size());
    G.nvirt = int(gv.size());
    for (long long k : gb) band.push_back(pop_node(int(k % nx), int(k / nx), L.pitch));
    for (long long k : gv) {
      WallSten q{};
      for (int b = 1; b < 9; ++b) {
        const long long k2 = nbr(k, b);
        q.i[b - 1] = solid(k2) ? kWallNone : uint16_t(bmap.at(k2));
      }
      virt.push_back(q);
    }
    for (size_t m = i; m < j; ++m) {
      const long long k0 = (long long)ofb[m].y * nx + ofb[m].x;
      for (int a = 1; a < 9; ++a) {
        const long long k = nbr(k0, a);
        sten[m].i[a - 1] = solid(k) ? uint16_t(G.nband + vmap.at(k)) : uint16_t(bmap.at(k));
      }
    }
    groups.push_back(G);
    i = j;
  }
  band.insert(band.end(), 4, 0);   // the last group's final 16-byte piece stays in bounds
}

}  // namespace lbcg
