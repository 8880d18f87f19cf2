// Host test of the wall-kernel work units (lbcg_geom.cpp), built and run by
// tests/test_wall_groups.py without a GPU.  For seeded random geometries of every boundary kind
// it checks that classify() lists exactly the fluid nodes with a solid D2Q9 neighbour, and
// that build_wall_groups() covers that list with groups within their caps whose every local
// index resolves to the node it stands for: a fluid neighbour to its band entry, a solid
// neighbour to a virtual entry whose own stencil lists exactly that node's fluid neighbours.
#include <cstdio>
#include <random>
#include <vector>

#include "lbcg_geom.h"

using namespace lbcg;

static int check(int nx, int ny, int bcx, int bcy, unsigned seed, int gmax, double fill) {
  std::mt19937 rng(seed);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  std::vector<uint8_t> solid((size_t)nx * ny, 0);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      bool s = (bcy == LBCG_BCY_CLOSED && (y == 0 || y == ny - 1)) ||
               (bcx == LBCG_BCX_CLOSED && (x == 0 || x == nx - 1));
      if (U(rng) < fill) s = true;
      solid[(size_t)y * nx + x] = s;
    }
  lbcg_geometry g{};
  g.nx = nx;
  g.ny = ny;
  g.solid = solid.data();
  g.bc_x = bcx;
  g.bc_y = bcy;
  lbcg_params p{};
  p.theta = 1.0;
  std::vector<uint8_t> fl, mk;
  std::vector<OfbEntry> ofb;
  classify(&g, &p, 0, fl, mk, ofb);
  const bool px = bcx == LBCG_BCX_PERIODIC, py = bcy == LBCG_BCY_PERIODIC;
  const int pitch = (nx + 31) / 32 * 32, segs = pitch / 32;
  auto S = [&](int x, int y) { return solid[(size_t)y * nx + x] != 0; };
  auto nb = [&](int x, int y, int a, int& xx, int& yy) {
    xx = wrap_clamp(x + EXH[a], nx, px);
    yy = wrap_clamp(y + EYH[a], ny, py);
  };
  int bad = 0;
  // the outermost fluid list, row-major
  size_t m = 0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (S(x, y)) continue;
      bool any = false;
      for (int a = 1; a < 9; ++a) {
        int xx, yy;
        nb(x, y, a, xx, yy);
        any |= S(xx, yy);
      }
      if (!any) continue;
      if (m >= ofb.size() || ofb[m].x != x || ofb[m].y != y) ++bad;
      ++m;
    }
  if (m != ofb.size()) ++bad;
  std::vector<LatGeom> lats{LatGeom{nx, ny, pitch, bcx, bcy, solid.data()}};
  std::vector<WallGroup> G;
  std::vector<int> band;
  std::vector<WallSten> virt, sten;
  build_wall_groups(lats, ofb, gmax, G, band, virt, sten);
  auto dec = [&](int off, int& x, int& y) {
    const int seg = off / kSeg;
    x = (seg % segs) * 32 + (off % kSeg) / 2;
    y = seg / segs;
  };
  size_t covered = 0;
  for (const WallGroup& q : G) {
    if (q.nwall < 1 || q.nwall > gmax || q.nband < 1 || q.nband + q.nvirt > kWallCap || q.nvirt > kWallVirtCap ||
        q.wall0 != (int)covered || q.band0 % 4 != 0 || q.band0 + 4 * ((q.nband + 3) / 4) > (int)band.size())
      ++bad;
    covered += q.nwall;
    for (int i = 0; i < q.nband; ++i) {
      int x, y;
      dec(band[q.band0 + i], x, y);
      if (x >= nx || y >= ny || S(x, y)) ++bad;
    }
    for (int w = q.wall0; w < q.wall0 + q.nwall; ++w)
      for (int a = 1; a < 9; ++a) {
        int xx, yy;
        nb(ofb[w].x, ofb[w].y, a, xx, yy);
        const int li = sten[w].i[a - 1];
        if (!S(xx, yy)) {
          int x, y;
          if (li >= q.nband) {
            ++bad;
            continue;
          }
          dec(band[q.band0 + li], x, y);
          if (x != xx || y != yy) ++bad;
          continue;
        }
        if (li < q.nband || li >= q.nband + q.nvirt) {
          ++bad;
          continue;
        }
        const WallSten& vs = virt[q.virt0 + li - q.nband];
        for (int b = 1; b < 9; ++b) {
          int x2, y2;
          nb(xx, yy, b, x2, y2);
          if (S(x2, y2)) {
            if (vs.i[b - 1] != kWallNone) ++bad;
            continue;
          }
          if (vs.i[b - 1] >= q.nband) {
            ++bad;
            continue;
          }
          int x, y;
          dec(band[q.band0 + vs.i[b - 1]], x, y);
          if (x != x2 || y != y2) ++bad;
        }
      }
  }
  if (covered != ofb.size()) ++bad;
  std::printf("%dx%d bc=(%d,%d) fill=%.2f gmax=%d: %zu outermost fluid, %zu groups, %zu band, %zu virtual: %s\n", nx,
              ny, bcx, bcy, fill, gmax, ofb.size(), G.size(), band.size(), virt.size(), bad ? "FAIL" : "ok");
  return bad;
}

int main() {
  int bad = 0;
  bad += check(1500, 130, LBCG_BCX_INOUT, LBCG_BCY_CLOSED, 1, 256, 0.0);    // displacement channel
  bad += check(200, 100, LBCG_BCX_PERIODIC, LBCG_BCY_CLOSED, 2, 64, 0.05);  // rough periodic channel
  bad += check(97, 61, LBCG_BCX_PERIODIC, LBCG_BCY_PERIODIC, 3, 32, 0.3);   // porous, doubly periodic
  bad += check(300, 41, LBCG_BCX_CLOSED, LBCG_BCY_CLOSED, 4, 256, 0.15);    // closed box
  bad += check(60, 30, LBCG_BCX_INOUT, LBCG_BCY_CLOSED, 5, 128, 0.45);      // dense obstacles
  bad += check(33, 7, LBCG_BCX_PERIODIC, LBCG_BCY_CLOSED, 6, 256, 0.9);     // nearly solid, ragged pitch
  bad += check(5, 5, LBCG_BCX_INOUT, LBCG_BCY_CLOSED, 7, 32, 0.2);          // tiny
  std::printf(bad ? "FAIL\n" : "ALL OK\n");
  return bad != 0;
}
