// Automatic selection of the collision region (host code).
//
// The paper takes the collision-aware region x2 and its proxy surface from
// the user (Sec. 3.1, Fig. 2a) and names their automatic selection as future
// work (Sec. 5).  This selection works from the rest geometry alone: a
// boundary vertex can take part in contact when another boundary vertex lies
// within `radius` of it in space but more than `rings` edges away along the
// surface (two sides of a slit, two bodies across a gap: the lips, the
// slabs).  The proxy is every boundary triangle whose three vertices can take
// part in contact and are not all pinned; W is the selection of its
// vertices, so x2 is their free support.
//
// Precisely (the oracle's oracle/region.py states the same rule):
//  * boundary triangles: the faces (v0 v1 v2), (v0 v1 v3), (v0 v2 v3),
//    (v1 v2 v3) of the tets that belong to exactly one tet;
//  * surface graph: the edges of the boundary triangles;
//  * u, v close: ((dx dx + dy dy) + dz dz) < radius^2 in float64, evaluated
//    in this order without fused multiply-adds (the build compiles this file
//    with -ffp-contract=off);
//  * output triangles: sorted vertex triples in lexicographic order, proxy
//    vertices in increasing mesh order, triangles numbered by proxy vertex.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "../../include/fsim.h"

namespace {

struct Key3Hash {
  size_t operator()(const std::array<int32_t, 3>& k) const {
    uint64_t h = (uint64_t)(uint32_t)k[0] * 0x9E3779B97F4A7C15ULL;
    h ^= (uint64_t)(uint32_t)k[1] + 0x7F4A7C159E3779B9ULL + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k[2] + 0x2545F4914F6CDD1DULL + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

int select(const double* X, int64_t n, const int32_t* tets, int64_t T, const uint8_t* pinned,
           double radius, int rings, std::vector<std::array<int32_t, 3>>& faces_out,
           std::vector<int32_t>& verts_out) {
  // boundary triangles: faces met exactly once
  std::unordered_map<std::array<int32_t, 3>, int, Key3Hash> count;
  count.reserve((size_t)T * 4);
  static const int kFace[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  for (int64_t t = 0; t < T; ++t)
    for (const auto& f : kFace) {
      std::array<int32_t, 3> k = {tets[4 * t + f[0]], tets[4 * t + f[1]], tets[4 * t + f[2]]};
      std::sort(k.begin(), k.end());
      ++count[k];
    }
  std::vector<std::array<int32_t, 3>> bfaces;
  for (const auto& kv : count)
    if (kv.second == 1) bfaces.push_back(kv.first);
  std::sort(bfaces.begin(), bfaces.end());
  // surface graph over the boundary vertices
  std::vector<char> onb(n, 0);
  std::vector<std::vector<int32_t>> adj(n);
  for (const auto& f : bfaces)
    for (int a = 0; a < 3; ++a) {
      onb[f[a]] = 1;
      const int32_t u = f[a], v = f[(a + 1) % 3];
      adj[u].push_back(v);
      adj[v].push_back(u);
    }
  for (auto& l : adj) {
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
  }
  // uniform grid of cell size radius over the boundary vertices
  const double r2 = radius * radius;
  double lo[3] = {INFINITY, INFINITY, INFINITY};
  for (int64_t v = 0; v < n; ++v)
    if (onb[v])
      for (int d = 0; d < 3; ++d) lo[d] = std::min(lo[d], X[3 * v + d]);
  auto cell = [&](int64_t v, int d) { return (int64_t)std::floor((X[3 * v + d] - lo[d]) / radius); };
  struct CellHash {
    size_t operator()(const std::array<int64_t, 3>& c) const {
      return (size_t)(c[0] * 73856093LL ^ c[1] * 19349663LL ^ c[2] * 83492791LL);
    }
  };
  std::unordered_map<std::array<int64_t, 3>, std::vector<int32_t>, CellHash> grid;
  for (int64_t v = 0; v < n; ++v)
    if (onb[v]) grid[{cell(v, 0), cell(v, 1), cell(v, 2)}].push_back((int32_t)v);
  // contact-capable vertices: a close vertex outside the rings-neighbourhood
  std::vector<char> capable(n, 0);
  std::vector<int> depth(n, -1);
  std::vector<int32_t> frontier, next, touched;
  for (int64_t v = 0; v < n; ++v) {
    if (!onb[v]) continue;
    // vertices within `rings` surface edges of v (breadth-first, bounded)
    touched.clear();
    frontier.assign(1, (int32_t)v);
    depth[v] = 0;
    touched.push_back((int32_t)v);
    for (int k = 0; k < rings && !frontier.empty(); ++k) {
      next.clear();
      for (int32_t a : frontier)
        for (int32_t b : adj[a])
          if (depth[b] < 0) {
            depth[b] = k + 1;
            touched.push_back(b);
            next.push_back(b);
          }
      frontier.swap(next);
    }
    const int64_t cx = cell(v, 0), cy = cell(v, 1), cz = cell(v, 2);
    bool found = false;
    for (int64_t ix = cx - 1; ix <= cx + 1 && !found; ++ix)
      for (int64_t iy = cy - 1; iy <= cy + 1 && !found; ++iy)
        for (int64_t iz = cz - 1; iz <= cz + 1 && !found; ++iz) {
          auto it = grid.find({ix, iy, iz});
          if (it == grid.end()) continue;
          for (int32_t u : it->second) {
            if (u == v || depth[u] >= 0) continue;
            const double dx = X[3 * (int64_t)u] - X[3 * v];
            const double dy = X[3 * (int64_t)u + 1] - X[3 * v + 1];
            const double dz = X[3 * (int64_t)u + 2] - X[3 * v + 2];
            const double d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 < r2) { found = true; break; }
          }
        }
    capable[v] = found ? 1 : 0;
    for (int32_t a : touched) depth[a] = -1;
  }
  faces_out.clear();
  for (const auto& f : bfaces) {
    if (!capable[f[0]] || !capable[f[1]] || !capable[f[2]]) continue;
    if (pinned && pinned[f[0]] && pinned[f[1]] && pinned[f[2]]) continue;
    faces_out.push_back(f);
  }
  std::vector<char> inproxy(n, 0);
  for (const auto& f : faces_out)
    for (int a = 0; a < 3; ++a) inproxy[f[a]] = 1;
  verts_out.clear();
  for (int64_t v = 0; v < n; ++v)
    if (inproxy[v]) verts_out.push_back((int32_t)v);
  return FSIM_OK;
}

}  // namespace

extern "C" fsim_status fsim_select_region(const double* rest_xyz, int64_t n, const int32_t* tets,
                                          int64_t T, const uint8_t* pinned, double radius,
                                          int32_t rings, int32_t* proxy_tris, int64_t tris_cap,
                                          int64_t* n_tris, int32_t* proxy_verts, int64_t verts_cap,
                                          int64_t* n_verts) {
  if (!rest_xyz || !tets || n <= 0 || T <= 0 || n >= (1LL << 31) || !(radius > 0.0) ||
      !std::isfinite(radius) || rings < 0 || !n_tris || !n_verts)
    return FSIM_EINVAL;
  if ((tris_cap > 0 && !proxy_tris) || (verts_cap > 0 && !proxy_verts)) return FSIM_EINVAL;
  for (int64_t k = 0; k < 4 * T; ++k)
    if (tets[k] < 0 || tets[k] >= n) return FSIM_EINVAL;
  std::vector<std::array<int32_t, 3>> faces;
  std::vector<int32_t> verts;
  const int rc = select(rest_xyz, n, tets, T, pinned, radius, rings, faces, verts);
  if (rc != FSIM_OK) return rc;
  *n_tris = (int64_t)faces.size();
  *n_verts = (int64_t)verts.size();
  if (tris_cap <= 0 && verts_cap <= 0) return FSIM_OK;      // sizes only
  if ((int64_t)faces.size() > tris_cap || (int64_t)verts.size() > verts_cap) return FSIM_EINVAL;
  std::vector<int32_t> local(n, -1);
  for (size_t i = 0; i < verts.size(); ++i) {
    local[verts[i]] = (int32_t)i;
    proxy_verts[i] = verts[i];
  }
  for (size_t f = 0; f < faces.size(); ++f)
    for (int a = 0; a < 3; ++a) proxy_tris[3 * f + a] = local[faces[f][a]];
  return FSIM_OK;
}
