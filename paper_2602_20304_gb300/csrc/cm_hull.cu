// cm_hull.cu -- convex hull of a point set on the host, registered as a HULL geometry.
//
// A convex polyhedron enters the method in its two representations (Sec. IV-A):
// a mesh (vertices and edges, for the vertex-SDF and edge-edge candidates) and
// its face planes (for the smooth SDF, the LSE over planes of Sec. IV-B2).  This
// file builds both from a plain point set, so that a caller needs no hull code
// of its own, and offers the read-back of any registered geometry.
//
// Hull: incremental construction in double precision.  A tetrahedron of four
// affinely independent extreme points starts it; every further point, in input
// order, that lies more than eps above at least one face removes the faces it
// sees and is joined to the horizon (the edges between a seen and an unseen
// face), each new triangle keeping the horizon edge's orientation so that
// every face stays outward.  Points within eps of the hull (eps = 1e-9 x the
// bounding-box diagonal) count as on or inside it.  The triangulated surface is
// then checked to be a closed, consistently oriented sphere, and its triangles
// are merged into facets: neighbours whose vertices lie within eps of each
// other's plane (a box face built from two triangles) form one facet with one
// plane, so the LSE SDF counts each face once (a face split into m equal planes
// would add tau ln m to it).  Output conventions: vertices (the endpoints of
// facet edges) in the order of their index in the input, edges the facet
// boundaries sorted by (smaller, larger) index, one plane (unit outward n, offset
// n . p) per facet.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <unordered_set>
#include <vector>

#include "cm_context.h"

namespace {

using cm::rt::fail;

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct Face {
  int v[3];   // outward: (v1 - v0) x (v2 - v0) points away from the interior
  V3 n;       // unit outward normal
  double o;   // offset n . v0
  bool alive;
};

Face make_face(const std::vector<V3>& P, int a, int b, int c) {
  Face f{{a, b, c}, {0, 0, 0}, 0.0, true};
  V3 n = cross(sub(P[b], P[a]), sub(P[c], P[a]));
  double l = norm(n);
  if (l > 0) n = {n.x / l, n.y / l, n.z / l};
  f.n = n;
  f.o = dot(n, P[a]);
  return f;
}

inline uint64_t dkey(int a, int b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }

}  // namespace

extern "C" cm_status cm_create_hull_geometry(cm_context* c, const double* points, int32_t n_points,
                                            int32_t* geom_id) {
  if (!c || !points || !geom_id) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  if (n_points < 4 || n_points > CM_MAX_HULL_POINTS)
    return fail(CM_ERR_INVALID_ARG, "a hull takes 4..65536 points");
  std::vector<V3> P(n_points);
  V3 lo{1e300, 1e300, 1e300}, hi{-1e300, -1e300, -1e300};
  for (int i = 0; i < n_points; ++i) {
    P[i] = {points[3 * i], points[3 * i + 1], points[3 * i + 2]};
    if (!std::isfinite(P[i].x) || !std::isfinite(P[i].y) || !std::isfinite(P[i].z))
      return fail(CM_ERR_INVALID_ARG, "non-finite hull point");
    lo = {std::min(lo.x, P[i].x), std::min(lo.y, P[i].y), std::min(lo.z, P[i].z)};
    hi = {std::max(hi.x, P[i].x), std::max(hi.y, P[i].y), std::max(hi.z, P[i].z)};
  }
  const double diag = norm(sub(hi, lo));
  const double eps = 1e-9 * diag;
  if (!(diag > 0)) return fail(CM_ERR_INVALID_ARG, "hull points are all equal");

  // initial tetrahedron: the point of smallest x, the farthest from it, the farthest
  // from their line, the farthest from their plane
  int i0 = 0;
  for (int i = 1; i < n_points; ++i)
    if (P[i].x < P[i0].x) i0 = i;
  int i1 = -1;
  double best = 0;
  for (int i = 0; i < n_points; ++i) {
    double d = norm(sub(P[i], P[i0]));
    if (d > best) best = d, i1 = i;
  }
  if (i1 < 0 || best <= eps) return fail(CM_ERR_INVALID_ARG, "hull points are all equal");
  V3 u = sub(P[i1], P[i0]);
  int i2 = -1;
  best = 0;
  for (int i = 0; i < n_points; ++i) {
    double d = norm(cross(u, sub(P[i], P[i0]))) / norm(u);
    if (d > best) best = d, i2 = i;
  }
  if (i2 < 0 || best <= eps) return fail(CM_ERR_INVALID_ARG, "hull points are collinear");
  V3 n012 = cross(sub(P[i1], P[i0]), sub(P[i2], P[i0]));
  n012 = {n012.x / norm(n012), n012.y / norm(n012), n012.z / norm(n012)};
  int i3 = -1;
  best = 0;
  for (int i = 0; i < n_points; ++i) {
    double d = std::fabs(dot(n012, sub(P[i], P[i0])));
    if (d > best) best = d, i3 = i;
  }
  if (i3 < 0 || best <= eps) return fail(CM_ERR_INVALID_ARG, "hull points are coplanar");

  std::vector<Face> F;
  F.reserve(4096);
  {
    // orient the base triangle away from the fourth point
    bool below = dot(n012, sub(P[i3], P[i0])) < 0;
    int a = i0, b = below ? i1 : i2, cc = below ? i2 : i1;
    F.push_back(make_face(P, a, b, cc));
    F.push_back(make_face(P, a, i3, b));
    F.push_back(make_face(P, b, i3, cc));
    F.push_back(make_face(P, cc, i3, a));
  }
  std::vector<char> in_tet(n_points, 0);
  in_tet[i0] = in_tet[i1] = in_tet[i2] = in_tet[i3] = 1;

  std::vector<int> seen;
  std::unordered_set<uint64_t> seen_edges;
  size_t alive = F.size();
  for (int p = 0; p < n_points; ++p) {
    if (in_tet[p]) continue;
    seen.clear();
    for (int f = 0; f < (int)F.size(); ++f)
      if (F[f].alive && dot(F[f].n, P[p]) - F[f].o > eps) seen.push_back(f);
    if (seen.empty()) continue;  // inside or on the hull
    seen_edges.clear();
    for (int f : seen)
      for (int k = 0; k < 3; ++k) seen_edges.insert(dkey(F[f].v[k], F[f].v[(k + 1) % 3]));
    for (int f : seen) F[f].alive = false;
    alive -= seen.size();
    // horizon: a directed edge of a seen face whose reverse belongs to no seen face
    for (int f : seen)
      for (int k = 0; k < 3; ++k) {
        int a = F[f].v[k], b = F[f].v[(k + 1) % 3];
        if (!seen_edges.count(dkey(b, a))) {
          F.push_back(make_face(P, a, b, p));
          ++alive;
        }
      }
    if (F.size() > 2 * alive + 1024) {  // drop the dead faces once they outnumber the live ones
      std::vector<Face> G;
      G.reserve(2 * alive);
      for (const Face& f : F)
        if (f.alive) G.push_back(f);
      F.swap(G);
    }
  }

  std::vector<Face> T;  // the live triangles
  for (const Face& f : F)
    if (f.alive) T.push_back(f);
  const int nt = (int)T.size();
  // a closed, consistently oriented triangulated sphere: every directed edge once, its
  // reverse present, V - E + F = 2 (near-degenerate input can break this; refuse it)
  std::map<uint64_t, int> owner;  // directed edge -> triangle
  {
    bool ok = true;
    std::vector<char> used(n_points, 0);
    for (int t = 0; t < nt && ok; ++t)
      for (int k = 0; k < 3 && ok; ++k) {
        ok = owner.emplace(dkey(T[t].v[k], T[t].v[(k + 1) % 3]), t).second;
        used[T[t].v[k]] = 1;
      }
    for (const auto& kv : owner)
      if (ok && !owner.count(((kv.first & 0xffffffffull) << 32) | (kv.first >> 32))) ok = false;
    int nv0 = 0;
    for (char u : used) nv0 += u;
    if (!ok || nv0 - (int)owner.size() / 2 + nt != 2)
      return fail(CM_ERR_INVALID_ARG, "the point set is too close to degenerate for a closed hull");
  }
  // facets: triangles joined across an edge when each one's vertices lie within eps of
  // the other's plane and their normals point the same way (a flat face of the hull,
  // e.g. a box face split into two triangles, is one facet with one plane)
  std::vector<int> root(nt);
  for (int t = 0; t < nt; ++t) root[t] = t;
  auto find = [&](int t) {
    while (root[t] != t) t = root[t] = root[root[t]];
    return t;
  };
  auto coplanar = [&](const Face& a, const Face& b) {
    if (dot(a.n, b.n) <= 0.0) return false;
    for (int k = 0; k < 3; ++k)
      if (std::fabs(dot(a.n, P[b.v[k]]) - a.o) > eps || std::fabs(dot(b.n, P[a.v[k]]) - b.o) > eps) return false;
    return true;
  };
  for (const auto& kv : owner) {
    const int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffull);
    const int t0 = kv.second, t1 = owner[dkey(b, a)];
    if (a < b && coplanar(T[t0], T[t1])) root[find(t0)] = find(t1);
  }
  // the facets' boundaries: undirected edges whose two triangles lie in different facets
  std::vector<std::pair<int, int>> E;
  for (const auto& kv : owner) {
    const int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffull);
    if (a < b && find(kv.second) != find(owner[dkey(b, a)])) E.emplace_back(a, b);
  }
  // one plane per facet: the area-weighted mean normal of its triangles, offset through
  // their vertices' mean
  std::map<int, int> facet_of_root;
  std::vector<V3> fn;
  std::vector<double> fo, fcnt;
  for (int t = 0; t < nt; ++t) {
    const int r = find(t);
    auto it = facet_of_root.find(r);
    int fi;
    if (it == facet_of_root.end()) {
      fi = (int)fn.size();
      facet_of_root[r] = fi;
      fn.push_back({0, 0, 0});
      fo.push_back(0.0);
      fcnt.push_back(0.0);
    } else {
      fi = it->second;
    }
    const V3 area = cross(sub(P[T[t].v[1]], P[T[t].v[0]]), sub(P[T[t].v[2]], P[T[t].v[0]]));
    fn[fi] = {fn[fi].x + area.x, fn[fi].y + area.y, fn[fi].z + area.z};
  }
  for (int t = 0; t < nt; ++t) {
    const int fi = facet_of_root[find(t)];
    const double l = norm(fn[fi]);
    const V3 u = {fn[fi].x / l, fn[fi].y / l, fn[fi].z / l};
    for (int k = 0; k < 3; ++k) fo[fi] += dot(u, P[T[t].v[k]]);
    fcnt[fi] += 3.0;
  }
  const int nf = (int)fn.size();
  std::vector<float> planes;
  for (int fi = 0; fi < nf; ++fi) {
    const double l = norm(fn[fi]);
    planes.insert(planes.end(), {(float)(fn[fi].x / l), (float)(fn[fi].y / l), (float)(fn[fi].z / l),
                                 (float)(fo[fi] / fcnt[fi])});
  }
  // compact vertex list in input order: the endpoints of the remaining edges (a point in
  // the middle of a flat facet is not a vertex of the polyhedron)
  std::vector<int> remap(n_points, -1);
  for (auto& e : E) remap[e.first] = remap[e.second] = 0;
  std::vector<float> verts;
  int nv = 0;
  for (int i = 0; i < n_points; ++i)
    if (remap[i] == 0) {
      remap[i] = nv++;
      verts.insert(verts.end(), {(float)P[i].x, (float)P[i].y, (float)P[i].z, 0.f});
    }
  for (auto& e : E) {
    const int a = remap[e.first], b = remap[e.second];
    e = {std::min(a, b), std::max(a, b)};
  }
  std::sort(E.begin(), E.end());
  if (nv - (int)E.size() + nf != 2)
    return fail(CM_ERR_INVALID_ARG, "the point set is too close to degenerate for a closed hull");
  if (nv > CM_MAX_VERTS || (int)E.size() > CM_MAX_EDGES || nf > CM_MAX_PLANES)
    return fail(CM_ERR_INVALID_ARG, "the hull exceeds the geometry limits (256 vertices, 768 edges, 512 planes)");
  std::vector<int32_t> edges;
  for (auto& e : E) edges.insert(edges.end(), {e.first, e.second});

  cm_geometry_desc d{};
  d.kind = CM_HULL;
  d.dims[0] = d.dims[1] = d.dims[2] = 1.f;
  d.n_verts = nv;
  d.verts = verts.data();
  d.n_edges = (int32_t)E.size();
  d.edges = edges.data();
  d.n_planes = nf;
  d.planes = planes.data();
  return cm_create_geometry(c, &d, geom_id);
}

namespace {

// Unit template meshes of the analytic primitives.  A row (u_x, u_y, u_z, s) maps to a
// body-frame vertex from the dims in use: BOX / ELLIPSOID (d0 u_x, d1 u_y, d2 u_z),
// CYLINDER (r u_x, r u_y, h u_z), CAPSULE (r u_x, r u_y, r u_z + s h).  Every vertex lies
// on the exact surface of its primitive.
struct Mesh {
  std::vector<float> v;        // rows of 4
  std::vector<int32_t> e;      // pairs
  int nv() const { return (int)v.size() / 4; }
  void vert(double x, double y, double z, double s) {
    v.insert(v.end(), {(float)x, (float)y, (float)z, (float)s});
  }
  void edge(int a, int b) { e.insert(e.end(), {std::min(a, b), std::max(a, b)}); }
};

constexpr double kPi = 3.14159265358979323846;

// box: the 8 corners of [-1, 1]^3 and the 12 edges between corners that differ in one axis
void box_mesh(Mesh& m) {
  for (int i = 0; i < 8; ++i) m.vert(i & 4 ? 1 : -1, i & 2 ? 1 : -1, i & 1 ? 1 : -1, 0);
  for (int i = 0; i < 8; ++i)
    for (int j = i + 1; j < 8; ++j) {
      int d = i ^ j;
      if (d == 1 || d == 2 || d == 4) m.edge(i, j);
    }
}

// cylinder: n points on each rim (z = -1, +1), the rim polygons and n vertical edges
void cylinder_mesh(Mesh& m, int n) {
  for (int r = 0; r < 2; ++r)
    for (int i = 0; i < n; ++i) m.vert(std::cos(2 * kPi * i / n), std::sin(2 * kPi * i / n), r ? 1 : -1, 0);
  for (int r = 0; r < 2; ++r)
    for (int i = 0; i < n; ++i) m.edge(r * n + i, r * n + (i + 1) % n);
  for (int i = 0; i < n; ++i) m.edge(i, n + i);
}

// capsule: per cap (s = -1, +1) rings of n points at latitudes 0 and pi/4 and a pole; ring
// polygons, meridian edges ring to ring and ring to pole, and the n edges between the
// two equators (the cylinder part)
void capsule_mesh(Mesh& m, int n) {
  const double lats[2] = {0.0, kPi / 4};
  int ring[2][2];
  for (int c = 0; c < 2; ++c) {
    double s = c ? 1.0 : -1.0;
    for (int l = 0; l < 2; ++l) {
      ring[c][l] = m.nv();
      for (int i = 0; i < n; ++i) {
        double t = 2 * kPi * i / n;
        m.vert(std::cos(lats[l]) * std::cos(t), std::cos(lats[l]) * std::sin(t), s * std::sin(lats[l]), s);
      }
    }
  }
  int pole[2];
  for (int c = 0; c < 2; ++c) {
    pole[c] = m.nv();
    m.vert(0, 0, c ? 1 : -1, c ? 1 : -1);
  }
  for (int c = 0; c < 2; ++c)
    for (int l = 0; l < 2; ++l)
      for (int i = 0; i < n; ++i) m.edge(ring[c][l] + i, ring[c][l] + (i + 1) % n);
  for (int c = 0; c < 2; ++c) {
    for (int i = 0; i < n; ++i) m.edge(ring[c][0] + i, ring[c][1] + i);
    for (int i = 0; i < n; ++i) m.edge(ring[c][1] + i, pole[c]);
  }
  for (int i = 0; i < n; ++i) m.edge(ring[0][0] + i, ring[1][0] + i);
}

// ellipsoid: the icosahedron on the unit sphere, each triangle split in four `level`
// times with the new vertices pushed onto the sphere; the edges of the triangles
void icosphere_mesh(Mesh& m, int level) {
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  std::vector<V3> P;
  // the 12 icosahedron vertices are the cyclic permutations of (0, +-1, +-g)
  for (int perm = 0; perm < 3; ++perm)
    for (int a = -1; a <= 1; a += 2)
      for (int b = -1; b <= 1; b += 2) {
        double q[3];
        q[perm] = 0.0, q[(perm + 1) % 3] = a, q[(perm + 2) % 3] = b * g;
        double l = std::sqrt(1.0 + g * g);
        P.push_back({q[0] / l, q[1] / l, q[2] / l});
      }
  // the 20 faces: triples of mutually adjacent vertices (edge length 2 before scaling)
  const double edge2 = 4.0 / (1.0 + g * g);
  auto adj = [&](int i, int j) { return std::fabs(dot(sub(P[i], P[j]), sub(P[i], P[j])) - edge2) < 1e-9; };
  std::vector<std::array<int, 3>> F;
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j)
      for (int k = j + 1; k < 12; ++k)
        if (adj(i, j) && adj(j, k) && adj(i, k)) F.push_back({i, j, k});
  for (int it = 0; it < level; ++it) {
    std::map<std::pair<int, int>, int> mid;
    auto midpoint = [&](int a, int b) {
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto f = mid.find(key);
      if (f != mid.end()) return f->second;
      V3 s{P[a].x + P[b].x, P[a].y + P[b].y, P[a].z + P[b].z};
      double l = norm(s);
      P.push_back({s.x / l, s.y / l, s.z / l});
      return mid[key] = (int)P.size() - 1;
    };
    std::vector<std::array<int, 3>> G;
    for (auto& f : F) {
      int ab = midpoint(f[0], f[1]), bc = midpoint(f[1], f[2]), ca = midpoint(f[2], f[0]);
      G.push_back({f[0], ab, ca});
      G.push_back({f[1], bc, ab});
      G.push_back({f[2], ca, bc});
      G.push_back({ab, bc, ca});
    }
    F.swap(G);
  }
  for (const V3& p : P) m.vert(p.x, p.y, p.z, 0);
  std::vector<std::pair<int, int>> E;
  for (auto& f : F)
    for (int k = 0; k < 3; ++k) E.emplace_back(std::min(f[k], f[(k + 1) % 3]), std::max(f[k], f[(k + 1) % 3]));
  std::sort(E.begin(), E.end());
  E.erase(std::unique(E.begin(), E.end()), E.end());
  for (auto& e : E) m.edge(e.first, e.second);
}

}  // namespace

extern "C" cm_status cm_create_primitive_geometry(cm_context* c, int32_t kind, const float* dims, int32_t tess,
                                                 int32_t* geom_id) {
  if (!c || !dims || !geom_id) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  Mesh m;
  switch (kind) {
    case CM_BOX:
      box_mesh(m);
      break;
    case CM_CYLINDER:
      if (tess < 3 || tess > 128) return fail(CM_ERR_INVALID_ARG, "cylinder tess (points per rim) must be in 3..128");
      cylinder_mesh(m, tess);
      break;
    case CM_CAPSULE:
      if (tess < 3 || tess > 63) return fail(CM_ERR_INVALID_ARG, "capsule tess (points per ring) must be in 3..63");
      capsule_mesh(m, tess);
      break;
    case CM_ELLIPSOID:
      if (tess < 0 || tess > 2) return fail(CM_ERR_INVALID_ARG, "ellipsoid tess (icosphere level) must be in 0..2");
      icosphere_mesh(m, tess);
      break;
    default:
      return fail(CM_ERR_INVALID_ARG, "cm_create_primitive_geometry takes BOX, CAPSULE, CYLINDER or ELLIPSOID");
  }
  cm_geometry_desc d{};
  d.kind = kind;
  for (int i = 0; i < 3; ++i) d.dims[i] = dims[i];
  d.n_verts = m.nv();
  d.verts = m.v.data();
  d.n_edges = (int32_t)m.e.size() / 2;
  d.edges = m.e.data();
  d.n_planes = 0;
  d.planes = nullptr;
  return cm_create_geometry(c, &d, geom_id);
}

extern "C" cm_status cm_get_geometry(const cm_context* c, int32_t geom_id, cm_geometry_info* info, float* verts,
                                     int32_t* edges, float* planes) {
  if (!c || !info) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  if (geom_id < 0 || geom_id >= (int32_t)c->hdr.size() || c->hdr[geom_id].n_verts <= 0)
    return fail(CM_ERR_INVALID_ARG, "unknown or destroyed geometry id");
  const cm::GeomHeader& h = c->hdr[geom_id];
  info->kind = h.kind;
  for (int i = 0; i < 3; ++i) info->dims[i] = h.dims[i];
  info->n_verts = h.n_verts;
  info->n_edges = h.n_edges;
  info->n_planes = h.kind == CM_HULL ? h.n_planes : 0;
  if (verts)
    for (int i = 0; i < h.n_verts; ++i) {
      const float4& v = c->verts[h.v_off + i];
      verts[4 * i] = v.x, verts[4 * i + 1] = v.y, verts[4 * i + 2] = v.z, verts[4 * i + 3] = v.w;
    }
  if (edges)
    for (int i = 0; i < h.n_edges; ++i) {
      uint32_t e = c->edges[h.e_off + i];
      edges[2 * i] = (int32_t)(e & 0xffffu);
      edges[2 * i + 1] = (int32_t)(e >> 16);
    }
  if (planes && h.kind == CM_HULL)
    for (int i = 0; i < h.n_planes; ++i) {
      const float4& p = c->planes[h.p_off + i];
      planes[4 * i] = p.x, planes[4 * i + 1] = p.y, planes[4 * i + 2] = p.z, planes[4 * i + 3] = p.w;
    }
  return CM_OK;
}
