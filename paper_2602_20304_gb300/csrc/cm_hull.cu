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
// bounding-box diagonal) count as on or inside it.  The result is a
// triangulated surface: coplanar facets (a box face) come as several triangles
// with equal planes.  Output conventions: vertices in the order of their index
// in the input, edges the unique undirected edges of the triangles sorted by
// (smaller, larger) index, one plane (unit outward n, offset n . p) per
// triangle.
#include <algorithm>
#include <cmath>
#include <cstdint>
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

  // compact vertex list in input order, edges, planes
  std::vector<int> remap(n_points, -1);
  int nf = 0;
  for (const Face& f : F)
    if (f.alive) {
      ++nf;
      for (int k = 0; k < 3; ++k) remap[f.v[k]] = 0;
    }
  std::vector<float> verts;
  int nv = 0;
  for (int i = 0; i < n_points; ++i)
    if (remap[i] == 0) {
      remap[i] = nv++;
      verts.insert(verts.end(), {(float)P[i].x, (float)P[i].y, (float)P[i].z, 0.f});
    }
  std::vector<std::pair<int, int>> E;
  std::vector<float> planes;
  for (const Face& f : F) {
    if (!f.alive) continue;
    for (int k = 0; k < 3; ++k) {
      int a = remap[f.v[k]], b = remap[f.v[(k + 1) % 3]];
      E.emplace_back(std::min(a, b), std::max(a, b));
    }
    planes.insert(planes.end(), {(float)f.n.x, (float)f.n.y, (float)f.n.z, (float)f.o});
  }
  std::sort(E.begin(), E.end());
  E.erase(std::unique(E.begin(), E.end()), E.end());
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

extern "C" cm_status cm_get_geometry(const cm_context* cc, int32_t geom_id, cm_geometry_info* info, float* verts,
                                     int32_t* edges, float* planes) {
  cm_context* c = const_cast<cm_context*>(cc);
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
