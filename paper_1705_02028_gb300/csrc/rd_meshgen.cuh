// rd_meshgen.cuh -- per-element steps of the parallel Delaunay refinement of a
// periodic domain (Sec. 2.3-2.4 and Sec. 4.1): quality test, point location by
// walking, insertion cavities with priority locks, three-way splits and
// parallel edge flips.  Every function acts on one element (triangle,
// candidate vertex or edge) and is compiled for the device (one thread per
// element) and for the host (the same steps in a serial loop, used to check
// the index logic without a GPU).
//
// Geometry is exact: vertex coordinates are integers on a grid of 2^30 units
// per period of x (the period of y is rounded to the same unit), so Orient2D
// and InCircle2D (Eqs. eqOrient, eqInCircle) are evaluated exactly in 64- and
// 128-bit integer arithmetic instead of the adaptive floating-point predicates
// the paper uses.  Points closer than one unit are never distinguished, which
// is 1e-9 of the domain.
//
// Periodicity: a triangle stores, for each corner, the image shift (sx, sy) in
// periods that places the vertex next to the other two corners ("frame" of the
// triangle).  Shifts are normalised to {0, 1} per triangle.  Moving across an
// edge maps a point from one triangle's frame to the neighbour's by the shift
// difference of a shared vertex.
#pragma once

#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define MG_HD __host__ __device__ __forceinline__
#else
#define MG_HD inline
#endif

namespace rd {
namespace mg {

constexpr int64_t UNIT_BITS = 30;
constexpr int MAX_WALK = 256;    // point-location steps before a candidate is deferred
constexpr int MAX_CAVITY = 48;   // triangles in a cavity (plus its 1-ring) before deferral

// Device-side mesh being refined (capacities fixed at creation).
struct Mesh {
  int32_t* vx;      // [cap_v] x in units, 0 <= x < Px
  int32_t* vy;      // [cap_v]
  int32_t* tv;      // [cap_t][3] corners (counter-clockwise)
  int8_t* ts;       // [cap_t][3][2] image shift of each corner, in {0, 1}
  int32_t* tn;      // [cap_t][3] neighbour across the edge opposite each corner
  int8_t* tc;       // [cap_t][3] that edge's corner index in the neighbour
  uint8_t* dirty;   // [cap_t] 1: triangle rewritten since its edges were last found Delaunay (nullable)
  int64_t Px, Py;   // periods in units
};

struct P64 {
  int64_t x, y;
};

MG_HD P64 corner(const Mesh& m, int32_t t, int k) {
  const int32_t v = m.tv[3 * (size_t)t + k];
  return P64{(int64_t)m.vx[v] + m.Px * m.ts[6 * (size_t)t + 2 * k], (int64_t)m.vy[v] + m.Py * m.ts[6 * (size_t)t + 2 * k + 1]};
}

// Orient2D(a, b, c) > 0 when (a, b, c) turn counter-clockwise (Eq. eqOrient), exact.
MG_HD int orient(P64 a, P64 b, P64 c) {
  const __int128 d = (__int128)(a.x - c.x) * (b.y - c.y) - (__int128)(a.y - c.y) * (b.x - c.x);
  return d > 0 ? 1 : (d < 0 ? -1 : 0);
}

// InCircle2D(a, b, c, d) > 0 when d lies inside the circle through the
// counter-clockwise a, b, c (Eq. eqInCircle), exact for coordinate differences
// below 2^31 (every term stays below 2^126).
MG_HD int incircle(P64 a, P64 b, P64 c, P64 d) {
  const int64_t adx = a.x - d.x, ady = a.y - d.y, bdx = b.x - d.x, bdy = b.y - d.y, cdx = c.x - d.x, cdy = c.y - d.y;
  const __int128 al = (__int128)adx * adx + (__int128)ady * ady;
  const __int128 bl = (__int128)bdx * bdx + (__int128)bdy * bdy;
  const __int128 cl = (__int128)cdx * cdx + (__int128)cdy * cdy;
  const __int128 det = al * ((__int128)bdx * cdy - (__int128)cdx * bdy) - bl * ((__int128)adx * cdy - (__int128)cdx * ady) +
                       cl * ((__int128)adx * bdy - (__int128)bdx * ady);
  return det > 0 ? 1 : (det < 0 ? -1 : 0);
}

// Shift that maps a point in the frame of triangle t into the frame of its
// neighbour across the edge opposite corner k.
MG_HD P64 frame_offset(const Mesh& m, int32_t t, int k) {
  const int32_t n = m.tn[3 * (size_t)t + k];
  const int j = m.tc[3 * (size_t)t + k];
  // the edge's start vertex (corner k+1 of t) is corner j+2 of n
  const int kt = (k + 1) % 3, kn = (j + 2) % 3;
  return P64{m.Px * (m.ts[6 * (size_t)n + 2 * kn] - m.ts[6 * (size_t)t + 2 * kt]),
             m.Py * (m.ts[6 * (size_t)n + 2 * kn + 1] - m.ts[6 * (size_t)t + 2 * kt + 1])};
}

// ---------------------------------------------------------------------------
// quality test (Sec. 2.4.1): circumradius r = l_a l_b l_c / (2 Orient2D) and
// beta = r / shortest edge; a triangle with r > R or beta > B gets a vertex at
// its circumcentre, returned here in the triangle's frame (rounded to the grid).
// ---------------------------------------------------------------------------
MG_HD bool quality_test(const Mesh& m, int32_t t, double R_units, double B, P64& centre) {
  const P64 a = corner(m, t, 0), b = corner(m, t, 1), c = corner(m, t, 2);
  const double bx = (double)(b.x - a.x), by = (double)(b.y - a.y), cx = (double)(c.x - a.x), cy = (double)(c.y - a.y);
  const double ex = (double)(b.x - c.x), ey = (double)(b.y - c.y);
  const double la2 = ex * ex + ey * ey;
  const double lb2 = cx * cx + cy * cy, lc2 = bx * bx + by * by;
  const double D = 2.0 * (bx * cy - by * cx);  // twice Orient2D, > 0 for a valid triangle
  if (!(D > 0.0)) return false;
  const double r = sqrt(la2 * lb2 * lc2) / D;
  double lmin2 = la2 < lb2 ? la2 : lb2;
  lmin2 = lc2 < lmin2 ? lc2 : lmin2;
  const bool bad = r > R_units || r * r > B * B * lmin2;
  if (!bad) return false;
  // circumcentre relative to a
  const double ux = (cy * lc2 - by * lb2) / D, uy = (bx * lb2 - cx * lc2) / D;
  centre.x = a.x + (int64_t)llround(ux);
  centre.y = a.y + (int64_t)llround(uy);
  return true;
}

// Point location by walking (Sec. 2.4.2): start in t, cross an edge that has p
// on its outer side, mapping p into each new frame.  Returns the containing
// triangle with p in its frame and sets `edge` to the corner opposite the edge
// p lies on (-1 if p is strictly inside); -1 if p falls on a vertex, -2 if the
// walk did not end within MAX_WALK steps (the candidate is deferred).
MG_HD int32_t locate(const Mesh& m, int32_t t, P64& p, int& edge) {
  int from = -1;  // edge we entered through (tested last)
  edge = -1;
  for (int step = 0; step < MAX_WALK; ++step) {
    int out = -1, zeros = 0, zk = -1;
    for (int q = 0; q < 3; ++q) {
      const int k = (from < 0 ? q : (from + 1 + q) % 3);
      const int o = orient(corner(m, t, (k + 1) % 3), corner(m, t, (k + 2) % 3), p);
      if (o < 0) {
        out = k;
        break;
      }
      if (o == 0) {
        ++zeros;
        zk = k;
      }
    }
    if (out < 0) {
      if (zeros > 1) return -1;
      edge = zk;
      return t;
    }
    const P64 off = frame_offset(m, t, out);
    p.x += off.x;
    p.y += off.y;
    const int32_t n = m.tn[3 * (size_t)t + out];
    from = m.tc[3 * (size_t)t + out];
    t = n;
  }
  return -2;
}

// Insertion cavity (Sec. 4.1.1): the triangles whose circumcircle contains p,
// grown from the containing triangle across edges, plus the containing
// triangle's three neighbours (whose adjacency the split rewrites).  Fills
// list[0..n) and returns n, or -1 if more than MAX_CAVITY triangles.
MG_HD int cavity(const Mesh& m, int32_t t0, P64 p0, int edge, int32_t* list) {
  int n = 0;
  P64 pts[MAX_CAVITY];
  list[n] = t0;
  pts[n++] = p0;
  // the triangles the split rewrites and their neighbours: t0's 1-ring, and for a
  // point on an edge also the 1-ring of the triangle across it
  for (int side = 0; side < (edge >= 0 ? 2 : 1); ++side) {
    const int32_t tt = side == 0 ? t0 : m.tn[3 * (size_t)t0 + edge];
    P64 pt = p0;
    if (side == 1) {
      const P64 off = frame_offset(m, t0, edge);
      pt = P64{p0.x + off.x, p0.y + off.y};
    }
    for (int k = 0; k < 3; ++k) {
      const int32_t nb = m.tn[3 * (size_t)tt + k];
      bool dup = false;
      for (int q = 0; q < n; ++q) dup = dup || list[q] == nb;
      if (dup) continue;
      const P64 off = frame_offset(m, tt, k);
      list[n] = nb;
      pts[n++] = P64{pt.x + off.x, pt.y + off.y};
    }
  }
  // breadth-first growth through triangles whose circumcircle contains p
  for (int h = 0; h < n; ++h) {
    const int32_t t = list[h];
    if (h > 0 && incircle(corner(m, t, 0), corner(m, t, 1), corner(m, t, 2), pts[h]) <= 0) continue;
    for (int k = 0; k < 3; ++k) {
      const int32_t nb = m.tn[3 * (size_t)t + k];
      bool dup = false;
      for (int q = 0; q < n; ++q) dup = dup || list[q] == nb;
      if (dup) continue;
      const P64 off = frame_offset(m, t, k);
      const P64 pn{pts[h].x + off.x, pts[h].y + off.y};
      if (incircle(corner(m, nb, 0), corner(m, nb, 1), corner(m, nb, 2), pn) <= 0) continue;
      if (n >= MAX_CAVITY) return -1;
      list[n] = nb;
      pts[n++] = pn;
    }
  }
  return n;
}

MG_HD void normalise_shifts(int8_t* s) {
  int mx = s[0], my = s[1];
  for (int k = 1; k < 3; ++k) {
    mx = s[2 * k] < mx ? s[2 * k] : mx;
    my = s[2 * k + 1] < my ? s[2 * k + 1] : my;
  }
  for (int k = 0; k < 3; ++k) {
    s[2 * k] = (int8_t)(s[2 * k] - mx);
    s[2 * k + 1] = (int8_t)(s[2 * k + 1] - my);
  }
}

MG_HD void write_triangle(Mesh& m, int32_t t, const int32_t v[3], const int8_t s[6], const int32_t nb[3],
                          const int8_t nc[3]) {
  int8_t sh[6] = {s[0], s[1], s[2], s[3], s[4], s[5]};
  normalise_shifts(sh);
  if (m.dirty) m.dirty[t] = 1;
  for (int k = 0; k < 3; ++k) {
    m.tv[3 * (size_t)t + k] = v[k];
    m.tn[3 * (size_t)t + k] = nb[k];
    m.tc[3 * (size_t)t + k] = nc[k];
    m.ts[6 * (size_t)t + 2 * k] = sh[2 * k];
    m.ts[6 * (size_t)t + 2 * k + 1] = sh[2 * k + 1];
  }
}

// Three-way split of t by the new vertex pv (coordinates p in t's frame):
// T_k = (v_{k+1}, v_{k+2}, pv) for k = 0, 1, 2 with ids (t, t1, t2).  The outer
// neighbour across the old edge opposite corner k now faces T_k's corner 2.
MG_HD void split3(Mesh& m, int32_t t, int32_t pv, P64 p, int32_t t1, int32_t t2) {
  int32_t v[3], nb[3];
  int8_t nc[3], s[6];
  for (int k = 0; k < 3; ++k) {
    v[k] = m.tv[3 * (size_t)t + k];
    nb[k] = m.tn[3 * (size_t)t + k];
    nc[k] = m.tc[3 * (size_t)t + k];
    s[2 * k] = m.ts[6 * (size_t)t + 2 * k];
    s[2 * k + 1] = m.ts[6 * (size_t)t + 2 * k + 1];
  }
  // stored (wrapped) coordinates of the new vertex and its shift in t's frame
  int64_t wx = p.x % m.Px, wy = p.y % m.Py;
  if (wx < 0) wx += m.Px;
  if (wy < 0) wy += m.Py;
  m.vx[pv] = (int32_t)wx;
  m.vy[pv] = (int32_t)wy;
  const int8_t psx = (int8_t)((p.x - wx) / m.Px), psy = (int8_t)((p.y - wy) / m.Py);
  const int32_t id[3] = {t, t1, t2};
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    const int32_t tv3[3] = {v[a], v[b], pv};
    const int8_t ts3[6] = {s[2 * a], s[2 * a + 1], s[2 * b], s[2 * b + 1], psx, psy};
    // corner 0 (v_a) faces (v_b, p): shared with T_{k+1}'s corner 1; corner 1 faces (p, v_a):
    // shared with T_{k-1}'s corner 0; corner 2 faces the old edge.
    const int32_t nb3[3] = {id[(k + 1) % 3], id[(k + 2) % 3], nb[k]};
    const int8_t nc3[3] = {1, 0, nc[k]};
    write_triangle(m, id[k], tv3, ts3, nb3, nc3);
  }
  for (int k = 0; k < 3; ++k) {
    m.tn[3 * (size_t)nb[k] + nc[k]] = id[k];
    m.tc[3 * (size_t)nb[k] + nc[k]] = 2;
  }
}

// Split of the two triangles on either side of the edge opposite corner k of t
// by the new vertex pv lying on that edge (p in t's frame): with t = (c, a, b)
// and n = (d, b, a), the four triangles (c, a, p) [id t], (c, p, b) [t1],
// (d, b, p) [id n] and (d, p, a) [t2].
MG_HD void split4(Mesh& m, int32_t t, int k, int32_t pv, P64 p, int32_t t1, int32_t t2) {
  const int32_t n = m.tn[3 * (size_t)t + k];
  const int j = m.tc[3 * (size_t)t + k];
  const int ka = (k + 1) % 3, kb = (k + 2) % 3, jb = (j + 1) % 3, ja = (j + 2) % 3;
  const P64 off = frame_offset(m, t, k);
  const int32_t c = m.tv[3 * (size_t)t + k], a = m.tv[3 * (size_t)t + ka], b = m.tv[3 * (size_t)t + kb];
  const int32_t d = m.tv[3 * (size_t)n + j];
  const int8_t* st = m.ts + 6 * (size_t)t;
  const int8_t* sn = m.ts + 6 * (size_t)n;
  const int8_t dsx = (int8_t)(sn[2 * j] - off.x / m.Px), dsy = (int8_t)(sn[2 * j + 1] - off.y / m.Py);
  const int32_t o_ca = m.tn[3 * (size_t)t + kb], o_bc = m.tn[3 * (size_t)t + ka];
  const int8_t c_ca = m.tc[3 * (size_t)t + kb], c_bc = m.tc[3 * (size_t)t + ka];
  const int32_t o_db = m.tn[3 * (size_t)n + ja], o_ad = m.tn[3 * (size_t)n + jb];
  const int8_t c_db = m.tc[3 * (size_t)n + ja], c_ad = m.tc[3 * (size_t)n + jb];
  const int8_t s_c[2] = {st[2 * k], st[2 * k + 1]}, s_a[2] = {st[2 * ka], st[2 * ka + 1]},
               s_b[2] = {st[2 * kb], st[2 * kb + 1]};
  int64_t wx = p.x % m.Px, wy = p.y % m.Py;
  if (wx < 0) wx += m.Px;
  if (wy < 0) wy += m.Py;
  m.vx[pv] = (int32_t)wx;
  m.vy[pv] = (int32_t)wy;
  const int8_t psx = (int8_t)((p.x - wx) / m.Px), psy = (int8_t)((p.y - wy) / m.Py);
  {  // (c, a, p): c faces (a, p) -> (d, p, a) corner 0; a faces (p, c) -> (c, p, b) corner 2; p faces (c, a)
    const int32_t v[3] = {c, a, pv};
    const int8_t s[6] = {s_c[0], s_c[1], s_a[0], s_a[1], psx, psy};
    const int32_t nb[3] = {t2, t1, o_ca};
    const int8_t nc[3] = {0, 2, c_ca};
    write_triangle(m, t, v, s, nb, nc);
  }
  {  // (c, p, b): c faces (p, b) -> (d, b, p) corner 0; p faces (b, c); b faces (c, p) -> (c, a, p) corner 1
    const int32_t v[3] = {c, pv, b};
    const int8_t s[6] = {s_c[0], s_c[1], psx, psy, s_b[0], s_b[1]};
    const int32_t nb[3] = {n, o_bc, t};
    const int8_t nc[3] = {0, c_bc, 1};
    write_triangle(m, t1, v, s, nb, nc);
  }
  {  // (d, b, p): d faces (b, p) -> (c, p, b) corner 0; b faces (p, d) -> (d, p, a) corner 2; p faces (d, b)
    const int32_t v[3] = {d, b, pv};
    const int8_t s[6] = {dsx, dsy, s_b[0], s_b[1], psx, psy};
    const int32_t nb[3] = {t1, t2, o_db};
    const int8_t nc[3] = {0, 2, c_db};
    write_triangle(m, n, v, s, nb, nc);
  }
  {  // (d, p, a): d faces (p, a) -> (c, a, p) corner 0; p faces (a, d); a faces (d, p) -> (d, b, p) corner 1
    const int32_t v[3] = {d, pv, a};
    const int8_t s[6] = {dsx, dsy, psx, psy, s_a[0], s_a[1]};
    const int32_t nb[3] = {t, o_ad, n};
    const int8_t nc[3] = {0, c_ad, 1};
    write_triangle(m, t2, v, s, nb, nc);
  }
  m.tn[3 * (size_t)o_ca + c_ca] = t;
  m.tc[3 * (size_t)o_ca + c_ca] = 2;
  m.tn[3 * (size_t)o_bc + c_bc] = t1;
  m.tc[3 * (size_t)o_bc + c_bc] = 1;
  m.tn[3 * (size_t)o_db + c_db] = n;
  m.tc[3 * (size_t)o_db + c_db] = 2;
  m.tn[3 * (size_t)o_ad + c_ad] = t2;
  m.tc[3 * (size_t)o_ad + c_ad] = 1;
}

// Is the edge opposite corner k of t (shared with n = tn[t][k]) not locally
// Delaunay (Sec. 2.4.6)?  The far vertex of n is tested against t's
// circumcircle.  An edge can only turn non-Delaunay when one of its two
// triangles is rewritten, so the flip rounds test the edges of rewritten
// ("dirty") triangles only -- from either side, as Sec. 4.1.1 restricts the
// checks to edges of the cavities and new edges.
MG_HD bool edge_bad(const Mesh& m, int32_t t, int k) {
  const int32_t n = m.tn[3 * (size_t)t + k];
  const int j = m.tc[3 * (size_t)t + k];
  const P64 off = frame_offset(m, t, k);
  P64 d = corner(m, n, j);
  d.x -= off.x;
  d.y -= off.y;
  return incircle(corner(m, t, 0), corner(m, t, 1), corner(m, t, 2), d) > 0;
}

// Flip of the edge opposite corner k of t (Fig. figEdgeFlip): t = (c, a, b) with
// c at corner k, n = (d, b, a) with d at corner j; new t' = (c, a, d), n' = (d, b, c).
MG_HD void flip(Mesh& m, int32_t t, int k) {
  const int32_t n = m.tn[3 * (size_t)t + k];
  const int j = m.tc[3 * (size_t)t + k];
  const int ka = (k + 1) % 3, kb = (k + 2) % 3, jb = (j + 1) % 3, ja = (j + 2) % 3;
  const P64 off = frame_offset(m, t, k);
  // positions in t's frame as shifts relative to t's stored corners
  const int32_t c = m.tv[3 * (size_t)t + k], a = m.tv[3 * (size_t)t + ka], b = m.tv[3 * (size_t)t + kb];
  const int32_t d = m.tv[3 * (size_t)n + j];
  const int8_t* st = m.ts + 6 * (size_t)t;
  const int8_t* sn = m.ts + 6 * (size_t)n;
  const int8_t dsx = (int8_t)(sn[2 * j] - off.x / m.Px), dsy = (int8_t)(sn[2 * j + 1] - off.y / m.Py);
  // outer neighbours
  const int32_t n_ad = m.tn[3 * (size_t)n + jb], n_bd = m.tn[3 * (size_t)n + ja];
  const int8_t c_ad = m.tc[3 * (size_t)n + jb], c_bd = m.tc[3 * (size_t)n + ja];
  const int32_t n_ca = m.tn[3 * (size_t)t + kb], n_bc = m.tn[3 * (size_t)t + ka];
  const int8_t c_ca = m.tc[3 * (size_t)t + kb], c_bc = m.tc[3 * (size_t)t + ka];
  const int8_t s_c[2] = {st[2 * k], st[2 * k + 1]}, s_a[2] = {st[2 * ka], st[2 * ka + 1]},
               s_b[2] = {st[2 * kb], st[2 * kb + 1]};
  // t' = (c, a, d): opposite c -> (a, d) [was n's edge opposite b], opposite a -> (d, c) [n' corner 1],
  //                 opposite d -> (c, a) [was t's edge opposite b]
  {
    const int32_t v[3] = {c, a, d};
    const int8_t s[6] = {s_c[0], s_c[1], s_a[0], s_a[1], dsx, dsy};
    const int32_t nb[3] = {n_ad, n, n_ca};
    const int8_t nc[3] = {c_ad, 1, c_ca};
    write_triangle(m, t, v, s, nb, nc);
  }
  // n' = (d, b, c): opposite d -> (b, c) [was t's edge opposite a], opposite b -> (c, d) [t' corner 1],
  //                 opposite c -> (d, b) [was n's edge opposite a]
  {
    const int32_t v[3] = {d, b, c};
    const int8_t s[6] = {dsx, dsy, s_b[0], s_b[1], s_c[0], s_c[1]};
    const int32_t nb[3] = {n_bc, t, n_bd};
    const int8_t nc[3] = {c_bc, 1, c_bd};
    write_triangle(m, n, v, s, nb, nc);
  }
  m.tn[3 * (size_t)n_ad + c_ad] = t;
  m.tc[3 * (size_t)n_ad + c_ad] = 0;
  m.tn[3 * (size_t)n_ca + c_ca] = t;
  m.tc[3 * (size_t)n_ca + c_ca] = 2;
  m.tn[3 * (size_t)n_bc + c_bc] = n;
  m.tc[3 * (size_t)n_bc + c_bc] = 0;
  m.tn[3 * (size_t)n_bd + c_bd] = n;
  m.tc[3 * (size_t)n_bd + c_bd] = 2;
}

// Priority of a candidate (Sec. 4.1.1: random integers): 64-bit, unique per index.
MG_HD uint64_t priority(uint64_t seed, uint32_t round, uint32_t index) {
  uint64_t z = seed ^ ((uint64_t)round << 32) ^ (uint64_t)index;
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((z >> 32) << 32) | (uint64_t)(index + 1u);
}

}  // namespace mg
}  // namespace rd
