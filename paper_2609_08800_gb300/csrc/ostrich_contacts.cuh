// Contact-slot activation, decided in FP32 with explicitly rounded operations
// (__fmul_rn / __fadd_rn never fuse into FMA), so that the active index set is a
// deterministic function of the FP32-rounded state on every GPU.  The operation
// order is fixed: dot = (x*x' + y*y') + z*z', cross term by term, rotation of v by
// q/|q| as (v + w t) + qv x t with t = 2 (qv x v).
#pragma once
#include "ostrich_scene.h"

namespace ost {

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 mkf3(float a, float b, float c) { f3 r; r.x = a; r.y = b; r.z = c; return r; }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rdot(f3 a, f3 b) {
  float t = rmul(a.x, b.x);
  t = radd(t, rmul(a.y, b.y));
  return radd(t, rmul(a.z, b.z));
}
__device__ __forceinline__ f3 rcross(f3 a, f3 b) {
  return mkf3(rsub(rmul(a.y, b.z), rmul(a.z, b.y)), rsub(rmul(a.z, b.x), rmul(a.x, b.z)),
              rsub(rmul(a.x, b.y), rmul(a.y, b.x)));
}
__device__ __forceinline__ f3 radd3(f3 a, f3 b) { return mkf3(radd(a.x, b.x), radd(a.y, b.y), radd(a.z, b.z)); }
__device__ __forceinline__ f3 rsub3(f3 a, f3 b) { return mkf3(rsub(a.x, b.x), rsub(a.y, b.y), rsub(a.z, b.z)); }
__device__ __forceinline__ f3 rscale(f3 a, float s) { return mkf3(rmul(a.x, s), rmul(a.y, s), rmul(a.z, s)); }
__device__ __forceinline__ f3 rrot(const float* q, f3 v) {
  float n2 = rmul(q[0], q[0]);
  n2 = radd(n2, rmul(q[1], q[1]));
  n2 = radd(n2, rmul(q[2], q[2]));
  n2 = radd(n2, rmul(q[3], q[3]));
  float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
  float w = rmul(q[0], inv);
  f3 qv = mkf3(rmul(q[1], inv), rmul(q[2], inv), rmul(q[3], inv));
  f3 t = rcross(qv, v);
  t = mkf3(rmul(t.x, 2.0f), rmul(t.y, 2.0f), rmul(t.z, 2.0f));
  f3 c = rcross(qv, t);
  return mkf3(radd(radd(v.x, rmul(w, t.x)), c.x), radd(radd(v.y, rmul(w, t.y)), c.y),
              radd(radd(v.z, rmul(w, t.z)), c.z));
}

// deepest point of a rim circle (centre c, unit axle a, radius r) along -n
__device__ __forceinline__ f3 rrim_deepest(f3 c, f3 a, float r, f3 n) {
  float nd = rdot(n, a);
  f3 perp = rsub3(n, rscale(a, nd));
  float pl = __fsqrt_rn(rdot(perp, perp));
  if (!(pl > 1e-6f)) return c;
  float inv = __fdiv_rn(1.0f, pl);
  return rsub3(c, rscale(perp, rmul(r, inv)));
}

struct Cand { int valid, ftype; f3 n; float d, ex, ez; };

// Features of the box obstacle for one rim: 0 ground, 1 top, 2 near face, 3 near top edge.
__device__ __forceinline__ Cand rbox_feature(const DevScene& s, int f, f3 c, f3 a, float r) {
  Cand k; k.valid = 0; k.ftype = 0; k.n = mkf3(0.f, 0.f, 1.f); k.d = 0.f; k.ex = 0.f; k.ez = 0.f;
  float x0 = (float)s.box[0], x1 = (float)s.box[1], y0 = (float)s.box[2], y1 = (float)s.box[3], H = (float)s.box[4];
  float xm = rmul(0.5f, radd(x0, x1));
  bool front = c.x < xm;
  if (f == 0) { k.valid = 1; return k; }
  if (f == 1) {
    k.d = H;
    f3 x = rrim_deepest(c, a, r, k.n);
    k.valid = (x.x >= x0 && x.x <= x1 && x.y >= y0 && x.y <= y1);
    return k;
  }
  if (f == 2) {
    k.n = front ? mkf3(-1.f, 0.f, 0.f) : mkf3(1.f, 0.f, 0.f);
    k.d = front ? -x0 : x1;
    f3 x = rrim_deepest(c, a, r, k.n);
    k.valid = (x.z >= 0.0f && x.z <= H && x.y >= y0 && x.y <= y1);
    return k;
  }
  float ex = front ? x0 : x1;
  bool region = (front ? (c.x < x0) : (c.x > x1)) && c.z > H && c.y >= y0 && c.y <= y1;
  float dx = rsub(c.x, ex), dz = rsub(c.z, H);
  float len = __fsqrt_rn(radd(rmul(dx, dx), rmul(dz, dz)));
  if (!region || !(len > 1e-6f)) return k;
  float inv = __fdiv_rn(1.0f, len);
  k.n = mkf3(rmul(dx, inv), 0.0f, rmul(dz, inv));
  k.d = radd(rmul(k.n.x, ex), rmul(k.n.z, H));
  k.ftype = 1; k.ex = ex; k.ez = H; k.valid = 1;
  return k;
}

// Per-slot activation result
struct SlotAct { int active, id, ftype; float n[3], d, ex, ez; };

// Velocity-advanced activation test of one candidate point x on plane (n, d) of body
// b (position p, velocity v, angular velocity w): the signed distance, advanced over
// one step with the predicted approach speed (plus one step of gravity), below margin.
__device__ __forceinline__ bool rpredicate(f3 x, f3 n, float d, f3 p, f3 v, f3 w, float hf, float hg, float margin) {
  f3 rr = rsub3(x, p);
  f3 cw = rcross(w, rr);
  f3 vp = mkf3(radd(v.x, cw.x), radd(v.y, cw.y), radd(radd(v.z, hg), cw.z));
  float dist = rsub(rdot(n, x), d);
  float app = rdot(n, vp);
  float pred = radd(dist, rmul(hf, app < 0.0f ? app : 0.0f));
  return pred < margin;
}

// ---------------------------------------------------------------------------
// Heightmap terrain (Sec. IV-D): a triangle mesh over a regular grid.  Vertex (i, j)
// sits at (ox + i sp, oy + j sp, H[i n + j]); cell (i, j) is split along its
// (i, j)-(i+1, j+1) diagonal into face 0 {(i,j), (i+1,j), (i+1,j+1)} and face 1
// {(i,j), (i+1,j+1), (i,j+1)}; face id = 2 ((n - 1) i + j) + t.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hm_x(const DevScene& s, int i) { return radd((float)s.hox, rmul((float)i, (float)s.hsp)); }
__device__ __forceinline__ float hm_y(const DevScene& s, int j) { return radd((float)s.hoy, rmul((float)j, (float)s.hsp)); }
__device__ __forceinline__ f3 hm_vertex(const DevScene& s, int i, int j) {
  return mkf3(hm_x(s, i), hm_y(s, j), __ldg(s.heights + (size_t)i * s.hn + j));
}

// plane (n, d) of a face: n = normalised cross product of the two edges from (i, j)
__device__ __forceinline__ void hm_face(const DevScene& s, int i, int j, int t, f3& n, float& d) {
  f3 A = hm_vertex(s, i, j);
  f3 B = t == 0 ? hm_vertex(s, i + 1, j) : hm_vertex(s, i + 1, j + 1);
  f3 C = t == 0 ? hm_vertex(s, i + 1, j + 1) : hm_vertex(s, i, j + 1);
  f3 nr = rcross(rsub3(B, A), rsub3(C, A));
  float inv = __fdiv_rn(1.0f, __fsqrt_rn(rdot(nr, nr)));
  n = rscale(nr, inv);
  d = rdot(n, A);
}

// cell under the horizontal position of x, clamped to the grid
__device__ __forceinline__ void hm_cell(const DevScene& s, f3 x, int& i, int& j) {
  float fi = floorf(__fdiv_rn(rsub(x.x, (float)s.hox), (float)s.hsp));
  float fj = floorf(__fdiv_rn(rsub(x.y, (float)s.hoy), (float)s.hsp));
  float top = (float)(s.hn - 2);
  i = fi >= 0.0f ? (fi <= top ? (int)fi : s.hn - 2) : 0;
  j = fj >= 0.0f ? (fj <= top ? (int)fj : s.hn - 2) : 0;
}

// does the horizontal position of x lie on face (i, j, t)?  (edges inclusive)
__device__ __forceinline__ bool hm_on_face(const DevScene& s, f3 x, int i, int j, int t) {
  float x0 = hm_x(s, i), x1 = hm_x(s, i + 1), y0 = hm_y(s, j), y1 = hm_y(s, j + 1);
  if (!(x.x >= x0 && x.x <= x1 && x.y >= y0 && x.y <= y1)) return false;
  float u = rsub(x.x, x0), v = rsub(x.y, y0);
  return t == 0 ? u >= v : u <= v;
}

// Activation of the nf slots of one rim of wheel b on the heightmap.  The rim's lowest
// point picks a face; the rim's deepest point against that face's plane picks the
// centre cell of a 3 x 3 block; each face of the block whose own deepest rim point lies
// on the face is a candidate, in scan order (cell row, cell column, face), filling the
// rim's slots; returns true when candidates were left over (more than nf).
__device__ __forceinline__ bool activate_rim_hm(const DevScene& s, int b, int rim, const float* q7, const float* u6,
                                                double h, SlotAct* out) {
  float hf = (float)h, hg = rmul(hf, (float)s.g), margin = (float)s.margin;
  const float* q = q7 + 3;
  f3 p = mkf3(q7[0], q7[1], q7[2]);
  f3 v = mkf3(u6[0], u6[1], u6[2]);
  f3 w = mkf3(u6[3], u6[4], u6[5]);
  float r = (float)s.radius[b], hw = (float)s.hw[b];
  f3 a = rrot(q, mkf3(0.f, 1.f, 0.f));
  f3 c = radd3(p, rrot(q, mkf3(0.f, rim ? hw : -hw, 0.f)));
  for (int f = 0; f < s.nf; ++f) {
    SlotAct& o = out[f];
    o.active = 0; o.id = -1; o.ftype = 0; o.n[0] = 0.f; o.n[1] = 0.f; o.n[2] = 1.f; o.d = 0.f; o.ex = 0.f; o.ez = 0.f;
  }
  f3 xl = rrim_deepest(c, a, r, mkf3(0.f, 0.f, 1.f));
  int i, j;
  hm_cell(s, xl, i, j);
  int t = rsub(xl.x, hm_x(s, i)) >= rsub(xl.y, hm_y(s, j)) ? 0 : 1;
  f3 n0; float d0;
  hm_face(s, i, j, t, n0, d0);
  hm_cell(s, rrim_deepest(c, a, r, n0), i, j);
  int k = 0;
  bool over = false;
  for (int ii = i - 1; ii <= i + 1; ++ii)
    for (int jj = j - 1; jj <= j + 1; ++jj) {
      if (ii < 0 || jj < 0 || ii > s.hn - 2 || jj > s.hn - 2) continue;
      for (int tt = 0; tt < 2; ++tt) {
        f3 n; float d;
        hm_face(s, ii, jj, tt, n, d);
        f3 x = rrim_deepest(c, a, r, n);
        if (!hm_on_face(s, x, ii, jj, tt)) continue;
        if (k == s.nf) { over = true; continue; }
        SlotAct& o = out[k++];
        o.n[0] = n.x; o.n[1] = n.y; o.n[2] = n.z; o.d = d;
        if (rpredicate(x, n, d, p, v, w, hf, hg, margin)) {
          o.active = 1;
          o.id = (b << 24) | (rim << 20) | (2 * ((s.hn - 1) * ii + jj) + tt);
        }
      }
    }
  return over;
}

// Activation of slot `sl` (global slot index) of one world, from the FP32 state of its body.
// q7: position + quaternion, u6: linear + angular velocity (world frame).
__device__ __forceinline__ SlotAct activate_slot(const DevScene& s, int b, int local, const float* q7, const float* u6,
                                                 double h) {
  SlotAct o; o.active = 0; o.id = -1; o.ftype = 0; o.n[0] = 0.f; o.n[1] = 0.f; o.n[2] = 1.f; o.d = 0.f; o.ex = 0.f; o.ez = 0.f;
  float hf = (float)h, hg = rmul(hf, (float)s.g), margin = (float)s.margin;
  const float* q = q7 + 3;
  f3 p = mkf3(q7[0], q7[1], q7[2]);
  f3 v = mkf3(u6[0], u6[1], u6[2]);
  f3 w = mkf3(u6[3], u6[4], u6[5]);
  f3 x, n; float d;
  if (s.shape[b] == SHAPE_BOX) {
    int k = local;
    float hx = (float)s.half[b][0], hy = (float)s.half[b][1], hz = (float)s.half[b][2];
    f3 rb = mkf3((k & 1) ? hx : -hx, (k & 2) ? hy : -hy, (k & 4) ? hz : -hz);
    x = radd3(p, rrot(q, rb));
    n = mkf3(0.f, 0.f, 1.f); d = 0.f;
    o.id = (b << 24) | (k << 20);
  } else {
    int rim = local / s.nf, f = local % s.nf;
    float r = (float)s.radius[b], hw = (float)s.hw[b];
    f3 a = rrot(q, mkf3(0.f, 1.f, 0.f));
    f3 c = radd3(p, rrot(q, mkf3(0.f, rim ? hw : -hw, 0.f)));
    Cand k;
    if (s.env == ENV_PLANE) { k.valid = 1; k.ftype = 0; k.n = mkf3(0.f, 0.f, 1.f); k.d = 0.f; k.ex = 0.f; k.ez = 0.f; }
    else k = rbox_feature(s, f, c, a, r);
    o.ftype = k.ftype; o.n[0] = k.n.x; o.n[1] = k.n.y; o.n[2] = k.n.z; o.d = k.d; o.ex = k.ex; o.ez = k.ez;
    if (!k.valid) return o;
    n = k.n; d = k.d;
    x = rrim_deepest(c, a, r, n);
    o.id = (b << 24) | (rim << 20) | f;
  }
  o.n[0] = n.x; o.n[1] = n.y; o.n[2] = n.z; o.d = d;
  o.active = rpredicate(x, n, d, p, v, w, hf, hg, margin) ? 1 : 0;
  if (!o.active) o.id = -1;
  return o;
}

}  // namespace ost
