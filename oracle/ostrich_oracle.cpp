// Plain FP64 CPU oracle of the Ostrich per-timestep solve and its adjoint.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
// leg of the benchmark may load this library.  It shares no code, header, table or
// helper with the CUDA path; both read their inputs from the seeded scene module.
//
// It follows the paper step by step, slowly and densely:
//   Sec. III-A  backward-Euler kinematics Eq. (1) and implicit dynamics Eq. (2);
//   Sec. III-B  bilateral joint rows Eq. (3), Fischer-Burmeister normal contact
//               Eq. (4), maximal-dissipation friction Eqs. (5)-(7) with the two
//               admissibility safeguards, implicit velocity servo Eq. (8);
//   Sec. III-C  stacked residual Eqs. (9)-(11), kinematic substitution, Schur step
//               Eq. (12) and back-substitution Eq. (13), solved with a dense LU
//               factorisation (no structure exploited) or, as the paper solves it, by
//               preconditioned conjugate residuals (Jacobi or block-Jacobi
//               preconditioner), best-iterate backtracking;
//   Sec. III-D  IFT adjoint Eqs. (14)-(19) reusing the Schur matrix at the returned
//               iterate; the vector-Jacobian products Eq. (17) (position pull-back
//               included) are forward-mode dual-number derivatives of one residual
//               evaluation at the converged state.
// Readings of passages the paper leaves open are listed beside the code that uses
// them.  Parity unpinned for the robot's and the terrain's general motion: no closed
// form; they are pinned through invariants (joint closure, servo law,
// complementarity, cone admissibility) and finite differences.  Closed forms pin the
// box drop and slide, the robot standing on the plane and two hinged boxes standing
// on the plane.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -shared -fPIC  (no FMA contraction, so
// the FP32 contact predicate rounds exactly like the CUDA one on x86 and on Arm).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <cstdio>

namespace {
int g_trace = 0;   // diagnostic: print the Newton history to stderr

// ---------------------------------------------------------------------------
// forward-mode dual numbers (value, derivative along one direction)
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual atan2(Dual y, Dual x) {
  const double r2 = x.v * x.v + y.v * y.v;
  return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
using std::atan2;
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt;

template <class S> inline S smax(S a, double b) { return val(a) > b ? a : S(b); }
template <class S> inline S smin(S a, double b) { return val(a) < b ? a : S(b); }

template <class S> struct V3 { S x, y, z; };
template <class S> inline V3<S> mk(S a, S b, S c) { return V3<S>{a, b, c}; }
template <class S> inline V3<S> operator+(const V3<S>& a, const V3<S>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> inline V3<S> operator-(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> inline V3<S> operator*(const V3<S>& a, S s) { return {a.x * s, a.y * s, a.z * s}; }
template <class S> inline S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> inline V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> inline V3<S> cvt(const double* p) { return {S(p[0]), S(p[1]), S(p[2])}; }

// 3x3 matrices as row-major arrays
template <class S> struct M3 { S a[3][3]; };
template <class S> inline V3<S> mul(const M3<S>& m, const V3<S>& v) {
  return {m.a[0][0] * v.x + m.a[0][1] * v.y + m.a[0][2] * v.z,
          m.a[1][0] * v.x + m.a[1][1] * v.y + m.a[1][2] * v.z,
          m.a[2][0] * v.x + m.a[2][1] * v.y + m.a[2][2] * v.z};
}
template <class S> inline V3<S> mulT(const M3<S>& m, const V3<S>& v) {
  return {m.a[0][0] * v.x + m.a[1][0] * v.y + m.a[2][0] * v.z,
          m.a[0][1] * v.x + m.a[1][1] * v.y + m.a[2][1] * v.z,
          m.a[0][2] * v.x + m.a[1][2] * v.y + m.a[2][2] * v.z};
}

// Rotation matrix of the normalised quaternion q/|q| (w, x, y, z; Hamilton).
template <class S> M3<S> rotmat(const S* q) {
  S n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  M3<S> R;
  R.a[0][0] = S(1.0) - S(2.0) * (y * y + z * z);
  R.a[0][1] = S(2.0) * (x * y - w * z);
  R.a[0][2] = S(2.0) * (x * z + w * y);
  R.a[1][0] = S(2.0) * (x * y + w * z);
  R.a[1][1] = S(1.0) - S(2.0) * (x * x + z * z);
  R.a[1][2] = S(2.0) * (y * z - w * x);
  R.a[2][0] = S(2.0) * (x * z - w * y);
  R.a[2][1] = S(2.0) * (y * z + w * x);
  R.a[2][2] = S(1.0) - S(2.0) * (x * x + y * y);
  return R;
}

// ---------------------------------------------------------------------------
// scene, configuration and layout
// ---------------------------------------------------------------------------
enum { SHAPE_NONE = 0, SHAPE_BOX = 1, SHAPE_WHEEL = 2 };
enum { ENV_PLANE = 0, ENV_BOX = 1, ENV_HEIGHTMAP = 2 };
enum { PULL_FULL = 0, PULL_TRUNC = 1 };
enum { ADJ_PAPER = 0, ADJ_EXACT = 1 };
const int MAXB = 16, MAXJ = 16;

struct OBody { double m, I[3]; int shape; double half[3]; double radius, hw; };
// Joint: revolute (type 0) or prismatic (type 1); a servo row when kp > 0, velocity
// target (mode 0) or position target (mode 1, damping kd).
struct OJoint { int parent, child; double ap[3], ac[3], axp[3], axc[3], p1[3], p2[3]; double kp; int type, mode; double kd; };

struct OScene {
  int nb = 0, nj = 0, env = 0;
  double mu = 0, g = -9.81;
  double box[5] = {0, 0, 0, 0, 0};
  int hn = 0; double hsp = 0, hox = 0, hoy = 0; const float* heights = nullptr;
  OBody b[MAXB];
  OJoint j[MAXJ];
  // layout
  int n_servo = 0, nf = 0, n_slots = 0, m_max = 0, n_state = 0;
  int slot_base[MAXB] = {0}, slot_count[MAXB] = {0};
  int servo_of_joint[MAXJ] = {0};
  int lam_joint(int jj) const { return 5 * jj; }
  int lam_servo(int s) const { return 5 * nj + s; }
  int lam_contact(int s) const { return 5 * nj + n_servo + 3 * s; }
};

// lin: 0 dense LU of the Schur matrix, 1 preconditioned conjugate residual (Sec. III-C);
// pc: the PCR preconditioner (0 Jacobi, 1 block Jacobi); pcr_iters: PCR iterations per Newton
// step; pcr_iters_adj / pcr_rtol_adj: the adjoint's PCR solve (at most that many iterations,
// stopping once |r| <= rtol |b|)
enum { LIN_DIRECT = 0, LIN_PCR = 1 };
enum { PC_JACOBI = 0, PC_BLOCK = 1 };
struct OCfg {
  int budget, kmin, ls, pullback; double tol, delta_rel, kappa, eps, margin;
  int lin = LIN_DIRECT, pc = PC_JACOBI, pcr_iters = 16, pcr_iters_adj = 256; double pcr_rtol_adj = 1e-12;
};

// flat scene format: header[14], then nb*10 body values, then nj*24 joint values
// (parent, child, anchor_p[3], anchor_c[3], axis_p[3], axis_c[3], perp1_p[3], perp2_p[3], kp,
//  type, servo mode, kd)
bool parse_scene(const double* p, const float* heights, OScene& s) {
  s.nb = (int)p[0]; s.nj = (int)p[1]; s.env = (int)p[2]; s.mu = p[3]; s.g = p[4];
  if (s.nb < 1 || s.nb > MAXB || s.nj < 0 || s.nj > MAXJ) return false;
  for (int i = 0; i < 5; ++i) s.box[i] = p[5 + i];
  s.hn = (int)p[10]; s.hsp = p[11]; s.hox = p[12]; s.hoy = p[13]; s.heights = heights;
  const double* q = p + 14;
  for (int i = 0; i < s.nb; ++i, q += 10) {
    OBody& b = s.b[i];
    b.m = q[0]; b.I[0] = q[1]; b.I[1] = q[2]; b.I[2] = q[3]; b.shape = (int)q[4];
    b.half[0] = q[5]; b.half[1] = q[6]; b.half[2] = q[7]; b.radius = q[8]; b.hw = q[9];
  }
  for (int i = 0; i < s.nj; ++i, q += 24) {
    OJoint& jt = s.j[i];
    jt.parent = (int)q[0]; jt.child = (int)q[1];
    for (int k = 0; k < 3; ++k) {
      jt.ap[k] = q[2 + k]; jt.ac[k] = q[5 + k]; jt.axp[k] = q[8 + k]; jt.axc[k] = q[11 + k];
      jt.p1[k] = q[14 + k]; jt.p2[k] = q[17 + k];
    }
    jt.kp = q[20]; jt.type = (int)q[21]; jt.mode = (int)q[22]; jt.kd = q[23];
    if (jt.type != 0 && jt.type != 1) return false;
    if (jt.mode != 0 && jt.mode != 1) return false;
    if (jt.kd < 0.0) return false;
  }
  s.nf = s.env == ENV_PLANE ? 1 : (s.env == ENV_BOX ? 4 : 8);
  // heightmap: at least one 2 x 2 cell block, face ids below 2^20 (contact id field)
  if (s.env == ENV_HEIGHTMAP && (!heights || s.hn < 3 || s.hn > 724 || !(s.hsp > 0))) return false;
  s.n_servo = 0;
  for (int i = 0; i < s.nj; ++i) s.servo_of_joint[i] = s.j[i].kp > 0 ? s.n_servo++ : -1;
  s.n_slots = 0;
  for (int i = 0; i < s.nb; ++i) {
    int c = s.b[i].shape == SHAPE_BOX ? 8 : (s.b[i].shape == SHAPE_WHEEL ? 2 * s.nf : 0);
    s.slot_base[i] = s.n_slots; s.slot_count[i] = c; s.n_slots += c;
  }
  s.m_max = 5 * s.nj + s.n_servo + 3 * s.n_slots;
  s.n_state = 13 * s.nb + s.m_max;
  return true;
}

void parse_cfg(const double* c, OCfg& o) {
  o.budget = (int)c[0]; o.kmin = (int)c[1]; o.tol = c[2]; o.delta_rel = c[3]; o.kappa = c[4];
  o.eps = c[5]; o.margin = c[6]; o.ls = (int)c[7]; o.pullback = (int)c[8];
  o.lin = (int)c[9]; o.pc = (int)c[10]; o.pcr_iters = (int)c[11]; o.pcr_iters_adj = (int)c[12];
  o.pcr_rtol_adj = c[13];
}

// ---------------------------------------------------------------------------
// contact generation: the discrete index set is decided in FP32 with a fixed
// operation order and no FMA contraction, so the CUDA path can reproduce it bit
// for bit.  (Collision detection is outside the paper's method; its role here is
// to fix the active set once per step, Sec. IV-D: geometry held within a step.)
// ---------------------------------------------------------------------------
struct F3 { float x, y, z; };
inline F3 f3(float a, float b, float c) { F3 r; r.x = a; r.y = b; r.z = c; return r; }
inline float fdot(F3 a, F3 b) { float t = a.x * b.x; t = t + a.y * b.y; return t + a.z * b.z; }
inline F3 fcross(F3 a, F3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline F3 fadd(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
inline F3 fsub(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
inline F3 fscale(F3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
// rotate v by q/|q|: t = 2 (qv x v); v' = (v + w t) + qv x t
inline F3 frot(const float* q, F3 v) {
  float n2 = q[0] * q[0]; n2 = n2 + q[1] * q[1]; n2 = n2 + q[2] * q[2]; n2 = n2 + q[3] * q[3];
  float inv = 1.0f / std::sqrt(n2);
  float w = q[0] * inv;
  F3 qv = f3(q[1] * inv, q[2] * inv, q[3] * inv);
  F3 t = fcross(qv, v);
  t = f3(t.x * 2.0f, t.y * 2.0f, t.z * 2.0f);
  F3 c = fcross(qv, t);
  return f3((v.x + w * t.x) + c.x, (v.y + w * t.y) + c.y, (v.z + w * t.z) + c.z);
}

struct Contact {
  int active = 0, body = -1, kind = 0;   // kind 0: box corner, 1: wheel rim
  int corner = 0, rim = 0, feature = 0;  // corner index / rim index (0: -y, 1: +y) / feature id
  int ftype = 0;                         // 0 fixed plane, 1 box edge (normal from the rim centre at q-)
  double n[3] = {0, 0, 1}, d = 0;        // fixed-plane feature
  double ex = 0, ez = 0;                 // edge line (x, z) for ftype 1
  int id = -1;
};

// Predicate result for one (rim or corner, feature) candidate.
struct Cand { int valid; F3 n; float d; int ftype; float ex, ez; };

// deepest point of a rim circle (centre c, unit axle a, radius r) along -n
inline F3 rim_deepest(F3 c, F3 a, float r, F3 n) {
  float nd = fdot(n, a);
  F3 perp = fsub(n, fscale(a, nd));
  float pl = std::sqrt(fdot(perp, perp));
  if (!(pl > 1e-6f)) return c;
  float inv = 1.0f / pl;
  return fsub(c, fscale(perp, r * inv));
}

Cand box_feature(const OScene& s, int f, F3 c, F3 a, float r) {
  Cand k; k.valid = 0; k.n = f3(0, 0, 1); k.d = 0; k.ftype = 0; k.ex = 0; k.ez = 0;
  float x0 = (float)s.box[0], x1 = (float)s.box[1], y0 = (float)s.box[2], y1 = (float)s.box[3], H = (float)s.box[4];
  float xm = 0.5f * (x0 + x1);
  bool front = c.x < xm;
  if (f == 0) { k.valid = 1; k.n = f3(0, 0, 1); k.d = 0.0f; return k; }
  if (f == 1) {
    k.n = f3(0, 0, 1); k.d = H;
    F3 x = rim_deepest(c, a, r, k.n);
    k.valid = (x.x >= x0 && x.x <= x1 && x.y >= y0 && x.y <= y1);
    return k;
  }
  if (f == 2) {
    k.n = front ? f3(-1, 0, 0) : f3(1, 0, 0);
    k.d = front ? -x0 : x1;
    F3 x = rim_deepest(c, a, r, k.n);
    k.valid = (x.z >= 0.0f && x.z <= H && x.y >= y0 && x.y <= y1);
    return k;
  }
  // f == 3: top edge on the near side, as the plane through the edge whose normal
  // points to the rim centre at step start
  float ex = front ? x0 : x1;
  bool region = (front ? (c.x < x0) : (c.x > x1)) && c.z > H && c.y >= y0 && c.y <= y1;
  float dx = c.x - ex, dz = c.z - H;
  float len = std::sqrt(dx * dx + dz * dz);
  if (!region || !(len > 1e-6f)) return k;
  float inv = 1.0f / len;
  k.n = f3(dx * inv, 0.0f, dz * inv);
  k.d = k.n.x * ex + k.n.z * H;
  k.ftype = 1; k.ex = ex; k.ez = H; k.valid = 1;
  return k;
}

// ---------------------------------------------------------------------------
// Heightmap terrain (Sec. IV-D): a triangle mesh over a regular grid.  Vertex (i, j)
// sits at (ox + i sp, oy + j sp, H[i n + j]); cell (i, j) is split along its
// (i, j)-(i+1, j+1) diagonal into face 0 {(i,j), (i+1,j), (i+1,j+1)} and face 1
// {(i,j), (i+1,j+1), (i,j+1)}; face id = 2 ((n - 1) i + j) + t.  Everything here is
// FP32 with one rounding per operation, like the other contact predicates.
// ---------------------------------------------------------------------------
inline float hm_x(const OScene& s, int i) { return (float)s.hox + (float)i * (float)s.hsp; }
inline float hm_y(const OScene& s, int j) { return (float)s.hoy + (float)j * (float)s.hsp; }
inline F3 hm_vertex(const OScene& s, int i, int j) { return f3(hm_x(s, i), hm_y(s, j), s.heights[(size_t)i * s.hn + j]); }

// plane (n, d) of a face, n upward (the cross product of the two edges from vertex
// (i, j) in the order listed above), normalised
inline void hm_face(const OScene& s, int i, int j, int t, F3& n, float& d) {
  F3 A = hm_vertex(s, i, j);
  F3 B = t == 0 ? hm_vertex(s, i + 1, j) : hm_vertex(s, i + 1, j + 1);
  F3 C = t == 0 ? hm_vertex(s, i + 1, j + 1) : hm_vertex(s, i, j + 1);
  F3 nr = fcross(fsub(B, A), fsub(C, A));
  float inv = 1.0f / std::sqrt(fdot(nr, nr));
  n = fscale(nr, inv);
  d = fdot(n, A);
}

// cell under the horizontal position of x, clamped to the grid
inline void hm_cell(const OScene& s, F3 x, int& i, int& j) {
  float fi = std::floor((x.x - (float)s.hox) / (float)s.hsp);
  float fj = std::floor((x.y - (float)s.hoy) / (float)s.hsp);
  float top = (float)(s.hn - 2);
  i = fi >= 0.0f ? (fi <= top ? (int)fi : s.hn - 2) : 0;
  j = fj >= 0.0f ? (fj <= top ? (int)fj : s.hn - 2) : 0;
}

// does the horizontal position of x lie on face (i, j, t)?  (edges inclusive)
inline bool hm_on_face(const OScene& s, F3 x, int i, int j, int t) {
  float x0 = hm_x(s, i), x1 = hm_x(s, i + 1), y0 = hm_y(s, j), y1 = hm_y(s, j + 1);
  if (!(x.x >= x0 && x.x <= x1 && x.y >= y0 && x.y <= y1)) return false;
  float u = x.x - x0, v = x.y - y0;
  return t == 0 ? u >= v : u <= v;
}

// Candidate faces of one rim (centre c, axle a, radius r): the rim's lowest point
// picks a face; the rim's deepest point against that face's plane picks the centre
// cell of a 3 x 3 block; each face of the block whose own deepest rim point lies on
// the face is a candidate, in scan order (cell row i, cell column j, face t), at most
// `cap` of them (more sets `overflow`).
struct HmCand { F3 n; float d; int face; F3 x; };
int hm_rim_candidates(const OScene& s, F3 c, F3 a, float r, HmCand* out, int cap, bool& overflow) {
  F3 xl = rim_deepest(c, a, r, f3(0.0f, 0.0f, 1.0f));
  int i, j;
  hm_cell(s, xl, i, j);
  int t = (xl.x - hm_x(s, i)) >= (xl.y - hm_y(s, j)) ? 0 : 1;
  F3 n0; float d0;
  hm_face(s, i, j, t, n0, d0);
  hm_cell(s, rim_deepest(c, a, r, n0), i, j);
  int k = 0;
  for (int ii = i - 1; ii <= i + 1; ++ii)
    for (int jj = j - 1; jj <= j + 1; ++jj) {
      if (ii < 0 || jj < 0 || ii > s.hn - 2 || jj > s.hn - 2) continue;
      for (int tt = 0; tt < 2; ++tt) {
        F3 n; float d;
        hm_face(s, ii, jj, tt, n, d);
        F3 x = rim_deepest(c, a, r, n);
        if (!hm_on_face(s, x, ii, jj, tt)) continue;
        if (k == cap) { overflow = true; continue; }
        out[k].n = n; out[k].d = d; out[k].face = 2 * ((s.hn - 1) * ii + jj) + tt; out[k].x = x;
        ++k;
      }
    }
  return k;
}

// Generate the slot table for one world at q-.  Activation: a candidate is active
// when its signed distance, advanced over one step with the predicted approach
// velocity (u- plus one step of gravity), is below the margin.
void generate_contacts(const OScene& s, const OCfg& cfg, const double* qm, const double* um, double h,
                       std::vector<Contact>& out, uint32_t& status) {
  out.assign(s.n_slots, Contact());
  float hf = (float)h, hg = hf * (float)s.g, margin = (float)cfg.margin;
  for (int b = 0; b < s.nb; ++b) {
    const OBody& bd = s.b[b];
    if (s.slot_count[b] == 0) continue;
    float q[4] = {(float)qm[7 * b + 3], (float)qm[7 * b + 4], (float)qm[7 * b + 5], (float)qm[7 * b + 6]};
    F3 p = f3((float)qm[7 * b], (float)qm[7 * b + 1], (float)qm[7 * b + 2]);
    F3 v = f3((float)um[6 * b], (float)um[6 * b + 1], (float)um[6 * b + 2]);
    F3 w = f3((float)um[6 * b + 3], (float)um[6 * b + 4], (float)um[6 * b + 5]);
    auto predicate = [&](F3 x, F3 n, float d) -> bool {
      F3 rr = fsub(x, p);
      F3 cw = fcross(w, rr);
      F3 vp = f3(v.x + cw.x, v.y + cw.y, (v.z + hg) + cw.z);
      float dist = fdot(n, x) - d;
      float app = fdot(n, vp);
      float pred = dist + hf * (app < 0.0f ? app : 0.0f);
      return pred < margin;
    };
    if (bd.shape == SHAPE_BOX) {
      for (int k = 0; k < 8; ++k) {
        F3 rb = f3((k & 1) ? (float)bd.half[0] : -(float)bd.half[0],
                   (k & 2) ? (float)bd.half[1] : -(float)bd.half[1],
                   (k & 4) ? (float)bd.half[2] : -(float)bd.half[2]);
        F3 x = fadd(p, frot(q, rb));
        F3 n = f3(0, 0, 1);
        Contact& c = out[s.slot_base[b] + k];
        c.body = b; c.kind = 0; c.corner = k; c.feature = 0; c.ftype = 0;
        c.n[0] = 0; c.n[1] = 0; c.n[2] = 1; c.d = 0;
        c.active = predicate(x, n, 0.0f) ? 1 : 0;
        c.id = c.active ? ((b << 24) | (k << 20) | 0) : -1;
      }
    } else if (bd.shape == SHAPE_WHEEL) {
      float r = (float)bd.radius, hw = (float)bd.hw;
      F3 a = frot(q, f3(0.0f, 1.0f, 0.0f));
      for (int rim = 0; rim < 2; ++rim) {
        F3 c = fadd(p, frot(q, f3(0.0f, rim ? hw : -hw, 0.0f)));
        if (s.env == ENV_HEIGHTMAP) {
          HmCand cand[8];
          bool over = false;
          int nc = hm_rim_candidates(s, c, a, r, cand, s.nf, over);
          if (over) status |= 4u;
          for (int f = 0; f < s.nf; ++f) {
            Contact& ct = out[s.slot_base[b] + rim * s.nf + f];
            ct.body = b; ct.kind = 1; ct.rim = rim; ct.ftype = 0; ct.active = 0; ct.id = -1;
            if (f >= nc) { ct.feature = -1; continue; }
            ct.feature = cand[f].face;
            ct.n[0] = cand[f].n.x; ct.n[1] = cand[f].n.y; ct.n[2] = cand[f].n.z; ct.d = cand[f].d;
            if (predicate(cand[f].x, cand[f].n, cand[f].d)) { ct.active = 1; ct.id = (b << 24) | (rim << 20) | cand[f].face; }
          }
          continue;
        }
        for (int f = 0; f < s.nf; ++f) {
          Cand k = (s.env == ENV_PLANE) ? Cand{1, f3(0, 0, 1), 0.0f, 0, 0.0f, 0.0f}
                                        : box_feature(s, f, c, a, r);
          Contact& ct = out[s.slot_base[b] + rim * s.nf + f];
          ct.body = b; ct.kind = 1; ct.rim = rim; ct.feature = f; ct.ftype = k.ftype;
          ct.n[0] = k.n.x; ct.n[1] = k.n.y; ct.n[2] = k.n.z; ct.d = k.d; ct.ex = k.ex; ct.ez = k.ez;
          ct.active = 0; ct.id = -1;
          if (!k.valid) continue;
          F3 x = rim_deepest(c, a, r, k.n);
          if (predicate(x, k.n, k.d)) { ct.active = 1; ct.id = (b << 24) | (rim << 20) | f; }
        }
      }
    }
  }
  (void)status;
}

// ---------------------------------------------------------------------------
// per-world geometry in working precision S
// ---------------------------------------------------------------------------
template <class S> struct Pose { V3<S> p; M3<S> R; };
template <class S> Pose<S> pose_of(const S* q7) { Pose<S> P; P.p = {q7[0], q7[1], q7[2]}; P.R = rotmat(q7 + 3); return P; }

// Eq. (1): q+ = q- + h G(q-) u, with the quaternion rate 1/2 [0, w] (x) q (world-frame w).
template <class S> void kin_update(int nb, const S* qm, const S* u, double h, S* qp) {
  for (int b = 0; b < nb; ++b) {
    const S* q = qm + 7 * b; const S* ub = u + 6 * b; S* o = qp + 7 * b;
    o[0] = q[0] + S(h) * ub[0]; o[1] = q[1] + S(h) * ub[1]; o[2] = q[2] + S(h) * ub[2];
    S wx = ub[3], wy = ub[4], wz = ub[5];
    S qw = q[3], qx = q[4], qy = q[5], qz = q[6];
    // (0, w) (x) q
    S rw = -(wx * qx + wy * qy + wz * qz);
    S rx = wx * qw + (wy * qz - wz * qy);
    S ry = wy * qw + (wz * qx - wx * qz);
    S rz = wz * qw + (wx * qy - wy * qx);
    S hh = S(0.5 * h);
    o[3] = qw + hh * rw; o[4] = qx + hh * rx; o[5] = qy + hh * ry; o[6] = qz + hh * rz;
  }
}

// World inertia at q-: I_w = R diag(I) R^T; the generalised mass of Eq. (2) is
// blockdiag(m I3, I_w) (reading of "G^T M G" for a position-quaternion body).
template <class S> M3<S> world_inertia(const OBody& b, const M3<S>& R, bool inverse) {
  M3<S> I;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S acc = S(0.0);
      for (int k = 0; k < 3; ++k) acc = acc + R.a[i][k] * S(inverse ? 1.0 / b.I[k] : b.I[k]) * R.a[j][k];
      I.a[i][j] = acc;
    }
  return I;
}

// tangent basis of a contact normal
template <class S> void tangents(const V3<S>& n, V3<S>& t1, V3<S>& t2) {
  V3<S> e = std::fabs(val(n.x)) < 0.9 ? mk(S(1.0), S(0.0), S(0.0)) : mk(S(0.0), S(1.0), S(0.0));
  V3<S> t = e - n * dot(n, e);
  S l = sqrt(dot(t, t));
  t1 = t * (S(1.0) / l);
  t2 = cross(n, t1);
}

// contact frame (n, d); edge features depend on the rim centre at q-
template <class S> void contact_frame(const OScene& s, const Contact& c, const S* qm, V3<S>& n, S& d) {
  if (c.ftype == 1) {
    const S* q = qm + 7 * c.body;
    Pose<S> P = pose_of(q);
    double hw = s.b[c.body].hw;
    V3<S> cen = P.p + mul(P.R, mk(S(0.0), S(c.rim ? hw : -hw), S(0.0)));
    S dx = cen.x - S(c.ex), dz = cen.z - S(c.ez);
    S len = sqrt(dx * dx + dz * dz);
    n = mk(dx / len, S(0.0), dz / len);
    d = n.x * S(c.ex) + n.z * S(c.ez);
  } else {
    n = mk(S(c.n[0]), S(c.n[1]), S(c.n[2]));
    d = S(c.d);
  }
}

// contact point on the body at pose P (box corner: material point; rim: deepest
// point of the rim circle along -n)
template <class S> V3<S> contact_point(const OScene& s, const Contact& c, const Pose<S>& P, const V3<S>& n) {
  const OBody& b = s.b[c.body];
  if (c.kind == 0) {
    V3<S> rb = mk(S((c.corner & 1) ? b.half[0] : -b.half[0]), S((c.corner & 2) ? b.half[1] : -b.half[1]),
                  S((c.corner & 4) ? b.half[2] : -b.half[2]));
    return P.p + mul(P.R, rb);
  }
  V3<S> a = mul(P.R, mk(S(0.0), S(1.0), S(0.0)));
  V3<S> cen = P.p + mul(P.R, mk(S(0.0), S(c.rim ? b.hw : -b.hw), S(0.0)));
  S nd = dot(n, a);
  V3<S> perp = n - a * nd;
  S pl = sqrt(dot(perp, perp));
  if (val(pl) <= 1e-12) return cen;
  return cen - perp * (S(b.radius) / pl);
}

// ---------------------------------------------------------------------------
// constraint rows
// ---------------------------------------------------------------------------
enum { ROW_JOINT = 0, ROW_SERVO = 1, ROW_NORMAL = 2, ROW_FRIC = 3 };
struct Row { int type, b0, b1, joint, sub, slot, lam; };  // lam: index into the lambda block

struct World {
  const OScene* s; const OCfg* cfg; double h;
  std::vector<Contact> con;
  std::vector<Row> rows;
  std::vector<double> what;   // per normal row: J_n M^-1 J_n^T at q- (scaling, frozen)
};

void build_rows(World& W) {
  const OScene& s = *W.s;
  W.rows.clear();
  for (int j = 0; j < s.nj; ++j)
    for (int k = 0; k < 5; ++k) W.rows.push_back({ROW_JOINT, s.j[j].parent, s.j[j].child, j, k, -1, s.lam_joint(j) + k});
  for (int j = 0; j < s.nj; ++j)
    if (s.servo_of_joint[j] >= 0)
      W.rows.push_back({ROW_SERVO, s.j[j].parent, s.j[j].child, j, 0, -1, s.lam_servo(s.servo_of_joint[j])});
  for (int sl = 0; sl < s.n_slots; ++sl) {
    if (!W.con[sl].active) continue;
    int b = W.con[sl].body;
    W.rows.push_back({ROW_NORMAL, b, -1, -1, 0, sl, s.lam_contact(sl)});
    W.rows.push_back({ROW_FRIC, b, -1, -1, 1, sl, s.lam_contact(sl) + 1});
    W.rows.push_back({ROW_FRIC, b, -1, -1, 2, sl, s.lam_contact(sl) + 2});
  }
}

// Jacobian row: 6 entries on b0 and 6 on b1 (b1 < 0: none)
template <class S> struct JRow { S j0[6], j1[6]; };

// Everything the rows need at one iterate.
template <class S> struct Geo {
  std::vector<Pose<S>> P;          // poses at q+
  std::vector<V3<S>> wk;           // per body angular velocity of the iterate (for E)
  double h = 0.0;
  std::vector<V3<S>> n, t1, t2;    // per slot
  std::vector<S> d;
  std::vector<V3<S>> x;            // per slot contact point at q+
};

template <class S> void geometry(const World& W, const S* qm, const S* qp, const S* u, Geo<S>& G) {
  const OScene& s = *W.s;
  G.P.resize(s.nb); G.wk.resize(s.nb); G.h = W.h;
  for (int b = 0; b < s.nb; ++b) {
    G.P[b] = pose_of(qp + 7 * b);
    G.wk[b] = u ? mk(u[6 * b + 3], u[6 * b + 4], u[6 * b + 5]) : mk(S(0.0), S(0.0), S(0.0));
  }
  G.n.resize(s.n_slots); G.t1.resize(s.n_slots); G.t2.resize(s.n_slots); G.d.resize(s.n_slots); G.x.resize(s.n_slots);
  for (int sl = 0; sl < s.n_slots; ++sl) {
    const Contact& c = W.con[sl];
    if (!c.active) continue;
    contact_frame(s, c, qm, G.n[sl], G.d[sl]);
    tangents(G.n[sl], G.t1[sl], G.t2[sl]);
    G.x[sl] = contact_point(s, c, G.P[c.body], G.n[sl]);
  }
}

// Analytic velocity Jacobian of a row at q+ (the paper evaluates J at q+).
// The kinematic map of Eq. (1) moves q+ through G(q-); at q+ = q- + h G(q-) u_k the
// rotation rate it induces for a body angular velocity w is E w with
//   E = (I + h/2 [w_k]x) / (1 + (h/2)^2 |w_k|^2),
// so the row Jacobian d c(q+(u))/du / h of a position constraint is the geometric
// Jacobian at q+ with its angular part multiplied by E^T.  All rows (and the force
// J^T lambda of Eq. (2)) use this J, which keeps the Schur matrix symmetric.
template <class S> V3<S> apply_Et(const V3<S>& a, const V3<S>& wk, double h) {
  S hh = S(0.5 * h);
  S den = S(1.0) + hh * hh * dot(wk, wk);
  return (a + cross(a, wk) * hh) * (S(1.0) / den);
}

// The two world vectors of an orientation row, parent vector bw and child vector aw, whose
// dot product the row holds at zero: revolute rows 3, 4 and prismatic rows 2, 3 align the
// axes (perp1_p / perp2_p against axis_c); prismatic row 4 locks the twist about the axis
// (perp2_p against the child's perp1, given in the child frame by the same coordinates).
template <class S>
void orientation_pair(const OJoint& jt, int sub, const Pose<S>& Pp, const Pose<S>& Pc, V3<S>& bw, V3<S>& aw) {
  const int k = jt.type == 0 ? sub - 3 : sub - 2;          // 0, 1: alignment rows; 2: twist
  if (k < 2) {
    bw = mul(Pp.R, cvt<S>(k == 0 ? jt.p1 : jt.p2));
    aw = mul(Pc.R, cvt<S>(jt.axc));
  } else {
    bw = mul(Pp.R, cvt<S>(jt.p2));
    aw = mul(Pc.R, cvt<S>(jt.p1));
  }
}

// Joint coordinate a position servo tracks (Eq. (8)), at poses Pp, Pc: the revolute angle
// about the parent axis a from the parent's perp1 to the child's (atan2 of the child's
// perp1 against perp1_p and a x perp1_p), or the prismatic slide a . d.
template <class S> S joint_coordinate(const OJoint& jt, const Pose<S>& Pp, const Pose<S>& Pc) {
  V3<S> a = mul(Pp.R, cvt<S>(jt.axp));
  if (jt.type == 0) {
    V3<S> f = mul(Pp.R, cvt<S>(jt.p1));
    V3<S> e = mul(Pc.R, cvt<S>(jt.p1));
    return atan2(dot(e, cross(a, f)), dot(e, f));
  }
  V3<S> rp = mul(Pp.R, cvt<S>(jt.ap)), rc = mul(Pc.R, cvt<S>(jt.ac));
  return dot(a, (Pc.p + rc) - (Pp.p + rp));
}

template <class S> JRow<S> row_jacobian(const World& W, const Row& r, const Geo<S>& G) {
  const OScene& s = *W.s;
  JRow<S> J;
  for (int k = 0; k < 6; ++k) { J.j0[k] = S(0.0); J.j1[k] = S(0.0); }
  int b0 = r.b0, b1 = r.b1;
  double h = G.h;
  auto set0 = [&](const V3<S>& lin, const V3<S>& ang) {
    V3<S> a = apply_Et(ang, G.wk[b0], h);
    J.j0[0] = lin.x; J.j0[1] = lin.y; J.j0[2] = lin.z; J.j0[3] = a.x; J.j0[4] = a.y; J.j0[5] = a.z;
  };
  auto set1 = [&](const V3<S>& lin, const V3<S>& ang) {
    V3<S> a = apply_Et(ang, G.wk[b1], h);
    J.j1[0] = lin.x; J.j1[1] = lin.y; J.j1[2] = lin.z; J.j1[3] = a.x; J.j1[4] = a.y; J.j1[5] = a.z;
  };
  V3<S> zero = mk(S(0.0), S(0.0), S(0.0));
  if (r.type == ROW_JOINT) {
    const OJoint& jt = s.j[r.joint];
    const Pose<S>& Pp = G.P[jt.parent];
    const Pose<S>& Pc = G.P[jt.child];
    V3<S> rp = mul(Pp.R, cvt<S>(jt.ap)), rc = mul(Pc.R, cvt<S>(jt.ac));
    if (jt.type == 0 && r.sub < 3) {
      // revolute anchor rows: (p_p + r_p) - (p_c + r_c), component sub
      V3<S> e = mk(S(r.sub == 0 ? 1.0 : 0.0), S(r.sub == 1 ? 1.0 : 0.0), S(r.sub == 2 ? 1.0 : 0.0));
      set0(e, cross(rp, e));
      set1(e * S(-1.0), cross(rc, e) * S(-1.0));
    } else if (jt.type == 1 && r.sub < 2) {
      // prismatic rows: the child anchor stays on the parent's axis line, b_k . d = 0 with
      // b_k = R_p perp_k and d = (p_c + r_c) - (p_p + r_p)
      V3<S> b = mul(Pp.R, cvt<S>(r.sub == 0 ? jt.p1 : jt.p2));
      V3<S> d = (Pc.p + rc) - (Pp.p + rp);
      set0(b * S(-1.0), cross(b, d + rp));
      set1(b, cross(rc, b));
    } else {
      // orientation rows: parent vector . child vector = 0 (axis alignment: perp_k . axis_c;
      // prismatic twist lock: perp2_p . perp1 of the child)
      V3<S> bw, aw;
      orientation_pair(jt, r.sub, Pp, Pc, bw, aw);
      V3<S> ba = cross(bw, aw);
      set0(zero, ba);
      set1(zero, ba * S(-1.0));
    }
  } else if (r.type == ROW_SERVO) {
    const OJoint& jt = s.j[r.joint];
    const Pose<S>& Pp = G.P[jt.parent];
    const Pose<S>& Pc = G.P[jt.child];
    V3<S> ax = mul(Pp.R, cvt<S>(jt.axp));
    if (jt.type == 0) {
      // relative angular velocity about the axle
      set0(zero, ax * S(-1.0));
      set1(zero, ax);
    } else {
      // slide velocity along the axis: d/dt (a . d)
      V3<S> rp = mul(Pp.R, cvt<S>(jt.ap)), rc = mul(Pc.R, cvt<S>(jt.ac));
      V3<S> d = (Pc.p + rc) - (Pp.p + rp);
      set0(ax * S(-1.0), cross(ax, d + rp));
      set1(ax, cross(rc, ax));
    }
  } else {
    V3<S> dir = r.type == ROW_NORMAL ? G.n[r.slot] : (r.sub == 1 ? G.t1[r.slot] : G.t2[r.slot]);
    V3<S> lever = G.x[r.slot] - G.P[r.b0].p;
    set0(dir, cross(lever, dir));
  }
  return J;
}

// position-level constraint value c(q+) of a joint row or a normal row
template <class S> S row_position_value(const World& W, const Row& r, const Geo<S>& G) {
  const OScene& s = *W.s;
  if (r.type == ROW_JOINT) {
    const OJoint& jt = s.j[r.joint];
    const Pose<S>& Pp = G.P[jt.parent];
    const Pose<S>& Pc = G.P[jt.child];
    V3<S> rp = mul(Pp.R, cvt<S>(jt.ap)), rc = mul(Pc.R, cvt<S>(jt.ac));
    if (jt.type == 0 && r.sub < 3) {
      V3<S> c = (Pp.p + rp) - (Pc.p + rc);
      return r.sub == 0 ? c.x : (r.sub == 1 ? c.y : c.z);
    }
    if (jt.type == 1 && r.sub < 2) {
      V3<S> b = mul(Pp.R, cvt<S>(r.sub == 0 ? jt.p1 : jt.p2));
      return dot(b, (Pc.p + rc) - (Pp.p + rp));
    }
    V3<S> bw, aw;
    orientation_pair(jt, r.sub, Pp, Pc, bw, aw);
    return dot(bw, aw);
  }
  // normal row
  return dot(G.n[r.slot], G.x[r.slot]) - G.d[r.slot];
}

// velocity-level row value J(q+) u for friction and servo rows
template <class S> S row_velocity_value(const World& W, const Row& r, const Geo<S>& G, const S* u) {
  JRow<S> J = row_jacobian(W, r, G);
  S acc = S(0.0);
  for (int k = 0; k < 6; ++k) acc = acc + J.j0[k] * u[6 * r.b0 + k];
  if (r.b1 >= 0) for (int k = 0; k < 6; ++k) acc = acc + J.j1[k] * u[6 * r.b1 + k];
  return acc;
}

// Smoothed Fischer-Burmeister function phi_eps(a, b) = a + b - sqrt(a^2 + b^2 + eps^2)
// (Eq. (4) with the eps-smoothing of Sec. III-D) and its partial derivatives.
template <class S> S fb(S a, S b, double eps) { return a + b - sqrt(a * a + b * b + S(eps * eps)); }
inline void fb_grad(double a, double b, double eps, double& fa, double& fb_) {
  double r = std::sqrt(a * a + b * b + eps * eps);
  fa = 1.0 - a / r; fb_ = 1.0 - b / r;
}

// Friction compliance weight W (reading of Eqs. (6)-(7)): FB on the slip speed v_t
// and the cone margin mu*lambda_n - |lambda_f| gives W = max(0, v_t - phi)/(mu lambda_n);
// W = 0 while sticking and v_t/(mu lambda_n) while sliding.  Norms are eps-smoothed,
// the denominator is guarded (Sec. III-D); W >= 0 is the second safeguard (Sec. III-B).
// The cone margin is a force; it enters the FB function scaled by h*what (what =
// J_n M^-1 J_n^T at q-) so that both FB arguments are velocities, as for the normal row.
template <class S, class Mu = double> S friction_W(S vt1, S vt2, S ln, S lf1, S lf2, Mu mu, double eps, double hw) {
  S vt = sqrt(vt1 * vt1 + vt2 * vt2 + S(eps * eps));
  S lfn = sqrt(lf1 * lf1 + lf2 * lf2 + S(eps * eps));
  S lnp = smax(ln, 0.0);
  S margin = S(hw) * (S(mu) * lnp - lfn);
  S num = smax(vt - fb(vt, margin, eps), 0.0);
  S den = smax(S(mu) * lnp, 1e-12);
  return num / den;
}

// One evaluation of the stacked residual at iterate (u, lambda).
//   rdyn   : Eq. (10) per body, 6 values (N s)
//   r      : per row, in velocity units (merit): joint c/h, normal phi, friction, servo
//   rlin   : per row, the row function whose derivative the adjoint VJP takes
//   C, sc  : (S = double) compliance diagonal and row scale of the Newton row
template <class S> struct Eval {
  std::vector<S> rdyn, r, rlin;
  std::vector<double> rhat;     // Newton right-hand side rows (S = double): joint c/h,
                                // normal phi/phi_a, friction and servo unweighted
  std::vector<double> C, W;     // W per slot (friction compliance at this iterate)
  std::vector<double> Cf;       // per slot: radial friction compliance block (c11, c12, c22)
  std::vector<JRow<S>> J;
  double merit = 0.0;
};

struct Frozen { const std::vector<double>* W; };   // paper-mode VJP: W held at the returned iterate

template <class S>
void evaluate(const World& W, const S* qm, const S* um, const S* ubar, const S* u, const S* lam,
              const Frozen* frz, bool trunc_vjp, const Geo<double>* Gstar, const double* qpstar,
              Eval<S>& E) {
  const OScene& s = *W.s;
  const OCfg& cfg = *W.cfg;
  const double h = W.h;
  int nb = s.nb;
  std::vector<S> qp(7 * nb);
  kin_update(nb, qm, u, h, qp.data());
  Geo<S> G;
  geometry(W, qm, qp.data(), u, G);
  size_t m = W.rows.size();
  E.r.assign(m, S(0.0)); E.rlin.assign(m, S(0.0)); E.J.resize(m);
  E.C.assign(m, 0.0); E.W.assign(s.n_slots, 0.0); E.rhat.assign(m, 0.0); E.Cf.assign(3 * s.n_slots, 0.0);
  E.rdyn.assign(6 * nb, S(0.0));
  // Eq. (2)/(10): M(q-)(u - u-) - h f_ext(q-, u-)
  for (int b = 0; b < nb; ++b) {
    Pose<S> Pm = pose_of(qm + 7 * b);
    M3<S> Iw = world_inertia(s.b[b], Pm.R, false);
    V3<S> w = mk(um[6 * b + 3], um[6 * b + 4], um[6 * b + 5]);
    V3<S> gyro = cross(w, mul(Iw, w)) * S(-1.0);
    V3<S> dw = mk(u[6 * b + 3] - um[6 * b + 3], u[6 * b + 4] - um[6 * b + 4], u[6 * b + 5] - um[6 * b + 5]);
    V3<S> Idw = mul(Iw, dw);
    S mb = S(s.b[b].m);
    E.rdyn[6 * b + 0] = mb * (u[6 * b + 0] - um[6 * b + 0]);
    E.rdyn[6 * b + 1] = mb * (u[6 * b + 1] - um[6 * b + 1]);
    E.rdyn[6 * b + 2] = mb * (u[6 * b + 2] - um[6 * b + 2]) - S(h) * mb * S(s.g);
    E.rdyn[6 * b + 3] = Idw.x - S(h) * gyro.x;
    E.rdyn[6 * b + 4] = Idw.y - S(h) * gyro.y;
    E.rdyn[6 * b + 5] = Idw.z - S(h) * gyro.z;
  }
  // rows
  for (size_t i = 0; i < m; ++i) {
    const Row& r = W.rows[i];
    bool frozen_geo = trunc_vjp && (r.type == ROW_NORMAL || r.type == ROW_FRIC);
    if (frozen_geo) {
      // truncated pull-back: contact frame and lever arm held at the converged state
      JRow<double> Jd = row_jacobian(W, r, *Gstar);
      for (int k = 0; k < 6; ++k) { E.J[i].j0[k] = S(Jd.j0[k]); E.J[i].j1[k] = S(0.0); }
    } else {
      E.J[i] = row_jacobian(W, r, G);
    }
    S lr = lam[r.lam];
    // -h J^T lambda into Eq. (10)
    for (int k = 0; k < 6; ++k) E.rdyn[6 * r.b0 + k] = E.rdyn[6 * r.b0 + k] - S(h) * E.J[i].j0[k] * lr;
    if (r.b1 >= 0) for (int k = 0; k < 6; ++k) E.rdyn[6 * r.b1 + k] = E.rdyn[6 * r.b1 + k] - S(h) * E.J[i].j1[k] * lr;
  }
  for (size_t i = 0; i < m; ++i) {
    const Row& r = W.rows[i];
    if (r.type == ROW_JOINT) {
      // Eq. (3) with E = 0, scaled by 1/h (velocity units)
      S c = row_position_value(W, r, G);
      E.r[i] = c / S(h); E.rlin[i] = E.r[i];
      E.C[i] = 0.0; E.rhat[i] = val(E.r[i]);
    } else if (r.type == ROW_SERVO) {
      // Eq. (8): J_c u + alpha lambda_c + b_c.  Velocity target: alpha = 1/k_p,
      // b_c = -ubar.  Position target: alpha = 1/(k_d + h k_p), b_c = the joint error at
      // the step's start divided by h, (x(q-) - ubar)/h, so J_c u + b_c is the first-order
      // joint error at q+ over h (the reading of "the joint error divided by h").
      const OJoint& jt = s.j[r.joint];
      S v = row_velocity_value(W, r, G, u);
      int si = s.servo_of_joint[r.joint];
      double alpha;
      S bc;
      if (jt.mode == 0) {
        alpha = 1.0 / jt.kp;
        bc = S(0.0) - ubar[si];
      } else {
        alpha = 1.0 / (jt.kd + h * jt.kp);
        Pose<S> Pp = pose_of(qm + 7 * jt.parent), Pc = pose_of(qm + 7 * jt.child);
        bc = (joint_coordinate(jt, Pp, Pc) - ubar[si]) / S(h);
      }
      E.r[i] = v + lam[r.lam] * S(alpha) + bc;
      E.rlin[i] = v + bc;
      E.C[i] = alpha; E.rhat[i] = val(E.r[i]);
    } else if (r.type == ROW_NORMAL) {
      // Eq. (4): phi_eps(c_n/h + kappa lambda_n, h what lambda_n); both arguments in m/s
      S c;
      if (trunc_vjp) {
        // first-order rigid motion of the converged contact point, frame frozen
        const Pose<double>& Ps = Gstar->P[r.b0];
        V3<double> rho = mulT(Ps.R, Gstar->x[r.slot] - Ps.p);     // body-frame material point
        V3<S> xp = G.P[r.b0].p + mul(G.P[r.b0].R, mk(S(rho.x), S(rho.y), S(rho.z)));
        V3<double> n = Gstar->n[r.slot];
        c = S(n.x) * xp.x + S(n.y) * xp.y + S(n.z) * xp.z - S(Gstar->d[r.slot]);
      } else {
        c = row_position_value(W, r, G);
      }
      S ln = lam[r.lam];
      S a = c / S(h) + S(cfg.kappa) * ln;
      S bb = S(h * W.what[r.slot]) * ln;
      E.r[i] = fb(a, bb, cfg.eps);
      E.rlin[i] = c / S(h);
      double fa, fbv;
      fb_grad(val(a), val(bb), cfg.eps, fa, fbv);
      double sc = std::max(fa, 1e-12);
      E.C[i] = cfg.kappa + h * W.what[r.slot] * fbv / sc;
      E.rhat[i] = val(E.r[i]) / sc;
    } else {
      // Eq. (7): J_f u + (W + kappa) lambda_f, W frozen within the iteration
      const Row& rn = W.rows[i - r.sub];     // the contact's normal row
      S v = (trunc_vjp) ? S(0.0) : row_velocity_value(W, r, G, u);
      if (!trunc_vjp) {
        int sl = r.slot;
        int i1 = (r.sub == 1) ? (int)i : (int)i - 1;
        S v1 = row_velocity_value(W, W.rows[i1], G, u);
        S v2 = row_velocity_value(W, W.rows[i1 + 1], G, u);
        S Wf;
        if (frz) Wf = S((*frz->W)[sl]);
        else Wf = friction_W(v1, v2, lam[rn.lam], lam[rn.lam + 1], lam[rn.lam + 2], s.mu, cfg.eps, h * W.what[sl]);
        E.W[sl] = val(Wf);
        // merit row: r_f scaled by h what/(h what + W), a positive weight that leaves the
        // root and the Newton direction unchanged but lets a separating contact (W -> inf,
        // lambda_f clamped to 0) contribute nothing, as the friction cone {0} requires
        double hw = h * W.what[sl];
        S rf = v + (Wf + S(cfg.kappa)) * lam[r.lam];
        E.r[i] = rf * (S(hw) / (S(hw) + Wf));
        E.rhat[i] = val(rf);
        E.rlin[i] = v;
        E.C[i] = val(Wf) + cfg.kappa;
        // Newton block of the contact's two friction rows: W I + lambda_f (dW/dlambda_f)^T.
        // Freezing W lags its dependence on lambda_n (and on u), which is what makes the
        // friction block symmetric (Sec. III-B); its dependence on |lambda_f| adds the
        // symmetric positive semidefinite radial term rho e e^T, e = lambda_f/|lambda_f|,
        // rho = phi_b h what |lambda_f| / (mu lambda_n), which is kept.
        if (r.sub == 1 && !frz) {
          double l1 = val(lam[rn.lam + 1]), l2 = val(lam[rn.lam + 2]), ln = std::max(val(lam[rn.lam]), 0.0);
          double lfn = std::sqrt(l1 * l1 + l2 * l2 + cfg.eps * cfg.eps);
          double a1 = val(v1), a2 = val(v2);
          double vt = std::sqrt(a1 * a1 + a2 * a2 + cfg.eps * cfg.eps);
          double g = hw * (s.mu * ln - lfn);
          double fa, fbv; fb_grad(vt, g, cfg.eps, fa, fbv);
          double num = vt - fb<double>(vt, g, cfg.eps);
          double D = std::max(s.mu * ln, 1e-12);
          if (num > 0.0) {
            double rho = fbv * hw * lfn / D;
            double e1 = l1 / lfn, e2 = l2 / lfn;
            E.Cf[3 * sl] = rho * e1 * e1; E.Cf[3 * sl + 1] = rho * e1 * e2; E.Cf[3 * sl + 2] = rho * e2 * e2;
          }
        }
      }
    }
  }
  // merit: |M^-1 r_dyn|^2 + |r|^2 (all in velocity units)
  double merit = 0.0;
  for (size_t i = 0; i < m; ++i) merit += val(E.r[i]) * val(E.r[i]);
  E.merit = merit;  // dynamics part added by the caller (needs M^-1 in double)
}

// ---------------------------------------------------------------------------
// dense linear algebra (LU with partial pivoting)
// ---------------------------------------------------------------------------
bool lu_solve(int n, std::vector<double> A, std::vector<double>& b) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k; double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i) if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); p = i; }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (p != k) { for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]); std::swap(b[k], b[p]); }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < n; ++j) acc -= A[i * n + j] * b[j];
    b[i] = acc / A[i * n + i];
  }
  return true;
}

// ---------------------------------------------------------------------------
// preconditioned conjugate residual (Sec. III-C solves Eq. (12) with it)
// ---------------------------------------------------------------------------
// The conjugate residual method for a symmetric positive definite A with a symmetric
// positive definite preconditioner P (dense, row-major, n x n), from x0 = 0:
//   r0 = b, z0 = P r0, p0 = z0;  per iteration k
//   alpha = (z_k, A z_k) / (A p_k, P A p_k)
//   x += alpha p_k,  r -= alpha A p_k,  z -= alpha P A p_k      (z_k = P r_k throughout)
//   beta = (z_k+1, A z_k+1) / (z_k, A z_k),  p_k+1 = z_k+1 + beta p_k,  A p_k+1 = A z_k+1 + beta A p_k.
// x_k minimises |L^T (b - A x)|_2, P = L L^T, over the Krylov space K_k(P A, P b) (the
// textbook method, e.g. Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.8 and
// 9.2).  At most `iters` iterations; with rtol > 0 it stops after the first iteration with
// |r_k| <= rtol |b| (r from the recurrence) and sets *conv.  It stops early, too, when a
// denominator is not positive (the exact solution reached, or breakdown).  Returns the
// iterations taken.
int pcr(int n, const std::vector<double>& A, const std::vector<double>& P, const std::vector<double>& b,
        std::vector<double>& x, int iters, double rtol, bool* conv) {
  auto mv = [n](const std::vector<double>& M, const std::vector<double>& v, std::vector<double>& o) {
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += M[i * n + j] * v[j];
      o[i] = acc;
    }
  };
  auto dot = [n](const std::vector<double>& a, const std::vector<double>& c) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += a[i] * c[i];
    return acc;
  };
  x.assign(n, 0.0);
  std::vector<double> r = b, z(n), p(n), Az(n), Ap(n), q(n);
  if (conv) *conv = false;
  const double bb = dot(b, b);
  if (bb == 0.0) { if (conv) *conv = true; return 0; }
  mv(P, r, z);
  p = z;
  mv(A, z, Az);
  Ap = Az;
  double rho = dot(z, Az);
  int k = 0;
  for (; k < iters; ++k) {
    mv(P, Ap, q);
    const double den = dot(Ap, q);
    if (!(den > 0.0) || !(rho > 0.0)) break;
    const double alpha = rho / den;
    for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; z[i] -= alpha * q[i]; }
    mv(A, z, Az);
    const double rho1 = dot(z, Az);
    const double beta = rho1 / rho;
    rho = rho1;
    for (int i = 0; i < n; ++i) { p[i] = z[i] + beta * p[i]; Ap[i] = Az[i] + beta * Ap[i]; }
    if (rtol > 0.0 && dot(r, r) <= rtol * rtol * bb) { if (conv) *conv = true; ++k; break; }
  }
  return k;
}

// The preconditioner P as a dense matrix: Jacobi, P = diag(A)^-1, or block Jacobi, P the
// inverse of A's diagonal blocks, block[i] naming the block of row i.  (The paper names
// no preconditioner; these two are the readings built.)
std::vector<double> precond_matrix(int n, const std::vector<double>& A, const std::vector<int>& block, int kind) {
  std::vector<double> P(n * n, 0.0);
  if (kind == PC_JACOBI) {
    for (int i = 0; i < n; ++i) P[i * n + i] = 1.0 / A[i * n + i];
    return P;
  }
  std::vector<int> seen;
  for (int i = 0; i < n; ++i) {
    if (std::find(seen.begin(), seen.end(), block[i]) != seen.end()) continue;
    seen.push_back(block[i]);
    std::vector<int> idx;
    for (int j = 0; j < n; ++j) if (block[j] == block[i]) idx.push_back(j);
    const int nk = (int)idx.size();
    std::vector<double> Ab(nk * nk);
    for (int a = 0; a < nk; ++a) for (int c = 0; c < nk; ++c) Ab[a * nk + c] = A[idx[a] * n + idx[c]];
    for (int c = 0; c < nk; ++c) {      // column c of the block's inverse
      std::vector<double> e(nk, 0.0);
      e[c] = 1.0;
      lu_solve(nk, Ab, e);
      for (int a = 0; a < nk; ++a) P[idx[a] * n + idx[c]] = e[a];
    }
  }
  return P;
}

// ---------------------------------------------------------------------------
// the per-world solver
// ---------------------------------------------------------------------------
struct Solver {
  World W;
  int nb = 0, nu = 0;
  std::vector<double> qm, um, ubar, lam_in;
  std::vector<M3<double>> Iw, Iwinv;
  std::vector<double> f;          // f_ext per body (6)
  // result
  std::vector<double> u, lam;     // returned iterate
  double merit = 0.0; int iters = 0, ret_k = 0; uint32_t status = 0;
};

void minv_apply(const Solver& S, const double* x, double* y) {
  for (int b = 0; b < S.nb; ++b) {
    double im = 1.0 / S.W.s->b[b].m;
    y[6 * b] = im * x[6 * b]; y[6 * b + 1] = im * x[6 * b + 1]; y[6 * b + 2] = im * x[6 * b + 2];
    V3<double> w = mul(S.Iwinv[b], mk(x[6 * b + 3], x[6 * b + 4], x[6 * b + 5]));
    y[6 * b + 3] = w.x; y[6 * b + 4] = w.y; y[6 * b + 5] = w.z;
  }
}

double full_merit(const Solver& S, const Eval<double>& E) {
  std::vector<double> y(S.nu);
  minv_apply(S, E.rdyn.data(), y.data());
  double m = E.merit;
  for (int i = 0; i < S.nu; ++i) m += y[i] * y[i];
  return m;
}

void clamp_friction(const Solver& S, double* lam) {
  // first safeguard (Sec. III-B): |lambda_f| <= mu lambda_n
  const OScene& s = *S.W.s;
  for (int sl = 0; sl < s.n_slots; ++sl) {
    if (!S.W.con[sl].active) continue;
    int li = s.lam_contact(sl);
    double rad = s.mu * std::max(lam[li], 0.0);
    double n2 = lam[li + 1] * lam[li + 1] + lam[li + 2] * lam[li + 2];
    double nn = std::sqrt(n2);
    if (nn > rad) {
      double f = nn > 0.0 ? rad / nn : 0.0;
      lam[li + 1] *= f; lam[li + 2] *= f;
    }
  }
}

void setup(Solver& S, const OScene& sc, const OCfg& cfg, const double* state, const double* ubar, double h) {
  S.W.s = &sc; S.W.cfg = &cfg; S.W.h = h;
  S.nb = sc.nb; S.nu = 6 * sc.nb;
  S.qm.assign(state, state + 7 * sc.nb);
  S.um.assign(state + 7 * sc.nb, state + 13 * sc.nb);
  S.lam_in.assign(state + 13 * sc.nb, state + 13 * sc.nb + sc.m_max);
  S.ubar.assign(ubar, ubar + sc.n_servo);
  S.status = 0;
  generate_contacts(sc, cfg, S.qm.data(), S.um.data(), h, S.W.con, S.status);
  build_rows(S.W);
  S.Iw.resize(sc.nb); S.Iwinv.resize(sc.nb); S.f.assign(6 * sc.nb, 0.0);
  for (int b = 0; b < sc.nb; ++b) {
    Pose<double> P = pose_of(S.qm.data() + 7 * b);
    S.Iw[b] = world_inertia(sc.b[b], P.R, false);
    S.Iwinv[b] = world_inertia(sc.b[b], P.R, true);
    V3<double> w = mk(S.um[6 * b + 3], S.um[6 * b + 4], S.um[6 * b + 5]);
    V3<double> gy = cross(w, mul(S.Iw[b], w)) * -1.0;
    S.f[6 * b + 2] = sc.b[b].m * sc.g;
    S.f[6 * b + 3] = gy.x; S.f[6 * b + 4] = gy.y; S.f[6 * b + 5] = gy.z;
  }
  // what_i = J_n M^-1 J_n^T at q- (scales the FB arguments to m/s; frozen in the step)
  S.W.what.assign(sc.n_slots, 0.0);
  Geo<double> G0;
  geometry<double>(S.W, S.qm.data(), S.qm.data(), nullptr, G0);
  for (size_t i = 0; i < S.W.rows.size(); ++i) {
    const Row& r = S.W.rows[i];
    if (r.type != ROW_NORMAL) continue;
    JRow<double> J = row_jacobian(S.W, r, G0);
    double y[6];
    double x[6]; for (int k = 0; k < 6; ++k) x[k] = J.j0[k];
    y[0] = x[0] / sc.b[r.b0].m; y[1] = x[1] / sc.b[r.b0].m; y[2] = x[2] / sc.b[r.b0].m;
    V3<double> wv = mul(S.Iwinv[r.b0], mk(x[3], x[4], x[5]));
    y[3] = wv.x; y[4] = wv.y; y[5] = wv.z;
    double acc = 0.0; for (int k = 0; k < 6; ++k) acc += x[k] * y[k];
    S.W.what[r.slot] = acc;
  }
}

void eval_d(const Solver& S, const double* u, const double* lam, Eval<double>& E) {
  evaluate<double>(S.W, S.qm.data(), S.um.data(), S.ubar.data(), u, lam, nullptr, false, nullptr, nullptr, E);
  E.merit = full_merit(S, E);
}

// Assemble A = h J M^-1 J^T + diag(C) + delta I (Eq. (12) with the paper's C
// absorbing 1/h) over the active rows.
void assemble(const Solver& S, const Eval<double>& E, std::vector<double>& A, std::vector<double>& MJt) {
  size_t m = S.W.rows.size();
  int nu = S.nu;
  // dense J (m x nu) and M^-1 J^T (nu x m)
  std::vector<double> J(m * nu, 0.0);
  for (size_t i = 0; i < m; ++i) {
    const Row& r = S.W.rows[i];
    for (int k = 0; k < 6; ++k) J[i * nu + 6 * r.b0 + k] += E.J[i].j0[k];
    if (r.b1 >= 0) for (int k = 0; k < 6; ++k) J[i * nu + 6 * r.b1 + k] += E.J[i].j1[k];
  }
  MJt.assign(nu * m, 0.0);
  std::vector<double> col(nu), y(nu);
  for (size_t i = 0; i < m; ++i) {
    for (int k = 0; k < nu; ++k) col[k] = J[i * nu + k];
    minv_apply(S, col.data(), y.data());
    for (int k = 0; k < nu; ++k) MJt[k * m + i] = y[k];
  }
  A.assign(m * m, 0.0);
  double diag = 0.0;
  for (size_t i = 0; i < m; ++i)
    for (size_t j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int k = 0; k < nu; ++k) acc += J[i * nu + k] * MJt[k * m + j];
      A[i * m + j] = S.W.h * acc;
      if (i == j) diag += S.W.h * acc;
    }
  double delta = m ? S.W.cfg->delta_rel * diag / (double)m : 0.0;
  for (size_t i = 0; i < m; ++i) A[i * m + i] += E.C[i] + delta;
  for (size_t i = 0; i < m; ++i) {
    const Row& r = S.W.rows[i];
    if (r.type != ROW_FRIC || r.sub != 1) continue;
    const double* cf = &E.Cf[3 * r.slot];
    A[i * m + i] += cf[0]; A[i * m + i + 1] += cf[1]; A[(i + 1) * m + i] += cf[1]; A[(i + 1) * m + i + 1] += cf[2];
  }
}

void jt_apply(const Solver& S, const Eval<double>& E, const double* x, double* out) {
  for (int k = 0; k < S.nu; ++k) out[k] = 0.0;
  for (size_t i = 0; i < S.W.rows.size(); ++i) {
    const Row& r = S.W.rows[i];
    for (int k = 0; k < 6; ++k) out[6 * r.b0 + k] += E.J[i].j0[k] * x[i];
    if (r.b1 >= 0) for (int k = 0; k < 6; ++k) out[6 * r.b1 + k] += E.J[i].j1[k] * x[i];
  }
}

void j_apply(const Solver& S, const Eval<double>& E, const double* v, double* out) {
  for (size_t i = 0; i < S.W.rows.size(); ++i) {
    const Row& r = S.W.rows[i];
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) acc += E.J[i].j0[k] * v[6 * r.b0 + k];
    if (r.b1 >= 0) for (int k = 0; k < 6; ++k) acc += E.J[i].j1[k] * v[6 * r.b1 + k];
    out[i] = acc;
  }
}

// Block of each row for the block-Jacobi preconditioner: the contact rows of one body
// (normal and friction rows of all its contacts) form a block, the joint and servo rows
// together another.
std::vector<int> row_blocks(const Solver& S) {
  std::vector<int> blk(S.W.rows.size());
  for (size_t i = 0; i < blk.size(); ++i) {
    const Row& r = S.W.rows[i];
    blk[i] = (r.type == ROW_NORMAL || r.type == ROW_FRIC) ? r.b0 : -1;
  }
  return blk;
}

// A x = b for the Schur matrix of Eq. (12) by the configured method: dense LU, or PCR
// (Newton steps: cfg.pcr_iters iterations; the adjoint: up to cfg.pcr_iters_adj, stopping
// at |r| <= cfg.pcr_rtol_adj |b|).  Returns false when LU meets a singular matrix.
bool schur_linear_solve(const Solver& S, const std::vector<double>& A, const std::vector<double>& b,
                        std::vector<double>& x, bool adjoint) {
  const OCfg& cfg = *S.W.cfg;
  const int m = (int)b.size();
  if (m == 0) { x.clear(); return true; }
  if (cfg.lin != LIN_PCR) { x = b; return lu_solve(m, A, x); }
  const std::vector<double> P = precond_matrix(m, A, row_blocks(S), cfg.pc);
  if (adjoint) pcr(m, A, P, b, x, cfg.pcr_iters_adj, cfg.pcr_rtol_adj, nullptr);
  else pcr(m, A, P, b, x, cfg.pcr_iters, 0.0, nullptr);
  return true;
}

// Newton iterate container
struct Iter { std::vector<double> u, lam; Eval<double> E; };

void solve_step(Solver& S) {
  const OScene& sc = *S.W.s;
  const OCfg& cfg = *S.W.cfg;
  const double h = S.W.h;
  int nu = S.nu;
  size_t m = S.W.rows.size();
  // warm start: u0 = u- + h M^-1 f_ext, lambda0 = lambda- on the active rows
  Iter cur;
  cur.u.assign(nu, 0.0);
  std::vector<double> mf(nu);
  minv_apply(S, S.f.data(), mf.data());
  for (int k = 0; k < nu; ++k) cur.u[k] = S.um[k] + h * mf[k];
  cur.lam.assign(sc.m_max, 0.0);
  for (size_t i = 0; i < m; ++i) cur.lam[S.W.rows[i].lam] = S.lam_in[S.W.rows[i].lam];
  clamp_friction(S, cur.lam.data());
  eval_d(S, cur.u.data(), cur.lam.data(), cur.E);

  Iter best; double best_merit = INFINITY; int best_k = -1;
  bool conv = false;
  int k = 0;
  std::vector<double> A, MJt, rhs(m), dl(m), tmp(nu), du(nu), mr(nu);
  for (k = 0; k < cfg.budget; ++k) {
    double mk_ = cur.E.merit;
    if (k >= cfg.kmin && mk_ < best_merit) { best = cur; best_merit = mk_; best_k = k; }
    if (std::sqrt(mk_) < cfg.tol) { conv = true; break; }
    // Schur step, Eq. (12): (h J M^-1 J^T + C + delta) dl = J M^-1 r_dyn - r_hat
    assemble(S, cur.E, A, MJt);
    minv_apply(S, cur.E.rdyn.data(), mr.data());
    std::vector<double> jm(m);
    j_apply(S, cur.E, mr.data(), jm.data());
    for (size_t i = 0; i < m; ++i) rhs[i] = jm[i] - cur.E.rhat[i];
    bool ok = schur_linear_solve(S, A, rhs, dl, false);
    if (!ok) for (size_t i = 0; i < m; ++i) dl[i] = NAN;
    // Eq. (13): du = M^-1 (h J^T dl - r_dyn)
    std::vector<double> jtdl(nu);
    jt_apply(S, cur.E, dl.data(), jtdl.data());
    for (int q = 0; q < nu; ++q) tmp[q] = h * jtdl[q] - cur.E.rdyn[q];
    minv_apply(S, tmp.data(), du.data());
    // step control.  Line search off (the paper, Sec. III-C): the full step is taken and
    // the best iterate decides.  Line search on: backtracking alpha in {1, 1/2, 1/4, 1/8},
    // the first alpha that decreases the merit is taken, else alpha = 1/8.
    Iter trial;
    int n_alpha = cfg.ls ? 4 : 1;
    double alpha = 1.0;
    for (int a = 0; a < n_alpha; ++a) {
      alpha = a == 0 ? 1.0 : alpha * 0.5;
      trial.u = cur.u; trial.lam = cur.lam;
      for (int q = 0; q < nu; ++q) trial.u[q] += alpha * du[q];
      for (size_t i = 0; i < m; ++i) trial.lam[S.W.rows[i].lam] += alpha * dl[i];
      clamp_friction(S, trial.lam.data());
      eval_d(S, trial.u.data(), trial.lam.data(), trial.E);
      if (trial.E.merit < mk_) break;
    }
    if (g_trace) {
      std::fprintf(stderr, "k=%d merit=%.3e -> %.3e alpha=%g |dl|max=", k, mk_, trial.E.merit, alpha);
      double mx = 0; for (size_t i = 0; i < m; ++i) mx = std::max(mx, std::fabs(dl[i]));
      std::fprintf(stderr, "%.3e\n", mx);
      if (g_trace > 1) {
        for (size_t i = 0; i < m; ++i) std::fprintf(stderr, "   row %zu type %d r=% .3e C=% .3e lam=% .4e dl=% .3e\n", i,
                                                     S.W.rows[i].type, cur.E.r[i], cur.E.C[i], cur.lam[S.W.rows[i].lam], dl[i]);
      }
    }
    cur = trial;
  }
  S.iters = k;
  if (conv) {
    S.u = cur.u; S.lam = cur.lam; S.merit = cur.E.merit; S.ret_k = k;
  } else {
    if (k >= cfg.kmin && cur.E.merit < best_merit) { best = cur; best_merit = cur.E.merit; best_k = k; }
    if (best_k < 0) { best = cur; best_k = k; best_merit = cur.E.merit; }
    S.u = best.u; S.lam = best.lam; S.merit = best_merit; S.ret_k = best_k;
    S.status |= 1u;
  }
  bool finite = std::isfinite(S.merit);
  for (double v : S.u) finite = finite && std::isfinite(v);
  for (double v : S.lam) finite = finite && std::isfinite(v);
  if (!finite) S.status |= 2u;
}

void write_outputs(const Solver& S, double* state_out, double* impulses, int32_t* ids) {
  const OScene& sc = *S.W.s;
  int nb = sc.nb;
  std::vector<double> qp(7 * nb);
  kin_update(nb, S.qm.data(), S.u.data(), S.W.h, qp.data());
  for (int b = 0; b < nb; ++b) {
    double* q = qp.data() + 7 * b + 3;
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) q[k] /= n;
  }
  if (state_out) {
    for (int i = 0; i < 7 * nb; ++i) state_out[i] = qp[i];
    for (int i = 0; i < 6 * nb; ++i) state_out[7 * nb + i] = S.u[i];
    for (int i = 0; i < sc.m_max; ++i) state_out[13 * nb + i] = S.lam[i];
  }
  if (impulses) for (int i = 0; i < sc.m_max; ++i) impulses[i] = S.W.h * S.lam[i];
  if (ids) for (int sl = 0; sl < sc.n_slots; ++sl) ids[sl] = S.W.con[sl].active ? S.W.con[sl].id : -1;
}

// ---------------------------------------------------------------------------
// adjoint (Sec. III-D)
// ---------------------------------------------------------------------------
// G(q-)^T applied to a position-quaternion cotangent (7 per body) -> 6 per body.
// The columns of G are read off the kinematic map of Eq. (1) itself: G e_k is the
// change of q under a unit velocity e_k over a unit step.
void Gt_apply(int nb, const double* qm, const double* gq, double* out) {
  std::vector<double> e(6 * nb, 0.0), q1(7 * nb);
  for (int c = 0; c < 6 * nb; ++c) {
    e[c] = 1.0;
    kin_update(nb, qm, e.data(), 1.0, q1.data());
    double acc = 0.0;
    for (int i = 0; i < 7 * nb; ++i) acc += gq[i] * (q1[i] - qm[i]);
    out[c] = acc;
    e[c] = 0.0;
  }
}

// Psi(q-, u-, ubar) = g_q . q+(q-, u*) + w_u . r_dyn + sum_rows w_row . rlin_row, at the
// returned iterate (u*, lambda*), so that dL/dxi = dPsi/dxi (Eq. (17)).
template <class S>
S psi(const Solver& Sv, const std::vector<double>& gq, const std::vector<double>& wu,
      const std::vector<double>& wl, const S* qm, const S* um, const S* ubar, bool trunc,
      const Geo<double>* Gstar, bool exact, const std::vector<double>* wfull) {
  const OScene& sc = *Sv.W.s;
  int nb = sc.nb;
  std::vector<S> u(6 * nb), lam(sc.m_max);
  for (int i = 0; i < 6 * nb; ++i) u[i] = S(Sv.u[i]);
  for (int i = 0; i < sc.m_max; ++i) lam[i] = S(Sv.lam[i]);
  std::vector<S> qp(7 * nb);
  kin_update(nb, qm, u.data(), Sv.W.h, qp.data());
  S acc = S(0.0);
  for (int i = 0; i < 7 * nb; ++i) acc = acc + S(gq[i]) * qp[i];
  Eval<S> E;
  Frozen fz{nullptr};
  std::vector<double> Wstar;
  if (!exact) {
    Eval<double> Ed;
    evaluate<double>(Sv.W, Sv.qm.data(), Sv.um.data(), Sv.ubar.data(), Sv.u.data(), Sv.lam.data(), nullptr, false,
                     nullptr, nullptr, Ed);
    Wstar = Ed.W;
    fz.W = &Wstar;
  }
  evaluate<S>(Sv.W, qm, um, ubar, u.data(), lam.data(), exact ? nullptr : &fz, trunc, Gstar, nullptr, E);
  for (int i = 0; i < 6 * nb; ++i) acc = acc + S(wu[i]) * E.rdyn[i];
  const std::vector<S>& rowv = exact ? E.r : E.rlin;
  for (size_t i = 0; i < Sv.W.rows.size(); ++i) acc = acc + S(exact ? (*wfull)[i] : wl[i]) * rowv[i];
  return acc;
}

struct AdjOut { std::vector<double> dq, du, dubar, dkp, dmass, dinertia; double dmu = 0.0; };

void adjoint(const Solver& Sv, const double* dL_dsp, int mode, AdjOut& out) {
  const OScene& sc = *Sv.W.s;
  const OCfg& cfg = *Sv.W.cfg;
  int nb = sc.nb, nu = Sv.nu;
  double h = Sv.W.h;
  size_t m = Sv.W.rows.size();
  // output quaternions are normalised: pull dL/dq_hat back through q_hat = q/|q|
  std::vector<double> qp(7 * nb);
  kin_update(nb, Sv.qm.data(), Sv.u.data(), h, qp.data());
  std::vector<double> gq(7 * nb), gu(nu);
  for (int b = 0; b < nb; ++b) {
    for (int k = 0; k < 3; ++k) gq[7 * b + k] = dL_dsp[7 * b + k];
    const double* q = qp.data() + 7 * b + 3;
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qh[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    const double* g = dL_dsp + 7 * b + 3;
    double dotv = qh[0] * g[0] + qh[1] * g[1] + qh[2] * g[2] + qh[3] * g[3];
    for (int k = 0; k < 4; ++k) gq[7 * b + 3 + k] = (g[k] - qh[k] * dotv) / n;
  }
  for (int i = 0; i < nu; ++i) gu[i] = dL_dsp[7 * nb + i];
  // g = grad_u L + h G(q-)^T grad_q L   (shared term of Eqs. (18), (19))
  std::vector<double> g(nu), gtg(nu);
  Gt_apply(nb, Sv.qm.data(), gq.data(), gtg.data());
  for (int i = 0; i < nu; ++i) g[i] = gu[i] + h * gtg[i];

  std::vector<double> wu(nu), wl(m, 0.0), wfull;
  Eval<double> E;
  eval_d(Sv, Sv.u.data(), Sv.lam.data(), E);
  if (mode == ADJ_PAPER) {
    // Eq. (18): A w_lambda = -h J M^-1 g with the forward A at the returned iterate
    std::vector<double> A, MJt;
    assemble(Sv, E, A, MJt);
    std::vector<double> mg(nu), jmg(m);
    minv_apply(Sv, g.data(), mg.data());
    j_apply(Sv, E, mg.data(), jmg.data());
    for (size_t i = 0; i < m; ++i) wl[i] = -h * jmg[i];
    std::vector<double> rhs = wl;
    schur_linear_solve(Sv, A, rhs, wl, true);
    // Eq. (19): w_u = -M^-1 (g + J^T w_lambda)
    std::vector<double> jtw(nu), t(nu);
    jt_apply(Sv, E, wl.data(), jtw.data());
    for (int i = 0; i < nu; ++i) t[i] = g[i] + jtw[i];
    minv_apply(Sv, t.data(), wu.data());
    for (int i = 0; i < nu; ++i) wu[i] = -wu[i];
  } else {
    // exact IFT: dense Jacobian of F = [r_dyn; r] in (u, lambda) by dual numbers,
    // W and the FB arguments live (no frozen quantities)
    int n = nu + (int)m;
    std::vector<double> Jf(n * n, 0.0);
    for (int c = 0; c < n; ++c) {
      std::vector<Dual> u(nu), lam(sc.m_max), qmD(7 * nb), umD(nu), ubD(sc.n_servo);
      for (int i = 0; i < nu; ++i) u[i] = Dual(Sv.u[i], c == i ? 1.0 : 0.0);
      for (int i = 0; i < sc.m_max; ++i) lam[i] = Dual(Sv.lam[i]);
      if (c >= nu) lam[Sv.W.rows[c - nu].lam].d = 1.0;
      for (int i = 0; i < 7 * nb; ++i) qmD[i] = Dual(Sv.qm[i]);
      for (int i = 0; i < nu; ++i) umD[i] = Dual(Sv.um[i]);
      for (int i = 0; i < sc.n_servo; ++i) ubD[i] = Dual(Sv.ubar[i]);
      Eval<Dual> Ed;
      evaluate<Dual>(Sv.W, qmD.data(), umD.data(), ubD.data(), u.data(), lam.data(), nullptr, false, nullptr, nullptr, Ed);
      for (int i = 0; i < nu; ++i) Jf[i * n + c] = Ed.rdyn[i].d;
      for (size_t i = 0; i < m; ++i) Jf[(nu + i) * n + c] = Ed.r[i].d;
    }
    // transpose solve: Jf^T w = -[g; 0]
    std::vector<double> JT(n * n);
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) JT[i * n + j] = Jf[j * n + i];
    wfull.assign(n, 0.0);
    for (int i = 0; i < nu; ++i) wfull[i] = -g[i];
    lu_solve(n, JT, wfull);
    for (int i = 0; i < nu; ++i) wu[i] = wfull[i];
    std::vector<double> wr(m);
    for (size_t i = 0; i < m; ++i) wr[i] = wfull[nu + i];
    wfull = wr;
  }
  // Eq. (17) by forward-mode duals over (q-, u-, ubar), one direction at a time
  bool trunc = cfg.pullback == PULL_TRUNC && mode == ADJ_PAPER;
  Geo<double> Gstar;
  if (trunc) {
    std::vector<double> qps(7 * nb);
    kin_update(nb, Sv.qm.data(), Sv.u.data(), h, qps.data());
    geometry(Sv.W, Sv.qm.data(), qps.data(), Sv.u.data(), Gstar);
  }
  int nin = 7 * nb + nu + sc.n_servo;
  out.dq.assign(7 * nb, 0.0); out.du.assign(nu, 0.0); out.dubar.assign(sc.n_servo, 0.0);
  for (int c = 0; c < nin; ++c) {
    std::vector<Dual> qmD(7 * nb), umD(nu), ubD(sc.n_servo);
    for (int i = 0; i < 7 * nb; ++i) qmD[i] = Dual(Sv.qm[i], c == i ? 1.0 : 0.0);
    for (int i = 0; i < nu; ++i) umD[i] = Dual(Sv.um[i], c == 7 * nb + i ? 1.0 : 0.0);
    for (int i = 0; i < sc.n_servo; ++i) ubD[i] = Dual(Sv.ubar[i], c == 7 * nb + nu + i ? 1.0 : 0.0);
    Dual p = psi<Dual>(Sv, gq, wu, wl, qmD.data(), umD.data(), ubD.data(), trunc, trunc ? &Gstar : nullptr,
                       mode == ADJ_EXACT, &wfull);
    if (c < 7 * nb) out.dq[c] = p.d;
    else if (c < 7 * nb + nu) out.du[c - 7 * nb] = p.d;
    else out.dubar[c - 7 * nb - nu] = p.d;
  }
  // Eq. (17) with xi = theta, the physical parameters: the explicit partial derivative
  // of the stacked residual at the returned iterate, contracted with the adjoint.
  //   servo gain k_p of a joint: only its servo row, Eq. (8), holds it, through
  //     lambda_c / k_p:  d/dk_p = -lambda_c / k_p^2;
  //   mass m_b of a body: only the linear rows of Eq. (10) for that body hold it
  //     (m (v - v-) - h m g):  d/dm_b = (v - v-) - h g e_z;
  //   principal moment I_k of a body: its angular rows, I_w (w - w-) + h w- x (I_w w-)
  //     with I_w = R diag(I) R^T at q-, so with r_k the k-th column of R,
  //     d/dI_k = r_k (r_k . (w - w-)) + h (r_k . w-) (w- x r_k).
  // (The FB scaling what = J M^-1 J^T of the normal rows also holds m_b, but in the
  // paper's adjoint it is a step-start constant like W, and the FB root does not move
  // under it.)
  const std::vector<double>& wr = mode == ADJ_EXACT ? wfull : wl;
  out.dkp.assign(sc.n_servo, 0.0);
  out.dmass.assign(nb, 0.0);
  out.dinertia.assign(3 * nb, 0.0);
  for (size_t i = 0; i < m; ++i) {
    const Row& r = Sv.W.rows[i];
    if (r.type != ROW_SERVO) continue;
    // alpha = 1/k_p (velocity target) or 1/(k_d + h k_p) (position target)
    const OJoint& jt = sc.j[r.joint];
    const double dalpha = jt.mode == 0 ? -1.0 / (jt.kp * jt.kp)
                                       : -h / ((jt.kd + h * jt.kp) * (jt.kd + h * jt.kp));
    out.dkp[sc.servo_of_joint[r.joint]] = wr[i] * Sv.lam[r.lam] * dalpha;
  }
  // Eq. (17) with xi = mu, the friction coefficient.  mu enters only the friction rows of
  // Eq. (7), through W (the cone margin h what (mu lambda_n - |lambda_f|) and the
  // denominator mu lambda_n) and through the positive row weight h what / (h what + W) of
  // the residual whose Jacobian the exact adjoint takes.  The paper's adjoint holds W at
  // its value at the returned iterate, so there the gradient is zero.
  out.dmu = 0.0;
  if (mode == ADJ_EXACT) {
    std::vector<double> qpu(7 * nb);
    kin_update(nb, Sv.qm.data(), Sv.u.data(), h, qpu.data());
    Geo<double> Gu;
    geometry(Sv.W, Sv.qm.data(), qpu.data(), Sv.u.data(), Gu);
    for (size_t i = 0; i < m; ++i) {
      const Row& r = Sv.W.rows[i];
      if (r.type != ROW_FRIC || r.sub != 1) continue;
      const Row& rn = Sv.W.rows[i - 1];
      const double v[2] = {row_velocity_value(Sv.W, Sv.W.rows[i], Gu, Sv.u.data()),
                           row_velocity_value(Sv.W, Sv.W.rows[i + 1], Gu, Sv.u.data())};
      const double hw = h * Sv.W.what[r.slot];
      Dual Wf = friction_W<Dual, Dual>(Dual(v[0]), Dual(v[1]), Dual(Sv.lam[rn.lam]), Dual(Sv.lam[rn.lam + 1]),
                                       Dual(Sv.lam[rn.lam + 2]), Dual(sc.mu, 1.0), cfg.eps, hw);
      for (int k = 0; k < 2; ++k) {
        Dual rf = Dual(v[k]) + (Wf + Dual(cfg.kappa)) * Dual(Sv.lam[rn.lam + 1 + k]);
        Dual rw = rf * (Dual(hw) / (Dual(hw) + Wf));
        out.dmu += wr[i + k] * rw.d;
      }
    }
  }
  for (int b = 0; b < nb; ++b) {
    double acc = 0.0;
    for (int k = 0; k < 3; ++k) acc += wu[6 * b + k] * (Sv.u[6 * b + k] - Sv.um[6 * b + k]);
    acc += wu[6 * b + 2] * (-h * sc.g);
    out.dmass[b] = acc;
    Pose<double> Pm = pose_of(Sv.qm.data() + 7 * b);
    V3<double> wm = mk(Sv.um[6 * b + 3], Sv.um[6 * b + 4], Sv.um[6 * b + 5]);
    V3<double> dw = mk(Sv.u[6 * b + 3] - wm.x, Sv.u[6 * b + 4] - wm.y, Sv.u[6 * b + 5] - wm.z);
    V3<double> ww = mk(wu[6 * b + 3], wu[6 * b + 4], wu[6 * b + 5]);
    for (int k = 0; k < 3; ++k) {
      V3<double> rk = mk(Pm.R.a[0][k], Pm.R.a[1][k], Pm.R.a[2][k]);
      V3<double> d = rk * dot(rk, dw) + cross(wm, rk) * (h * dot(rk, wm));
      out.dinertia[3 * b + k] = dot(ww, d);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI (ctypes); single world per call, world-major arrays
// ---------------------------------------------------------------------------
extern "C" {

void oracle_set_trace(int t) { g_trace = t; }


int oracle_layout(const double* scene, const float* heights, int* out4) {
  OScene s;
  if (!parse_scene(scene, heights, s)) return 1;
  out4[0] = s.n_slots; out4[1] = s.m_max; out4[2] = s.n_state; out4[3] = s.n_servo;
  return 0;
}

// Forward step of one world.  info[0] = Newton iterations run, info[1] = sqrt(merit)
// of the returned iterate, info[2] = returned iterate index, info[3] = active rows.
int oracle_step(const double* scene, const float* heights, const double* cfgv, const double* state_in,
                const double* ubar, double h, double* state_out, double* impulses, int32_t* ids,
                uint32_t* status, double* info) {
  OScene s; OCfg cfg;
  if (!parse_scene(scene, heights, s)) return 1;
  parse_cfg(cfgv, cfg);
  Solver S;
  setup(S, s, cfg, state_in, ubar, h);
  solve_step(S);
  write_outputs(S, state_out, impulses, ids);
  if (status) *status = S.status;
  if (info) { info[0] = S.iters; info[1] = std::sqrt(S.merit); info[2] = S.ret_k; info[3] = (double)S.W.rows.size(); }
  return 0;
}

// Forward step plus adjoint (mode 0: paper, frozen W, forward Schur matrix;
// mode 1: exact IFT).  dL_dstate_next has the state layout; lambda entries ignored.
// dL_dkp (n_servo), dL_dmass (nb) and dL_dinertia (3 nb, body-frame principal moments), the
// servo-gain, body-mass and inertia gradients, and dL_dmu (1), the friction-coefficient
// gradient (zero in paper mode), may be null.
int oracle_step_adjoint(const double* scene, const float* heights, const double* cfgv, const double* state_in,
                        const double* ubar, double h, const double* dL_dnext, int mode, double* state_out,
                        double* impulses, int32_t* ids, uint32_t* status, double* dL_dstate, double* dL_dubar,
                        double* info, double* dL_dkp, double* dL_dmass, double* dL_dinertia, double* dL_dmu) {
  OScene s; OCfg cfg;
  if (!parse_scene(scene, heights, s)) return 1;
  parse_cfg(cfgv, cfg);
  Solver S;
  setup(S, s, cfg, state_in, ubar, h);
  solve_step(S);
  write_outputs(S, state_out, impulses, ids);
  if (status) *status = S.status;
  if (info) { info[0] = S.iters; info[1] = std::sqrt(S.merit); info[2] = S.ret_k; info[3] = (double)S.W.rows.size(); }
  AdjOut A;
  adjoint(S, dL_dnext, mode, A);
  for (int i = 0; i < 7 * s.nb; ++i) dL_dstate[i] = A.dq[i];
  for (int i = 0; i < 6 * s.nb; ++i) dL_dstate[7 * s.nb + i] = A.du[i];
  for (int i = 0; i < s.m_max; ++i) dL_dstate[13 * s.nb + i] = 0.0;
  for (int i = 0; i < s.n_servo; ++i) dL_dubar[i] = A.dubar[i];
  if (dL_dkp) for (int i = 0; i < s.n_servo; ++i) dL_dkp[i] = A.dkp[i];
  if (dL_dmass) for (int b = 0; b < s.nb; ++b) dL_dmass[b] = A.dmass[b];
  if (dL_dinertia) for (int i = 0; i < 3 * s.nb; ++i) dL_dinertia[i] = A.dinertia[i];
  if (dL_dmu) *dL_dmu = A.dmu;
  return 0;
}

// The adjoint (Sec. III-D) taken at a given returned iterate (u+, lambda+) of the step
// from state_in, instead of at the oracle's own solution: the paper evaluates A and the
// VJPs at whatever iterate the forward step returns, so this is the reference for an
// adjoint computed at another implementation's iterate.  lam_ret uses the state's
// lambda layout (m_max entries).
int oracle_adjoint_at(const double* scene, const float* heights, const double* cfgv, const double* state_in,
                      const double* ubar, double h, const double* u_ret, const double* lam_ret,
                      const double* dL_dnext, int mode, double* dL_dstate, double* dL_dubar, double* dL_dkp,
                      double* dL_dmass, double* dL_dinertia, double* dL_dmu) {
  OScene s; OCfg cfg;
  if (!parse_scene(scene, heights, s)) return 1;
  parse_cfg(cfgv, cfg);
  Solver S;
  setup(S, s, cfg, state_in, ubar, h);
  S.u.assign(u_ret, u_ret + 6 * s.nb);
  S.lam.assign(lam_ret, lam_ret + s.m_max);
  AdjOut A;
  adjoint(S, dL_dnext, mode, A);
  for (int i = 0; i < 7 * s.nb; ++i) dL_dstate[i] = A.dq[i];
  for (int i = 0; i < 6 * s.nb; ++i) dL_dstate[7 * s.nb + i] = A.du[i];
  for (int i = 0; i < s.m_max; ++i) dL_dstate[13 * s.nb + i] = 0.0;
  for (int i = 0; i < s.n_servo; ++i) dL_dubar[i] = A.dubar[i];
  if (dL_dkp) for (int i = 0; i < s.n_servo; ++i) dL_dkp[i] = A.dkp[i];
  if (dL_dmass) for (int b = 0; b < s.nb; ++b) dL_dmass[b] = A.dmass[b];
  if (dL_dinertia) for (int i = 0; i < 3 * s.nb; ++i) dL_dinertia[i] = A.dinertia[i];
  if (dL_dmu) *dL_dmu = A.dmu;
  return 0;
}

// Pieces exposed for the pins -------------------------------------------------
void oracle_fb(double a, double b, double eps, double* out3) {
  out3[0] = fb<double>(a, b, eps);
  fb_grad(a, b, eps, out3[1], out3[2]);
}

double oracle_friction_W(double vt1, double vt2, double ln, double lf1, double lf2, double mu, double eps,
                         double hw) {
  return friction_W<double>(vt1, vt2, ln, lf1, lf2, mu, eps, hw);
}

void oracle_rotate(const double* q, const double* v, double* out) {
  M3<double> R = rotmat(q);
  V3<double> r = mul(R, mk(v[0], v[1], v[2]));
  out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

int oracle_lu_solve(int n, const double* A, const double* b, double* x) {
  std::vector<double> AA(A, A + n * n), bb(b, b + n);
  bool ok = lu_solve(n, AA, bb);
  for (int i = 0; i < n; ++i) x[i] = bb[i];
  return ok ? 0 : 1;
}

// PCR on a dense system, for the pins: P from precond_matrix(kind, block) (block: n ids).
// Returns the iterations taken; conv_out (may be null) receives 1 when |r| <= rtol |b|.
int oracle_pcr(int n, const double* A, const double* b, int kind, const int32_t* block, int iters, double rtol,
               double* x, int32_t* conv_out) {
  std::vector<double> AA(A, A + n * n), bb(b, b + n), xx;
  std::vector<int> blk(block, block + n);
  const std::vector<double> P = precond_matrix(n, AA, blk, kind);
  bool conv = false;
  const int k = pcr(n, AA, P, bb, xx, iters, rtol, &conv);
  for (int i = 0; i < n; ++i) x[i] = xx[i];
  if (conv_out) *conv_out = conv ? 1 : 0;
  return k;
}

// Contact slot table at q-: per slot active flag, packed id, normal and offset.
int oracle_contacts(const double* scene, const float* heights, const double* cfgv, const double* state_in, double h,
                    int32_t* active, int32_t* ids, double* nd) {
  OScene s; OCfg cfg;
  if (!parse_scene(scene, heights, s)) return 1;
  parse_cfg(cfgv, cfg);
  std::vector<Contact> con; uint32_t st = 0;
  generate_contacts(s, cfg, state_in, state_in + 7 * s.nb, h, con, st);
  for (int sl = 0; sl < s.n_slots; ++sl) {
    active[sl] = con[sl].active; ids[sl] = con[sl].active ? con[sl].id : -1;
    nd[4 * sl] = con[sl].n[0]; nd[4 * sl + 1] = con[sl].n[1]; nd[4 * sl + 2] = con[sl].n[2]; nd[4 * sl + 3] = con[sl].d;
  }
  return 0;
}

// Rows at an arbitrary iterate (u, lambda) for a state's contact set: per active row
// [type, b0, b1, lam index], the analytic Jacobian (12), the dual-number derivative of
// the row function along each of the 12 body-velocity directions (12), the unscaled
// residual and C.  Returns the number of rows (<= max_rows) or -1.
int oracle_rows(const double* scene, const float* heights, const double* cfgv, const double* state_in,
                const double* ubar, double h, const double* u, const double* lam, int max_rows,
                int32_t* meta, double* Jan, double* Jdual, double* r, double* C, double* rdyn) {
  OScene s; OCfg cfg;
  if (!parse_scene(scene, heights, s)) return -1;
  parse_cfg(cfgv, cfg);
  Solver S;
  setup(S, s, cfg, state_in, ubar, h);
  int m = (int)S.W.rows.size();
  if (m > max_rows) return -1;
  Eval<double> E;
  evaluate<double>(S.W, S.qm.data(), S.um.data(), S.ubar.data(), u, lam, nullptr, false, nullptr, nullptr, E);
  int nb = s.nb;
  std::vector<double> qp(7 * nb);
  kin_update(nb, S.qm.data(), u, h, qp.data());
  for (int i = 0; i < m; ++i) {
    const Row& rw = S.W.rows[i];
    meta[4 * i] = rw.type; meta[4 * i + 1] = rw.b0; meta[4 * i + 2] = rw.b1; meta[4 * i + 3] = rw.lam;
    for (int k = 0; k < 6; ++k) { Jan[12 * i + k] = E.J[i].j0[k]; Jan[12 * i + 6 + k] = E.J[i].j1[k]; }
    r[i] = E.r[i]; C[i] = E.C[i];
    // Jdual: the definition of the row Jacobian, d/du of the row's position-level
    // function through q+(u) = q- + h G(q-) u, divided by h: the constraint value for
    // joint and normal rows, t . x for friction rows with x the material point at the
    // contact and t frozen; servo rows repeat the analytic value (not pinned here).
    Geo<double> Gv;
    geometry<double>(S.W, S.qm.data(), qp.data(), u, Gv);
    for (int side = 0; side < 2; ++side) {
      int b = side == 0 ? rw.b0 : rw.b1;
      for (int k = 0; k < 6; ++k) {
        double& out = Jdual[12 * i + 6 * side + k];
        if (b < 0) { out = 0.0; continue; }
        if (rw.type == ROW_SERVO) { out = Jan[12 * i + 6 * side + k]; continue; }
        std::vector<Dual> uD(6 * nb), qmD(7 * nb), qpD(7 * nb);
        for (int t = 0; t < 6 * nb; ++t) uD[t] = Dual(u[t], t == 6 * b + k ? 1.0 : 0.0);
        for (int t = 0; t < 7 * nb; ++t) qmD[t] = Dual(S.qm[t]);
        kin_update(nb, qmD.data(), uD.data(), h, qpD.data());
        Geo<Dual> G;
        geometry(S.W, qmD.data(), qpD.data(), uD.data(), G);
        if (rw.type == ROW_JOINT || rw.type == ROW_NORMAL) {
          out = row_position_value(S.W, rw, G).d / h;
        } else {
          const Pose<double>& Ps = Gv.P[rw.b0];
          V3<double> rho = mulT(Ps.R, Gv.x[rw.slot] - Ps.p);
          V3<Dual> xm = G.P[rw.b0].p + mul(G.P[rw.b0].R, mk(Dual(rho.x), Dual(rho.y), Dual(rho.z)));
          V3<double> t = rw.sub == 1 ? Gv.t1[rw.slot] : Gv.t2[rw.slot];
          out = (xm.x * Dual(t.x) + xm.y * Dual(t.y) + xm.z * Dual(t.z)).d / h;
        }
      }
    }
  }
  for (int i = 0; i < 6 * nb; ++i) rdyn[i] = E.rdyn[i];
  return m;
}

}  // extern "C"
