// Ostrich per-timestep solve and IFT adjoint for many independent worlds, sm_103a.
//
// One CTA runs one world; its whole working set (bodies, constraint rows, contact
// slots, Schur blocks) lives in shared memory.  The work follows the paper:
//   Sec. III-A  backward-Euler kinematics Eq. (1), implicit dynamics Eq. (2);
//   Sec. III-B  joint rows Eq. (3), FB normal contact Eq. (4), friction Eq. (7)
//               with the two cone safeguards, velocity servo Eq. (8);
//   Sec. III-C  kinematic substitution, Schur step Eq. (12), back-substitution
//               Eq. (13), best-iterate backtracking (optional line search);
//   Sec. III-D  adjoint Eqs. (16)-(19) with the forward Schur factor read back from
//               the tape, vector-Jacobian products Eq. (17) with the position
//               pull-back evaluated by forward-mode duals, one row at a time.
// The Schur matrix A = h J M^-1 J^T + C + delta I is never formed densely: rows are
// ordered contact rows first, grouped by body (each group touches one body only,
// so groups do not couple), then the joint/servo rows (the separator).  That block-
// arrowhead structure is factored as Cholesky of each group block, elimination of
// the group-separator coupling, then Cholesky of the reduced separator block.
//
// Included once per precision (ostrich_kernels_f32.cu, ostrich_kernels_f64.cu, which
// define OST_REAL) so that the two compile in parallel.
#include <cuda_runtime.h>
#include <stdint.h>
#include "ostrich_scene.h"
#include "ostrich_math.cuh"
#include "ostrich_contacts.cuh"

namespace ost {

// ---------------------------------------------------------------------------
// shared-memory layout of one world
// ---------------------------------------------------------------------------
template <class Real> struct WS {
  // bodies
  Real *qm, *um, *ubar, *uk, *ut, *ub, *du, *f, *rdyn, *mr, *Iw, *Iwi, *R, *qp;
  Real *sbc;      // per servo: the bias b_c of Eq. (8) (-target, or (x(q-) - target)/h)
  // rows
  Real *J, *C, *rhat, *r2, *lk, *lt, *lb, *dl, *rhs;
  int16_t *meta;  // 4 per row: type | sub << 4, b0, b1 (or -1), lam index (state lambda block)
  int16_t *ref;   // slot or joint of the row
  // slots
  Real *sn, *sd, *st1, *st2, *swhat, *srad, *sedge;
  int *sact, *srow, *sid, *sftype;
  // per-body row lists
  int *bgrp, *bsepn, *bsep;
  // groups
  int *g0, *gn;
  int16_t *rgrp;  // group of a contact row
  // Schur storage (block-arrowhead, inverse form): G group blocks, E coupling rows,
  // H = E G, S reduced separator; prow a pivot-row buffer per warp
  Real *G, *E, *H, *S, *prow, *tmp, *tmp2;
  // scratch
  Real *red;
  int *ints;      // [0] rows, [1] contact rows, [2] items, [3] converged, [4] best_k, [5] iters, [6] status,
                  // [7] contact-generation status bits (4: candidates beyond the slots)
  Real *scal;     // [0] merit cur, [1] best merit, [2] delta, [3] merit trial
  Real *pcr;      // PCR mode: r, z, p, A p, A z, P A p and the Jacobi diagonal, m_max each
};

template <class T> __host__ __device__ __forceinline__ T* carve(char*& p, int n) {
  size_t a = alignof(T) < 8 ? 8 : alignof(T);
  uintptr_t q = (reinterpret_cast<uintptr_t>(p) + a - 1) & ~(uintptr_t)(a - 1);
  T* r = reinterpret_cast<T*>(q);
  p = reinterpret_cast<char*>(q + sizeof(T) * (size_t)(n > 0 ? n : 1));
  return r;
}


template <class Real> __host__ __device__ WS<Real> ws_carve(char* base, const DevScene& s) {
  WS<Real> w;
  char* p = base;
  int nb = s.nb, m = s.m_max, ns = s.n_slots > 0 ? s.n_slots : 1, ng = s.n_groups > 0 ? s.n_groups : 1;
  int ss = s.ss > 0 ? s.ss : 1, pg = s.pg > 0 ? s.pg : 1;
  w.qm = carve<Real>(p, 7 * nb); w.um = carve<Real>(p, 6 * nb); w.ubar = carve<Real>(p, s.n_servo + 1);
  w.uk = carve<Real>(p, 6 * nb); w.ut = carve<Real>(p, 6 * nb); w.ub = carve<Real>(p, 6 * nb);
  w.du = carve<Real>(p, 6 * nb); w.f = carve<Real>(p, 6 * nb); w.rdyn = carve<Real>(p, 6 * nb);
  w.mr = carve<Real>(p, 6 * nb);
  w.Iw = carve<Real>(p, 9 * nb); w.Iwi = carve<Real>(p, 9 * nb); w.R = carve<Real>(p, 9 * nb);
  w.qp = carve<Real>(p, 7 * nb);
  w.sbc = carve<Real>(p, s.n_servo + 1);
  w.J = carve<Real>(p, 12 * m);
  w.C = carve<Real>(p, m); w.rhat = carve<Real>(p, m); w.r2 = carve<Real>(p, m); w.lk = carve<Real>(p, m);
  w.lt = carve<Real>(p, m); w.lb = carve<Real>(p, m); w.dl = carve<Real>(p, m); w.rhs = carve<Real>(p, m);
  w.meta = carve<int16_t>(p, 4 * m); w.ref = carve<int16_t>(p, m);
  w.sn = carve<Real>(p, 3 * ns); w.st1 = carve<Real>(p, 3 * ns); w.st2 = carve<Real>(p, 3 * ns);
  w.srad = carve<Real>(p, 3 * ns); w.sd = carve<Real>(p, ns); w.swhat = carve<Real>(p, ns);
  w.sedge = carve<Real>(p, 2 * ns);
  w.sact = carve<int>(p, ns); w.srow = carve<int>(p, ns); w.sid = carve<int>(p, ns); w.sftype = carve<int>(p, ns);
  w.bgrp = carve<int>(p, nb); w.bsepn = carve<int>(p, nb); w.bsep = carve<int>(p, nb * ss);
  w.g0 = carve<int>(p, ng); w.gn = carve<int>(p, ng); w.rgrp = carve<int16_t>(p, m);
  int cm = s.cmax > 0 ? s.cmax : 1, ldg = s.ldg > 0 ? s.ldg : 1;
  int esz = ng * cm * ldg;
  int gsz = ng * tri_size(pg), rest = esz + ng * cm * ldg + tri_size(ss);
  if (gsz + rest < 14 * m) gsz = 14 * m - rest;
  w.G = carve<Real>(p, gsz); w.E = carve<Real>(p, esz); w.H = carve<Real>(p, ng * cm * ldg);
  w.S = carve<Real>(p, tri_size(ss));
  w.prow = carve<Real>(p, 4 * (pg > ss ? pg : ss));
  w.tmp = carve<Real>(p, m); w.tmp2 = carve<Real>(p, m);
  w.red = carve<Real>(p, 64); w.ints = carve<int>(p, 16); w.scal = carve<Real>(p, 8);
  w.pcr = s.lin == LIN_PCR ? carve<Real>(p, 7 * m) : nullptr;
  return w;
}

// Dynamic shared memory of one world: the carve itself, run from a 16-byte aligned base
// (the dynamic shared-memory base is 16-byte aligned and carve aligns to 8), rounded up
// to 16 bytes.
template <class Real> __host__ __device__ size_t ws_bytes(const DevScene& s) {
  char* base = reinterpret_cast<char*>(uintptr_t(16));
  WS<Real> w = ws_carve<Real>(base, s);
  size_t used = (size_t)(reinterpret_cast<char*>(w.pcr ? w.pcr + 7 * s.m_max : w.scal + 8) - base);
  return (used + 15) & ~(size_t)15;
}

// deterministic block reduction (fixed tree); result broadcast through w.red[0]
template <class Real> __device__ Real block_sum(WS<Real>& w, Real v) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) w.red[wid] = v;
  __syncthreads();
  if (tid == 0) {
    Real acc = Real(0);
    for (int i = 0; i < nw; ++i) acc += w.red[i];
    w.red[32] = acc;
  }
  __syncthreads();
  return w.red[32];
}

// two deterministic block sums at once (fixed tree, as block_sum): results in a, b
template <class Real> __device__ void block_sum2(WS<Real>& w, Real& a, Real& b) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) { w.red[wid] = a; w.red[16 + wid] = b; }
  __syncthreads();
  if (tid == 0) {
    Real sa = Real(0), sb = Real(0);
    for (int i = 0; i < nw; ++i) { sa += w.red[i]; sb += w.red[16 + i]; }
    w.red[32] = sa; w.red[48] = sb;
  }
  __syncthreads();
  a = w.red[32];
  b = w.red[48];
}

// block maximum (every thread gets it), through w.red[33..]
template <class Real> __device__ Real block_max(WS<Real>& w, Real v) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) w.red[33 + wid] = v;
  __syncthreads();
  Real mx = w.red[33];
  for (int i = 1; i < nw; ++i) mx = fmax(mx, w.red[33 + i]);
  __syncthreads();
  return mx;
}

// two block maxima at once (every thread gets both), through w.red[40..] and w.red[56..]
template <class Real> __device__ void block_max2(WS<Real>& w, Real& a, Real& b) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  __syncthreads();
  if (lane == 0) { w.red[40 + wid] = a; w.red[56 + wid] = b; }
  __syncthreads();
  Real ma = w.red[40], mb = w.red[56];
  for (int i = 1; i < nw; ++i) { ma = fmax(ma, w.red[40 + i]); mb = fmax(mb, w.red[56 + i]); }
  __syncthreads();
  a = ma;
  b = mb;
}

// ---------------------------------------------------------------------------
// geometry helpers in any scalar type S
// ---------------------------------------------------------------------------
template <class S> __device__ __forceinline__ void tangent_basis(vec3<S> n, vec3<S>& t1, vec3<S>& t2) {
  vec3<S> e = fabs((double)sval(n.x)) < 0.9 ? v3(S(1), S(0), S(0)) : v3(S(0), S(1), S(0));
  vec3<S> t = e - scale(n, dot3(n, e));
  S l = ssqrt(dot3(t, t));
  t1 = scale(t, S(1) / l);
  t2 = cross3(n, t1);
}

// contact point on body b at pose (p, q) for slot kind: box corner (material point) or
// rim (deepest point of the rim circle along -n)
template <class S> __device__ __forceinline__ vec3<S> slot_point(const DevScene& sc, int b, int local, vec3<S> p,
                                                                 const S* q, vec3<S> n) {
  if (sc.shape[b] == SHAPE_BOX) {
    int k = local;
    vec3<S> rb = v3(S((k & 1) ? sc.half[b][0] : -sc.half[b][0]), S((k & 2) ? sc.half[b][1] : -sc.half[b][1]),
                    S((k & 4) ? sc.half[b][2] : -sc.half[b][2]));
    return p + qrot(q, rb);
  }
  int rim = local / sc.nf;
  vec3<S> a = qrot(q, v3(S(0), S(1), S(0)));
  vec3<S> cen = p + qrot(q, v3(S(0), S(rim ? sc.hw[b] : -sc.hw[b]), S(0)));
  S nd = dot3(n, a);
  vec3<S> perp = n - scale(a, nd);
  S pl = ssqrt(dot3(perp, perp));
  if ((double)sval(pl) <= 1e-12) return cen;
  return cen - scale(perp, S(sc.radius[b]) / pl);
}

// frame (n, d) of a slot: fixed plane, or box edge with normal toward the rim centre at q-
template <class S, class Real> __device__ __forceinline__ void slot_frame2(const DevScene& sc, int b, int local, int ftype,
                                                                           const S* qm7, const Real* nstore, Real dstore,
                                                                           const Real* edge, vec3<S>& n, S& d) {
  if (ftype == 1) {
    int rim = local / sc.nf;
    vec3<S> p = v3(qm7[0], qm7[1], qm7[2]);
    vec3<S> cen = p + qrot(qm7 + 3, v3(S(0), S(rim ? sc.hw[b] : -sc.hw[b]), S(0)));
    S dx = cen.x - S(edge[0]), dz = cen.z - S(edge[1]);
    S len = ssqrt(dx * dx + dz * dz);
    n = v3(dx / len, S(0), dz / len);
    d = n.x * S(edge[0]) + n.z * S(edge[1]);
  } else {
    n = v3(S(nstore[0]), S(nstore[1]), S(nstore[2]));
    d = S(dstore);
  }
}

// ---------------------------------------------------------------------------
// joint geometry in any scalar type S, from body positions and rotation matrices
// ---------------------------------------------------------------------------
// Body-frame to world rotations for the joint helpers: a rotation matrix (the step's
// R(q) in shared memory) or a quaternion normalised once (the adjoint's dual numbers, where
// nine matrix entries per body would cost registers).
template <class S> struct MatRot {
  const S* R;
  __device__ __forceinline__ vec3<S> operator()(vec3<S> v) const { return mat3<S>(R, v); }
};
template <class S> struct QuatRot {
  S w;
  vec3<S> qv;
  __device__ __forceinline__ explicit QuatRot(const S* q) {
    const S inv = S(1) / ssqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    w = q[0] * inv;
    qv = v3(q[1] * inv, q[2] * inv, q[3] * inv);
  }
  // v + w t + qv x t, t = 2 qv x v (the rotation of qrot, with the normalisation done once)
  __device__ __forceinline__ vec3<S> operator()(vec3<S> v) const {
    vec3<S> t = cross3(qv, v);
    t = v3(t.x + t.x, t.y + t.y, t.z + t.z);
    const vec3<S> c = cross3(qv, t);
    return v3(v.x + w * t.x + c.x, v.y + w * t.y + c.y, v.z + w * t.z + c.z);
  }
};

template <class S> __device__ __forceinline__ vec3<S> cvec(const double* a) { return v3(S(a[0]), S(a[1]), S(a[2])); }

// The five rows of joint j (Eq. (3)): Jacobian parts before the rotation-rate map E and the
// constraint values, handed row by row (k = 0..4) to f(k, lin_p, ang_p, lin_c, ang_c, c) so
// that a caller contracts or stores each row without holding all five (each intermediate
// lives only as long as its rows need it).  rotp / rotc: the parent's / child's rotation.
// Revolute: anchor rows (p_p + r_p) - (p_c + r_c) by component, then the alignment rows
// perp_k,p . axis_c.  Prismatic: b_k . d (b_k = R_p perp_k, d = (p_c + r_c) - (p_p + r_p)),
// the alignment rows, and the twist lock perp2_p . perp1_c.
template <class S, class RP, class RC, class F>
__device__ __forceinline__ void joint_rows_each(const DevScene& sc, int j, vec3<S> pp, const RP& rotp, vec3<S> pc,
                                                const RC& rotc, F&& f) {
  const vec3<S> z = v3(S(0.0), S(0.0), S(0.0));
  if (sc.jtype[j] == JOINT_REVOLUTE) {
    {
      const vec3<S> rp = rotp(cvec<S>(sc.ap[j])), rc = rotc(cvec<S>(sc.ac[j]));
      const vec3<S> d = (pc + rc) - (pp + rp);
      const vec3<S> ex = v3(S(1.0), S(0.0), S(0.0)), ey = v3(S(0.0), S(1.0), S(0.0)), ez = v3(S(0.0), S(0.0), S(1.0));
      f(0, ex, cross3(rp, ex), scale(ex, S(-1.0)), scale(cross3(rc, ex), S(-1.0)), S(0.0) - d.x);
      f(1, ey, cross3(rp, ey), scale(ey, S(-1.0)), scale(cross3(rc, ey), S(-1.0)), S(0.0) - d.y);
      f(2, ez, cross3(rp, ez), scale(ez, S(-1.0)), scale(cross3(rc, ez), S(-1.0)), S(0.0) - d.z);
    }
    const vec3<S> aw = rotc(cvec<S>(sc.axc[j]));
    {
      const vec3<S> b1 = rotp(cvec<S>(sc.p1[j]));
      const vec3<S> a1 = cross3(b1, aw);
      f(3, z, a1, z, scale(a1, S(-1.0)), dot3(b1, aw));
    }
    const vec3<S> b2 = rotp(cvec<S>(sc.p2[j]));
    const vec3<S> a2 = cross3(b2, aw);
    f(4, z, a2, z, scale(a2, S(-1.0)), dot3(b2, aw));
  } else {
    const vec3<S> b1 = rotp(cvec<S>(sc.p1[j])), b2 = rotp(cvec<S>(sc.p2[j]));
    {
      const vec3<S> rp = rotp(cvec<S>(sc.ap[j])), rc = rotc(cvec<S>(sc.ac[j]));
      const vec3<S> d = (pc + rc) - (pp + rp);
      const vec3<S> dr = d + rp;
      f(0, scale(b1, S(-1.0)), cross3(b1, dr), b1, cross3(rc, b1), dot3(b1, d));
      f(1, scale(b2, S(-1.0)), cross3(b2, dr), b2, cross3(rc, b2), dot3(b2, d));
    }
    {
      const vec3<S> aw = rotc(cvec<S>(sc.axc[j]));
      const vec3<S> a1 = cross3(b1, aw), a2 = cross3(b2, aw);
      f(2, z, a1, z, scale(a1, S(-1.0)), dot3(b1, aw));
      f(3, z, a2, z, scale(a2, S(-1.0)), dot3(b2, aw));
    }
    const vec3<S> e1 = rotc(cvec<S>(sc.p1[j]));
    const vec3<S> a3 = cross3(b2, e1);
    f(4, z, a3, z, scale(a3, S(-1.0)), dot3(b2, e1));
  }
}

// The same five rows held in one structure (for callers that need them all at once)
template <class S> struct JRows {
  vec3<S> lin_p[5], ang_p[5], lin_c[5], ang_c[5];
  S c[5];
};

template <class S, class RP, class RC>
__device__ __forceinline__ void joint_rows_geom(const DevScene& sc, int j, vec3<S> pp, const RP& rotp, vec3<S> pc,
                                                const RC& rotc, JRows<S>& o) {
  joint_rows_each<S>(sc, j, pp, rotp, pc, rotc, [&](int k, vec3<S> lp, vec3<S> ap, vec3<S> lc, vec3<S> ac, S c) {
    o.lin_p[k] = lp; o.ang_p[k] = ap; o.lin_c[k] = lc; o.ang_c[k] = ac; o.c[k] = c;
  });
}

// Servo row of joint j (Eq. (8)): Jacobian parts before E of the joint rate, the relative
// angular velocity about the parent axis (revolute) or the slide rate d/dt (a . d)
// (prismatic).
template <class S> struct SRow { vec3<S> lin_p, ang_p, lin_c, ang_c; };

template <class S, class RP, class RC>
__device__ __forceinline__ void servo_row_geom(const DevScene& sc, int j, vec3<S> pp, const RP& rotp, vec3<S> pc,
                                               const RC& rotc, SRow<S>& o) {
  const vec3<S> a = rotp(cvec<S>(sc.axp[j]));
  if (sc.jtype[j] == JOINT_REVOLUTE) {
    o.lin_p = v3(S(0.0), S(0.0), S(0.0)); o.lin_c = o.lin_p;
    o.ang_p = scale(a, S(-1.0)); o.ang_c = a;
  } else {
    const vec3<S> rp = rotp(cvec<S>(sc.ap[j])), rc = rotc(cvec<S>(sc.ac[j]));
    const vec3<S> d = (pc + rc) - (pp + rp);
    o.lin_p = scale(a, S(-1.0)); o.ang_p = cross3(a, d + rp);
    o.lin_c = a; o.ang_c = cross3(rc, a);
  }
}

// The joint coordinate a position servo tracks: the revolute angle about the parent axis a
// from perp1_p to the child's perp1 (atan2), or the prismatic slide a . d.
__device__ __forceinline__ float satan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double satan2(double y, double x) { return atan2(y, x); }
template <class T> __device__ __forceinline__ dual<T> satan2(dual<T> y, dual<T> x) {
  const T r2 = x.v * x.v + y.v * y.v;
  return dual<T>(satan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}

template <class S, class RP, class RC>
__device__ __forceinline__ S joint_coord(const DevScene& sc, int j, vec3<S> pp, const RP& rotp, vec3<S> pc,
                                         const RC& rotc) {
  const vec3<S> a = rotp(cvec<S>(sc.axp[j]));
  if (sc.jtype[j] == JOINT_REVOLUTE) {
    const vec3<S> f = rotp(cvec<S>(sc.p1[j]));
    const vec3<S> e = rotc(cvec<S>(sc.p1[j]));
    return satan2(dot3(e, cross3(a, f)), dot3(e, f));
  }
  const vec3<S> rp = rotp(cvec<S>(sc.ap[j])), rc = rotc(cvec<S>(sc.ac[j]));
  return dot3(a, (pc + rc) - (pp + rp));
}

// Servo compliance alpha of Eq. (8): 1/kp (velocity target), 1/(kd + h kp) (position).
__device__ __forceinline__ double servo_alpha(const DevScene& sc, int j, double h) {
  return sc.smode[j] == SERVO_POSITION ? 1.0 / (sc.kd[j] + h * sc.kp[j]) : 1.0 / sc.kp[j];
}

// Joint of the k-th servo.
__device__ __forceinline__ int servo_joint(const DevScene& sc, int k) {
  int j = 0, cnt = -1;
  for (j = 0; j < sc.nj; ++j) if (sc.servo_of[j] >= 0 && ++cnt == k) break;
  return j;
}

// ---------------------------------------------------------------------------
// per-world setup: load inputs, contacts, rows, masses, warm start
// ---------------------------------------------------------------------------
// element i of an input vector lives at p[i * stride] (stride = ld for the structure-of-
// arrays state, 1 for a tape record)
template <class Real> struct Src { const Real* p; size_t stride; };

// Asynchronous global -> shared copy of one element (cp.async, cached in L1), committed
// as a group and awaited before use, so that the copies proceed while the CTA computes.
template <class Real> __device__ __forceinline__ void cp_async_elem(Real* smem_dst, const Real* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (sizeof(Real) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Integers in a tape of Real elements, bit for bit: the bits of a float, or the value of a
// double (exact for every int).
__device__ __forceinline__ float tape_from_int(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double tape_from_int(int v, double) { return (double)v; }
__device__ __forceinline__ int tape_to_int(float v) { return __float_as_int(v); }
__device__ __forceinline__ int tape_to_int(double v) { return (int)v; }

// ct_out: when not null, the contact slot table of this step is recorded there (a tape
// record's slot table); ct_in: when not null, the table is read from there instead of
// running the activation (the adjoint, at the taped step: the same set by construction).
template <class Real>
__device__ void world_setup(const DevScene& sc, WS<Real>& w, Src<Real> qmv, Src<Real> umv, Src<Real> ubarv,
                            double h, Real* ct_out = nullptr, const Real* ct_in = nullptr) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int nb = sc.nb;
  for (int i = tid; i < 7 * nb; i += nth) w.qm[i] = qmv.p[i * qmv.stride];
  for (int i = tid; i < 6 * nb; i += nth) w.um[i] = umv.p[i * umv.stride];
  for (int i = tid; i < sc.n_servo; i += nth) w.ubar[i] = ubarv.p[i * ubarv.stride];
  __syncthreads();
  // contact activation (FP32 predicate) and slot frames in working precision
  auto store_slot = [&](int sl, int b, int local, const SlotAct& a) {
    w.sact[sl] = a.active; w.sid[sl] = a.id; w.sftype[sl] = a.ftype;
    w.sedge[2 * sl] = (Real)a.ex; w.sedge[2 * sl + 1] = (Real)a.ez;
    vec3<Real> n; Real d;
    Real ns[3] = {(Real)a.n[0], (Real)a.n[1], (Real)a.n[2]};
    slot_frame2<Real, Real>(sc, b, local, a.ftype, w.qm + 7 * b, ns, (Real)a.d, w.sedge + 2 * sl, n, d);
    vec3<Real> t1, t2;
    tangent_basis(n, t1, t2);
    w.sn[3 * sl] = n.x; w.sn[3 * sl + 1] = n.y; w.sn[3 * sl + 2] = n.z; w.sd[sl] = d;
    w.st1[3 * sl] = t1.x; w.st1[3 * sl + 1] = t1.y; w.st1[3 * sl + 2] = t1.z;
    w.st2[3 * sl] = t2.x; w.st2[3 * sl + 1] = t2.y; w.st2[3 * sl + 2] = t2.z;
    if (ct_out) {
      Real* c = ct_out + CT_PER_SLOT * sl;
      c[0] = tape_from_int(a.active, Real(0)); c[1] = tape_from_int(a.id, Real(0)); c[2] = tape_from_int(a.ftype, Real(0));
      c[3] = Real(a.n[0]); c[4] = Real(a.n[1]); c[5] = Real(a.n[2]); c[6] = Real(a.d);
      c[7] = Real(a.ex); c[8] = Real(a.ez);
    }
  };
  if (tid == 0) w.ints[7] = 0;
  __syncthreads();
  if (ct_in) {
    for (int sl = tid; sl < sc.n_slots; sl += nth) {
      const Real* c = ct_in + CT_PER_SLOT * sl;
      SlotAct a;
      a.active = tape_to_int(c[0]); a.id = tape_to_int(c[1]); a.ftype = tape_to_int(c[2]);
      a.n[0] = (float)c[3]; a.n[1] = (float)c[4]; a.n[2] = (float)c[5]; a.d = (float)c[6];
      a.ex = (float)c[7]; a.ez = (float)c[8];
      const int b = sc.slot_body[sl];
      store_slot(sl, b, sl - sc.slot_base[b], a);
    }
  } else if (sc.env == ENV_HEIGHTMAP) {
    // one thread per wheel rim: the rim's candidate faces fill its nf slots in order
    for (int e = tid; e < 2 * nb; e += nth) {
      const int b = e >> 1, rim = e & 1;
      if (sc.shape[b] != SHAPE_WHEEL) continue;
      float q7[7], u6[6];
      for (int k = 0; k < 7; ++k) q7[k] = (float)w.qm[7 * b + k];
      for (int k = 0; k < 6; ++k) u6[k] = (float)w.um[6 * b + k];
      SlotAct acts[8];
      if (activate_rim_hm(sc, b, rim, q7, u6, h, acts)) atomicOr(&w.ints[7], 4);
      for (int f = 0; f < sc.nf; ++f) store_slot(sc.slot_base[b] + rim * sc.nf + f, b, rim * sc.nf + f, acts[f]);
    }
    for (int sl = tid; sl < sc.n_slots; sl += nth)      // box corners (no wheel rim)
      if (sc.shape[sc.slot_body[sl]] != SHAPE_WHEEL) {
        int b = sc.slot_body[sl];
        float q7[7], u6[6];
        for (int k = 0; k < 7; ++k) q7[k] = (float)w.qm[7 * b + k];
        for (int k = 0; k < 6; ++k) u6[k] = (float)w.um[6 * b + k];
        store_slot(sl, b, sl - sc.slot_base[b], activate_slot(sc, b, sl - sc.slot_base[b], q7, u6, h));
      }
  } else {
    for (int sl = tid; sl < sc.n_slots; sl += nth) {
      int b = sc.slot_body[sl];
      int local = sl - sc.slot_base[b];
      float q7[7], u6[6];
      for (int k = 0; k < 7; ++k) q7[k] = (float)w.qm[7 * b + k];
      for (int k = 0; k < 6; ++k) u6[k] = (float)w.um[6 * b + k];
      store_slot(sl, b, local, activate_slot(sc, b, local, q7, u6, h));
    }
  }
  // bodies: world inertia at q-, external force, warm-start velocity
  for (int b = tid; b < nb; b += nth) {
    Real R[9];
    qmat(w.qm + 7 * b + 3, R);
    for (int k = 0; k < 9; ++k) w.R[9 * b + k] = R[k];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Real a = 0, ai = 0;
        for (int k = 0; k < 3; ++k) {
          a += R[3 * i + k] * Real(sc.inertia[b][k]) * R[3 * j + k];
          ai += R[3 * i + k] * (Real(1) / Real(sc.inertia[b][k])) * R[3 * j + k];
        }
        w.Iw[9 * b + 3 * i + j] = a; w.Iwi[9 * b + 3 * i + j] = ai;
      }
    Real m = Real(sc.mass[b]);
    vec3<Real> om = v3(w.um[6 * b + 3], w.um[6 * b + 4], w.um[6 * b + 5]);
    vec3<Real> Io = mat3<Real>(w.Iw + 9 * b, om);
    vec3<Real> gy = cross3(om, Io);
    w.f[6 * b] = 0; w.f[6 * b + 1] = 0; w.f[6 * b + 2] = m * Real(sc.g);
    w.f[6 * b + 3] = -gy.x; w.f[6 * b + 4] = -gy.y; w.f[6 * b + 5] = -gy.z;
    vec3<Real> dw = mat3<Real>(w.Iwi + 9 * b, v3(w.f[6 * b + 3], w.f[6 * b + 4], w.f[6 * b + 5]));
    w.uk[6 * b] = w.um[6 * b];
    w.uk[6 * b + 1] = w.um[6 * b + 1];
    w.uk[6 * b + 2] = w.um[6 * b + 2] + Real(h) * Real(sc.g);
    w.uk[6 * b + 3] = w.um[6 * b + 3] + Real(h) * dw.x;
    w.uk[6 * b + 4] = w.um[6 * b + 4] + Real(h) * dw.y;
    w.uk[6 * b + 5] = w.um[6 * b + 5] + Real(h) * dw.z;
  }
  __syncthreads();
  // servo biases b_c of Eq. (8): -target (velocity target) or (x(q-) - target)/h (position
  // target, x the joint coordinate at the step's start; w.R holds R(q-) here)
  for (int k = tid; k < sc.n_servo; k += nth) {
    const int j = servo_joint(sc, k), bp = sc.jp[j], bc = sc.jc[j];
    if (sc.smode[j] == SERVO_POSITION) {
      const Real x = joint_coord<Real>(sc, j, v3(w.qm[7 * bp], w.qm[7 * bp + 1], w.qm[7 * bp + 2]),
                                       MatRot<Real>{w.R + 9 * bp},
                                       v3(w.qm[7 * bc], w.qm[7 * bc + 1], w.qm[7 * bc + 2]), MatRot<Real>{w.R + 9 * bc});
      w.sbc[k] = (x - w.ubar[k]) / Real(h);
    } else {
      w.sbc[k] = -w.ubar[k];
    }
  }
  // row compaction, fixed order: the contact rows of the active slots in slot order (so
  // grouped by body), then the separator rows.  A slot's first row is 3 x the number of
  // active slots before it: warp ballots over the slot table (at most 64 slots) give the
  // prefix counts, and each lane writes its own slot's rows.
  if (tid < 32) {
    const int lane = tid, ns = sc.n_slots;
    const unsigned m0 = __ballot_sync(0xffffffffu, lane < ns && w.sact[lane]);
    const unsigned m1 = __ballot_sync(0xffffffffu, 32 + lane < ns && w.sact[32 + lane]);
    const int c0 = __popc(m0);
    for (int c = 0; c < 2; ++c) {
      const int sl = 32 * c + lane;
      if (sl >= ns) continue;
      const unsigned mk = c == 0 ? m0 : m1;
      if (!((mk >> lane) & 1u)) { w.srow[sl] = -1; continue; }
      const int r0 = 3 * ((c == 0 ? 0 : c0) + __popc(mk & ((1u << lane) - 1u)));
      const int bb = sc.slot_body[sl];
      w.srow[sl] = r0;
      const int lam = 5 * sc.nj + sc.n_servo + 3 * sl;
      int gb = 0;
      while (sc.group_body[gb] != bb) ++gb;
      for (int k = 0; k < 3; ++k) {
        const int r = r0 + k;
        w.meta[4 * r] = (k == 0 ? ROW_NORMAL : ROW_FRIC) | (k << 4); w.meta[4 * r + 1] = bb; w.meta[4 * r + 2] = -1;
        w.meta[4 * r + 3] = lam + k;
        w.ref[r] = sl;
        w.rgrp[r] = gb;
      }
    }
    // groups: first row and row count of each body's slots
    for (int g = lane; g < sc.n_groups; g += 32) {
      const int bb = sc.group_body[g], lo = sc.slot_base[bb], hi = lo + sc.slot_count[bb];
      auto before = [&](int x) {   // active slots with index < x
        const unsigned lo0 = x >= 32 ? m0 : (m0 & ((1u << x) - 1u));
        const unsigned lo1 = x <= 32 ? 0u : (x >= 64 ? m1 : (m1 & ((1u << (x - 32)) - 1u)));
        return __popc(lo0) + __popc(lo1);
      };
      w.g0[g] = 3 * before(lo);
      w.gn[g] = 3 * (before(hi) - before(lo));
    }
    if (lane == 0) {
      const int mc = 3 * (c0 + __popc(m1));
      w.ints[1] = mc;
      w.ints[0] = mc + sc.ss;
    }
  }
  __syncthreads();
  {
    const int mc = w.ints[1];
    // separator rows: five per joint, then one per servo
    for (int a = tid; a < sc.ss; a += nth) {
      const int r = mc + a;
      if (a < 5 * sc.nj) {
        const int j = a / 5, k = a - 5 * j;
        w.meta[4 * r] = ROW_JOINT | (k << 4); w.meta[4 * r + 1] = sc.jp[j]; w.meta[4 * r + 2] = sc.jc[j];
        w.meta[4 * r + 3] = 5 * j + k; w.ref[r] = j;
      } else {
        const int j = servo_joint(sc, a - 5 * sc.nj);
        w.meta[4 * r] = ROW_SERVO; w.meta[4 * r + 1] = sc.jp[j]; w.meta[4 * r + 2] = sc.jc[j];
        w.meta[4 * r + 3] = 5 * sc.nj + sc.servo_of[j]; w.ref[r] = j;
      }
    }
    // per-body lists: its group and the separator rows that touch it, in row order
    const int ssd = sc.ss > 0 ? sc.ss : 1;
    for (int bb = tid; bb < nb; bb += nth) {
      int gb = -1;
      for (int g = 0; g < sc.n_groups; ++g) if (sc.group_body[g] == bb) gb = g;
      w.bgrp[bb] = gb;
      int cnt = 0;
      for (int a2 = 0; a2 < sc.ss; ++a2) {
        const int j = a2 < 5 * sc.nj ? a2 / 5 : servo_joint(sc, a2 - 5 * sc.nj);
        if (sc.jp[j] == bb || sc.jc[j] == bb) w.bsep[bb * ssd + cnt++] = mc + a2;
      }
      w.bsepn[bb] = cnt;
    }
  }
  __syncthreads();
  // normal-row scaling what = J_n M^-1 J_n^T at q- (geometric Jacobian, E = I)
  for (int sl = tid; sl < sc.n_slots; sl += nth) {
    if (!w.sact[sl]) { w.swhat[sl] = 0; continue; }
    int b = w.meta[4 * w.srow[sl] + 1];
    int local = sl - sc.slot_base[b];
    vec3<Real> n = v3(w.sn[3 * sl], w.sn[3 * sl + 1], w.sn[3 * sl + 2]);
    vec3<Real> p = v3(w.qm[7 * b], w.qm[7 * b + 1], w.qm[7 * b + 2]);
    vec3<Real> x = slot_point<Real>(sc, b, local, p, w.qm + 7 * b + 3, n);
    vec3<Real> a = cross3(x - p, n);
    vec3<Real> ia = mat3<Real>(w.Iwi + 9 * b, a);
    w.swhat[sl] = Real(1) / Real(sc.mass[b]) + dot3(a, ia);
  }
  __syncthreads();
}

template <class Real> __device__ __forceinline__ void clamp_cone(const DevScene& sc, WS<Real>& w, Real* lam) {
  // first safeguard of Sec. III-B: |lambda_f| <= mu lambda_n
  for (int sl = threadIdx.x; sl < sc.n_slots; sl += blockDim.x) {
    if (!w.sact[sl]) continue;
    int i = w.srow[sl];
    Real rad = Real(sc.mu) * (lam[i] > Real(0) ? lam[i] : Real(0));
    Real nn = ssqrt(lam[i + 1] * lam[i + 1] + lam[i + 2] * lam[i + 2]);
    if (nn > rad) {
      Real f = nn > Real(0) ? rad / nn : Real(0);
      lam[i + 1] *= f; lam[i + 2] *= f;
    }
  }
}

template <class Real> __device__ __forceinline__ Real rowdot(const Real* Ja, int sa, const Real* Yb, int sb) {
  return Ja[sa] * Yb[sb] + Ja[sa + 1] * Yb[sb + 1] + Ja[sa + 2] * Yb[sb + 2] + Ja[sa + 3] * Yb[sb + 3] +
         Ja[sa + 4] * Yb[sb + 4] + Ja[sa + 5] * Yb[sb + 5];
}

// y = M^-1 J_i^T for both body blocks of row i: (J_lin / m, Iw^-1 J_ang) per side (zero
// for a side without a body); the same values Eq. (2)'s M~^-1 gives the row.
template <class Real> __device__ __forceinline__ void minv_row(const DevScene& sc, const WS<Real>& w, int i, Real* y) {
  const Real* Jr = w.J + 12 * i;
  for (int side = 0; side < 2; ++side) {
    const int b = w.meta[4 * i + 1 + side];
    Real* ys = y + 6 * side;
    if (b < 0) { for (int q = 0; q < 6; ++q) ys[q] = Real(0); continue; }
    const Real* Js = Jr + 6 * side;
    const Real mi = Real(1) / Real(sc.mass[b]);
    ys[0] = Js[0] * mi; ys[1] = Js[1] * mi; ys[2] = Js[2] * mi;
    const vec3<Real> ia = mat3<Real>(w.Iwi + 9 * b, v3(Js[3], Js[4], Js[5]));
    ys[3] = ia.x; ys[4] = ia.y; ys[5] = ia.z;
  }
}

// ---------------------------------------------------------------------------
// one residual / Jacobian evaluation at iterate (u, lam); returns the merit
// ---------------------------------------------------------------------------
// dyn = false (the adjoint): the rows, their compliance and delta only; the dynamics
// residual and the merit are not formed (the returned merit is 0).
template <class Real>
__device__ Real evaluate(const DevScene& sc, WS<Real>& w, const Real* u, const Real* lam, double h, bool dyn = true) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int nb = sc.nb, m = w.ints[0], mc = w.ints[1];
  const Real hR = Real(h);
  // poses at q+ = q- + h G(q-) u
  for (int b = tid; b < nb; b += nth) {
    kin_body<Real, Real>(w.qm + 7 * b, u + 6 * b, h, w.qp + 7 * b);
    qmat(w.qp + 7 * b + 3, w.R + 9 * b);
  }
  __syncthreads();
  const int n_items = sc.n_slots + sc.nj + sc.n_servo;
  for (int it = tid; it < n_items; it += nth) {
    if (it < sc.n_slots) {
      int sl = it;
      if (!w.sact[sl]) continue;
      int i = w.srow[sl];
      int b = w.meta[4 * i + 1];
      int local = sl - sc.slot_base[b];
      vec3<Real> p = v3(w.qp[7 * b], w.qp[7 * b + 1], w.qp[7 * b + 2]);
      vec3<Real> n = v3(w.sn[3 * sl], w.sn[3 * sl + 1], w.sn[3 * sl + 2]);
      vec3<Real> t1 = v3(w.st1[3 * sl], w.st1[3 * sl + 1], w.st1[3 * sl + 2]);
      vec3<Real> t2 = v3(w.st2[3 * sl], w.st2[3 * sl + 1], w.st2[3 * sl + 2]);
      vec3<Real> x = slot_point<Real>(sc, b, local, p, w.qp + 7 * b + 3, n);
      vec3<Real> lev = x - p;
      vec3<Real> wk = v3(u[6 * b + 3], u[6 * b + 4], u[6 * b + 5]);
      vec3<Real> dirs[3] = {n, t1, t2};
      Real vel[3];
      const MapE<Real> Ek(wk, h);
      for (int k = 0; k < 3; ++k) {
        vec3<Real> ang = Ek(cross3(lev, dirs[k]));
        Real* Jr = w.J + 12 * (i + k);
        Jr[0] = dirs[k].x; Jr[1] = dirs[k].y; Jr[2] = dirs[k].z; Jr[3] = ang.x; Jr[4] = ang.y; Jr[5] = ang.z;
        for (int q = 6; q < 12; ++q) Jr[q] = 0;
        vel[k] = dirs[k].x * u[6 * b] + dirs[k].y * u[6 * b + 1] + dirs[k].z * u[6 * b + 2] + ang.x * u[6 * b + 3] +
                 ang.y * u[6 * b + 4] + ang.z * u[6 * b + 5];
      }
      const Real kap = Real(sc.kappa), eps = Real(sc.eps);
      const Real hw = hR * w.swhat[sl];
      // normal row, Eq. (4): phi_eps(c_n/h + kappa lambda_n, h what lambda_n)
      Real cn = dot3(n, x) - w.sd[sl];
      Real ln = lam[i], l1 = lam[i + 1], l2 = lam[i + 2];
      Real a = cn / hR + kap * ln, bb = hw * ln;
      // At an active contact b = h what lambda_n is large (~10 m/s) and a ~ 0, so the
      // textbook forms a + b - s, 1 - a/s and 1 - b/s cancel; in FP32 that leaves ~1e-6
      // m/s of noise in the row, which the small eigenvalue (~kappa) of the impulse split
      // between redundant contacts amplifies to ~1e-3 N and the Newton iteration stalls.
      // The same quantities in forms free of cancellation (exact rearrangements):
      // a + b - s = (2ab - eps^2)/(a + b + s) for a + b > 0;  1 - a/s = (b^2 + eps^2)/(s (s + a))
      // for a > 0;  1 - b/s likewise.
      Real s = ssqrt(a * a + bb * bb + eps * eps);
      const Real apb = a + bb;
      Real phi = apb > Real(0) ? (Real(2) * a * bb - eps * eps) / (apb + s) : apb - s;
      Real fa = a > Real(0) ? (bb * bb + eps * eps) / (s * (s + a)) : Real(1) - a / s;
      Real fb = bb > Real(0) ? (a * a + eps * eps) / (s * (s + bb)) : Real(1) - bb / s;
      Real scl = fa > Real(1e-12) ? fa : Real(1e-12);
      w.r2[i] = phi; w.rhat[i] = phi / scl; w.C[i] = kap + hw * fb / scl;
      // friction rows, Eq. (7): J_f u + (W + kappa) lambda_f with W from the FB reading
      Real vt = ssqrt(vel[1] * vel[1] + vel[2] * vel[2] + eps * eps);
      Real lfn = ssqrt(l1 * l1 + l2 * l2 + eps * eps);
      Real lnp = ln > Real(0) ? ln : Real(0);
      Real g = hw * (Real(sc.mu) * lnp - lfn);
      Real sg = ssqrt(vt * vt + g * g + eps * eps);
      // W's numerator max(0, vt - phi_eps(vt, g)) is sg - g >= 0; for g > 0 (sticking) it is
      // the small difference of two large numbers, taken as (vt^2 + eps^2)/(sg + g)
      Real num = g > Real(0) ? (vt * vt + eps * eps) / (sg + g) : sg - g;
      Real den = Real(sc.mu) * lnp; if (den < Real(1e-12)) den = Real(1e-12);
      Real W = num / den;
      Real rf1 = vel[1] + (W + kap) * l1, rf2 = vel[2] + (W + kap) * l2;
      Real wgt = hw / (hw + W);
      w.r2[i + 1] = rf1 * wgt; w.r2[i + 2] = rf2 * wgt;
      w.rhat[i + 1] = rf1; w.rhat[i + 2] = rf2;
      w.C[i + 1] = W + kap; w.C[i + 2] = W + kap;
      // radial part of the friction block: rho e e^T, e = lambda_f/|lambda_f|
      Real rho = Real(0);
      if (num > Real(0)) {
        Real fbg = num / sg;                  // 1 - g/sg
        rho = fbg * hw * lfn / den;
      }
      Real e1 = l1 / lfn, e2 = l2 / lfn;
      w.srad[3 * sl] = rho * e1 * e1; w.srad[3 * sl + 1] = rho * e1 * e2; w.srad[3 * sl + 2] = rho * e2 * e2;
    } else if (it < sc.n_slots + sc.nj) {
      const int j = it - sc.n_slots;
      const int i0 = mc + 5 * j;
      const int bp = sc.jp[j], bc = sc.jc[j];
      const vec3<Real> wp = v3(u[6 * bp + 3], u[6 * bp + 4], u[6 * bp + 5]);
      const vec3<Real> wc = v3(u[6 * bc + 3], u[6 * bc + 4], u[6 * bc + 5]);
      const MapE<Real> Ep(wp, h), Ec(wc, h);
      joint_rows_each<Real>(sc, j, v3(w.qp[7 * bp], w.qp[7 * bp + 1], w.qp[7 * bp + 2]), MatRot<Real>{w.R + 9 * bp},
                            v3(w.qp[7 * bc], w.qp[7 * bc + 1], w.qp[7 * bc + 2]), MatRot<Real>{w.R + 9 * bc},
                            [&](int k, vec3<Real> lp, vec3<Real> ap, vec3<Real> lc, vec3<Real> ac, Real c) {
        const vec3<Real> ap_ = Ep(ap), ac_ = Ec(ac);
        const int i = i0 + k;
        Real* Jr = w.J + 12 * i;
        Jr[0] = lp.x; Jr[1] = lp.y; Jr[2] = lp.z; Jr[3] = ap_.x; Jr[4] = ap_.y; Jr[5] = ap_.z;
        Jr[6] = lc.x; Jr[7] = lc.y; Jr[8] = lc.z; Jr[9] = ac_.x; Jr[10] = ac_.y; Jr[11] = ac_.z;
        w.r2[i] = c / hR; w.rhat[i] = c / hR; w.C[i] = Real(0);
      });
    } else {
      // k-th servo, Eq. (8): J_c u + alpha lambda_c + b_c
      const int k = it - sc.n_slots - sc.nj;
      const int j = servo_joint(sc, k);
      const int i = mc + 5 * sc.nj + k;
      const int bp = sc.jp[j], bc = sc.jc[j];
      SRow<Real> sr;
      servo_row_geom<Real>(sc, j, v3(w.qp[7 * bp], w.qp[7 * bp + 1], w.qp[7 * bp + 2]), MatRot<Real>{w.R + 9 * bp},
                           v3(w.qp[7 * bc], w.qp[7 * bc + 1], w.qp[7 * bc + 2]), MatRot<Real>{w.R + 9 * bc}, sr);
      const vec3<Real> wp = v3(u[6 * bp + 3], u[6 * bp + 4], u[6 * bp + 5]);
      const vec3<Real> wc = v3(u[6 * bc + 3], u[6 * bc + 4], u[6 * bc + 5]);
      const vec3<Real> ap_ = map_Et(sr.ang_p, wp, h), ac_ = map_Et(sr.ang_c, wc, h);
      Real* Jr = w.J + 12 * i;
      Jr[0] = sr.lin_p.x; Jr[1] = sr.lin_p.y; Jr[2] = sr.lin_p.z; Jr[3] = ap_.x; Jr[4] = ap_.y; Jr[5] = ap_.z;
      Jr[6] = sr.lin_c.x; Jr[7] = sr.lin_c.y; Jr[8] = sr.lin_c.z; Jr[9] = ac_.x; Jr[10] = ac_.y; Jr[11] = ac_.z;
      Real v = Real(0);
      for (int q = 0; q < 6; ++q) v += Jr[q] * u[6 * bp + q] + Jr[6 + q] * u[6 * bc + q];
      const Real alpha = Real(servo_alpha(sc, j, h));
      const Real r = v + alpha * lam[i] + w.sbc[k];
      w.r2[i] = r; w.rhat[i] = r; w.C[i] = alpha;
    }
  }
  __syncthreads();
  if (dyn) {
    // Eq. (10): r_dyn = M (u - u-) - h f - h J^T lambda, per body; merit part |M^-1 r_dyn|^2.
    // The inertia and constraint terms nearly cancel at convergence, so the sum is
    // accumulated with exact products and exact partial sums (acc2).
    const int ssd = sc.ss > 0 ? sc.ss : 1;
    for (int task = tid; task < 6 * nb; task += nth) {
      const int b = task / 6, k = task - 6 * (task / 6);
      acc2<Real> rd;
      int g = w.bgrp[b];
      if (g >= 0)
        for (int i = w.g0[g]; i < w.g0[g] + w.gn[g]; ++i) rd.add_prod(w.J[12 * i + k], -hR * lam[i]);
      for (int t = 0; t < w.bsepn[b]; ++t) {
        int i = w.bsep[b * ssd + t];
        int side = w.meta[4 * i + 1] == b ? 0 : 6;
        rd.add_prod(w.J[12 * i + side + k], -hR * lam[i]);
      }
      if (k < 3) {
        const Real m_ = Real(sc.mass[b]);
        rd.add_prod(m_, u[6 * b + k]);
        rd.add_prod(-m_, w.um[6 * b + k]);
      } else {
        for (int c = 0; c < 3; ++c) {
          rd.add_prod(w.Iw[9 * b + 3 * (k - 3) + c], u[6 * b + 3 + c]);
          rd.add_prod(-w.Iw[9 * b + 3 * (k - 3) + c], w.um[6 * b + 3 + c]);
        }
      }
      rd.add_prod(-hR, w.f[6 * b + k]);
      w.rdyn[6 * b + k] = rd.value();
    }
    __syncthreads();
  }
  Real part = Real(0);
  for (int b = tid; b < nb && dyn; b += nth) {
    const Real* rv = w.rdyn + 6 * b;
    Real mi = Real(1) / Real(sc.mass[b]);
    vec3<Real> iw = mat3<Real>(w.Iwi + 9 * b, v3(rv[3], rv[4], rv[5]));
    Real mr[6] = {rv[0] * mi, rv[1] * mi, rv[2] * mi, iw.x, iw.y, iw.z};
    for (int k = 0; k < 6; ++k) { w.mr[6 * b + k] = mr[k]; part += mr[k] * mr[k]; }
  }
  if (dyn)
    for (int i = tid; i < m; i += nth) part += w.r2[i] * w.r2[i];
  // with the merit: delta = delta_rel * mean diag(h J M^-1 J^T) of these rows, for the
  // assembly at this iterate (scal[2])
  Real dpart = 0;
  for (int i = tid; i < m; i += nth) {
    const Real* Ji = w.J + 12 * i;
    Real Yi[12];
    minv_row(sc, w, i, Yi);
    dpart += hR * (rowdot(Ji, 0, Yi, 0) + rowdot(Ji, 6, Yi, 6));
  }
  block_sum2(w, part, dpart);
  if (tid == 0) w.scal[2] = m > 0 ? Real(sc.delta_rel) * dpart / Real(m) : Real(0);
  __syncthreads();                         // scal[2] is read by the assembly that follows
  return part;
}

// ---------------------------------------------------------------------------
// Schur assembly, factorisation and solves
// ---------------------------------------------------------------------------


template <class Real> __device__ void assemble(const DevScene& sc, WS<Real>& w, double h) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int m = w.ints[0], mc = w.ints[1], gstr = tri_size(sc.pg), ss = sc.ss, ldg = sc.ldg;
  const Real hR = Real(h);
  // delta = delta_rel * mean diag(h J M^-1 J^T), formed by the evaluation at this iterate
  const Real delta = w.scal[2];
  // group blocks (full, symmetric) and their coupling rows E_g: a thread per contact row
  for (int r = tid; r < mc; r += nth) {
    const int g = w.rgrp[r], r0 = w.g0[g], i = r - r0, bg = sc.group_body[g];
    Real* Gb = w.G + g * gstr;
    const int ti = w.meta[4 * r] & 15, si = w.meta[4 * r] >> 4;
    Real Yr[12];
    minv_row(sc, w, r, Yr);
    // row i of the group block: h J M^-1 J^T for every column, then the diagonal and the
    // radial terms of the row's own contact (friction rows of one slot are adjacent)
    Real* Gi = Gb + tri(i, 0);
    int jj = r0;
    for (; jj + 1 <= r; jj += 2) {
      const Real v0 = hR * rowdot(w.J + 12 * jj, 0, Yr, 0);
      const Real v1 = hR * rowdot(w.J + 12 * (jj + 1), 0, Yr, 0);
      Gi[jj - r0] = v0;
      Gi[jj + 1 - r0] = v1;
    }
    if (jj <= r) Gi[jj - r0] = hR * rowdot(w.J + 12 * jj, 0, Yr, 0);
    Real dg = Gi[i] + (w.C[r] + delta);
    if (ti == ROW_FRIC) {
      const Real* rd = w.srad + 3 * w.ref[r];
      if (si == 1) {
        dg += rd[0];
      } else {
        dg += rd[2];
        Gi[i - 1] += rd[1];
      }
    }
    Gi[i] = dg;
    Real* Eb = w.E + g * sc.cmax * ldg;
    for (int k = 0; k < sc.cpl_n[g]; ++k) {
      const int row = mc + sc.cpl_row[g][k];
      const int side = w.meta[4 * row + 1] == bg ? 0 : 6;
      Eb[k * ldg + i] = hR * rowdot(w.J + 12 * row, side, Yr, 0);
    }
  }
  // separator block: a thread per separator row, counted from the last thread so that it
  // runs beside the contact rows (counted from the first) rather than after them
  for (int a = nth - 1 - tid; a >= 0 && a < ss; a += nth) {
    const int i = mc + a;
    const int ia0 = w.meta[4 * i + 1], ia1 = w.meta[4 * i + 2];
    Real Yi[12];
    minv_row(sc, w, i, Yi);
    for (int b = 0; b <= a; ++b) {
      const int j = mc + b;
      const int jb0 = w.meta[4 * j + 1], jb1 = w.meta[4 * j + 2];
      Real v = 0;
      if (ia0 == jb0) v += rowdot(w.J + 12 * j, 0, Yi, 0);
      if (ia0 == jb1) v += rowdot(w.J + 12 * j, 6, Yi, 0);
      if (ia1 >= 0 && ia1 == jb0) v += rowdot(w.J + 12 * j, 0, Yi, 6);
      if (ia1 >= 0 && ia1 == jb1) v += rowdot(w.J + 12 * j, 6, Yi, 6);
      v *= hR;
      if (a == b) v += w.C[i] + delta;
      w.S[tri(a, b)] = v;
    }
  }
  __syncthreads();
}

// L^-1 of an n x n symmetric positive definite block, in place, by a team of threads:
// one warp (TEAM = 0, __syncwarp) or the whole CTA (TEAM = 1, __syncthreads).  A (packed
// lower triangle, tri()) holds the block on entry and L^-1 on return, L L^T = A; colbuf
// holds n values.  Right-looking, one pivot k at a time:
//   pass 1: column k of L below the pivot goes to colbuf; row k of L^-1 is finished,
//           X[k][c] = Xt[k][c] / L[k][k] (its partial sums Xt already sit in row k);
//   pass 2: rank-one updates of the trailing block, A[i][j] -= L[i][k] L[j][k]
//           (k < j <= i), and of the rows of L^-1 below, Xt[i][c] -= L[i][k] X[k][c]
//           (c <= k).  Position (i, k) changes from L[i][k], now in colbuf and never
//           read again, to Xt[i][k].
// Each element of L and of L^-1 receives the same operations in the same order as the
// sequential column-by-column factor and forward substitution (k, resp. l,
// ascending), so the result does not depend on the team size.
template <int TEAM, class Real> __device__ void chol_inv_inplace(Real* A, int n, Real* colbuf) {
  // TEAM 0: one warp; 1: the whole CTA; 2: one half-warp (16 lanes)
  const int t = TEAM == 1 ? (int)threadIdx.x : (TEAM == 2 ? (int)(threadIdx.x & 15) : (int)(threadIdx.x & 31));
  const int T = TEAM == 1 ? (int)blockDim.x : (TEAM == 2 ? 16 : 32);
  const int cw = TEAM == 2 ? 16 : 32;                         // columns per pass
  const unsigned half = 0xffffu << (16 * ((threadIdx.x >> 4) & 1));
  auto team_sync = [&]() {
    if (TEAM == 1) __syncthreads();
    else if (TEAM == 2) __syncwarp(half);
    else __syncwarp();
  };
  for (int k = 0; k < n; ++k) {
    const Real akk = A[tri(k, k)];
    const Real inv = pivot_rsqrt(akk > Real(0) ? akk : Real(1e-30));
    const Real xkk = inv;                   // X[k][k], known to every thread
    for (int e = t; e < n; e += T) {        // the pivot entry itself is left for pass 2
      if (e > k) colbuf[e] = A[tri(e, k)] * inv;
      else if (e < k) A[tri(k, e)] *= inv;
    }
    team_sync();
    if (t == 0) A[tri(k, k)] = xkk;
    // lanes own columns (j = lane, lane + cw, ...), groups of cw lanes take every nw-th row
    const int nw = T / cw, lane = t % cw;
    for (int j = lane; j < n; j += cw) {
      // per column: the multiplier of l_ik (X[k][j], X[k][k] or l_jk) and whether the
      // entry keeps its value (no branch inside the row loop)
      const Real coef = j < k ? A[tri(k, j)] : (j == k ? xkk : colbuf[j]);
      const bool keep = j != k;
      int i = (k + 1 > j ? k + 1 : j) + t / cw;
      for (; i + 3 * nw < n; i += 4 * nw) {             // four independent rows per pass
        const int i1 = i + nw, i2 = i1 + nw, i3 = i2 + nw;
        const Real l0 = colbuf[i], l1 = colbuf[i1], l2 = colbuf[i2], l3 = colbuf[i3];
        Real* a0 = A + tri(i, j);
        Real* a1 = A + tri(i1, j);
        Real* a2 = A + tri(i2, j);
        Real* a3 = A + tri(i3, j);
        const Real o0 = keep ? *a0 : Real(0), o1 = keep ? *a1 : Real(0);
        const Real o2 = keep ? *a2 : Real(0), o3 = keep ? *a3 : Real(0);
        *a0 = o0 - l0 * coef; *a1 = o1 - l1 * coef; *a2 = o2 - l2 * coef; *a3 = o3 - l3 * coef;
      }
      for (; i < n; i += nw) {
        const Real lik = colbuf[i];
        Real* aij = A + tri(i, j);
        const Real old = keep ? *aij : Real(0);
        *aij = old - lik * coef;
      }
    }
    team_sync();
  }
}

// One round of P pivots (k .. k+P-1) of the in-place L^-1 by the whole CTA, P <= 4.  Every
// thread forms the P x P pivot block itself: the inverse pivots ip[p] = 1/L[k+p][k+p], the
// block's L below the diagonal and its inverse X.  Pass 1 gives columns k .. k+P-1 of L
// below the block (colbuf, n values per column) and finishes rows k .. k+P-1 of L^-1 left
// of it; pass 2 applies the P rank-one updates, in pivot order, to the trailing block and
// to the rows of L^-1 below.  Every element receives the operations of the one-pivot-per-
// round factor in the same order (k ascending); a round costs two barriers.
template <int P, class Real> __device__ void chol_round(Real* A, int n, int k, Real* colbuf) {
  const int t = threadIdx.x, T = blockDim.x;
  Real a[P][P], l[P][P], x[P][P], xt[P][P], ip[P];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int q = 0; q < P; ++q) { a[p][q] = q <= p ? A[tri(k + p, k + q)] : Real(0); xt[p][q] = Real(0); }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    ip[p] = pivot_rsqrt(a[p][p] > Real(0) ? a[p][p] : Real(1e-30));
#pragma unroll
    for (int r = p + 1; r < P; ++r) l[r][p] = a[r][p] * ip[p];
#pragma unroll
    for (int r = p + 1; r < P; ++r)
#pragma unroll
      for (int c = p + 1; c <= r; ++c) a[r][c] = a[r][c] - l[r][p] * l[c][p];
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int q = 0; q < p; ++q) x[p][q] = xt[p][q] * ip[p];
    x[p][p] = ip[p];
#pragma unroll
    for (int r = p + 1; r < P; ++r) {
#pragma unroll
      for (int q = 0; q < p; ++q) xt[r][q] = xt[r][q] - l[r][p] * x[p][q];
      xt[r][p] = Real(0) - l[r][p] * x[p][p];
    }
  }
  // pass 1 writes neither the pivot block nor any entry another thread reads in this pass
  for (int e = t; e < n; e += T) {
    if (e >= k + P) {
      Real v[P];
#pragma unroll
      for (int p = 0; p < P; ++p) v[p] = A[tri(e, k + p)];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const Real c = v[p] * ip[p];
        colbuf[p * n + e] = c;
#pragma unroll
        for (int r = p + 1; r < P; ++r) v[r] = v[r] - c * l[r][p];
      }
    } else if (e < k) {
      Real y[P];
#pragma unroll
      for (int p = 0; p < P; ++p) y[p] = A[tri(k + p, e)];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const Real xe = y[p] * ip[p];
        A[tri(k + p, e)] = xe;
#pragma unroll
        for (int r = p + 1; r < P; ++r) y[r] = y[r] - l[r][p] * xe;
      }
    }
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int q = 0; q <= p; ++q) A[tri(k + p, k + q)] = x[p][q];
  }
  const int nw = T >> 5, lane = t & 31;
  for (int j = lane; j < n; j += 32) {
    // the P multipliers of column j, the first pivot that updates it (columns of the pivot
    // block took the earlier pivots' updates into colbuf) and whether the entry keeps its value
    Real m[P];
    int qs = 0;
    bool keep = true;
    if (j < k) {
#pragma unroll
      for (int p = 0; p < P; ++p) m[p] = A[tri(k + p, j)];
    } else if (j < k + P) {
      qs = j - k;
      keep = false;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        Real xv = Real(0);
#pragma unroll
        for (int q = 0; q < P; ++q) if (q == j - k && q <= p) xv = x[p][q];
        m[p] = xv;
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) m[p] = colbuf[p * n + j];
    }
    int i = (k + P > j ? k + P : j) + (t >> 5);
    for (; i + 3 * nw < n; i += 4 * nw) {                  // four independent rows per pass
      int ii[4] = {i, i + nw, i + 2 * nw, i + 3 * nw};
      Real v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = keep ? A[tri(ii[r], j)] : Real(0);
#pragma unroll
      for (int p = 0; p < P; ++p)
        if (p >= qs)
#pragma unroll
          for (int r = 0; r < 4; ++r) v[r] = v[r] - colbuf[p * n + ii[r]] * m[p];
#pragma unroll
      for (int r = 0; r < 4; ++r) A[tri(ii[r], j)] = v[r];
    }
    for (; i < n; i += nw) {
      Real v = keep ? A[tri(i, j)] : Real(0);
#pragma unroll
      for (int p = 0; p < P; ++p)
        if (p >= qs) v = v - colbuf[p * n + i] * m[p];
      A[tri(i, j)] = v;
    }
  }
  __syncthreads();
}

// In-place L^-1 of an n x n SPD block by the whole CTA: four pivots per round, the
// remainder two and one at a time.  colbuf holds 4 n values.
template <class Real> __device__ void chol_inv_inplace4(Real* A, int n, Real* colbuf) {
  int k = 0;
  for (; k + 3 < n; k += 4) chol_round<4>(A, n, k, colbuf);
  for (; k + 1 < n; k += 2) chol_round<2>(A, n, k, colbuf);
  if (k < n) chol_round<1>(A, n, k, colbuf);
}

// Two-accumulator dot products (even and odd terms apart, halving the dependent chain):
// a contiguous one, and one down a column of a packed triangle (element (l, c), l = c0 ..
// n-1, at tri(l, c), the offset growing by l + 1 per row).
template <class Real> __device__ __forceinline__ Real dot2c(const Real* a, const Real* b, int n) {
  Real s0 = Real(0), s1 = Real(0);
  int l = 0;
  for (; l + 1 < n; l += 2) { s0 += a[l] * b[l]; s1 += a[l + 1] * b[l + 1]; }
  if (l < n) s0 += a[l] * b[l];
  return s0 + s1;
}
template <class Real> __device__ __forceinline__ Real dot2col(const Real* T, int c, int c0, int n, const Real* b) {
  Real s0 = Real(0), s1 = Real(0);
  int l = c0, off = tri(c0, c);
  for (; l + 1 < n; l += 2) {
    s0 += T[off] * b[l];
    off += l + 1;
    s1 += T[off] * b[l + 1];
    off += l + 2;
  }
  if (l < n) s0 += T[off] * b[l];
  return s0 + s1;
}

// Block-arrowhead factorisation kept in inverse form for row-parallel solves:
//   Li_g = L_g^-1 with L_g L_g^T = A_g (contact groups; stored in G, packed),
//   F_g = E_g L_g^-T (coupled separator rows; stored in H),
//   Lsi = L_s^-1 with L_s L_s^T = S - sum_g F_g F_g^T, the reduced separator (stored in S,
//   packed).
template <class Real> __device__ void factor(const DevScene& sc, WS<Real>& w, double h) {
  const int tid = threadIdx.x, nth = blockDim.x, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const Real hR = Real(h);
  const int pg = sc.pg, ss = sc.ss, ldg = sc.ldg, cm = sc.cmax, gstr = tri_size(pg);
  const int rb = pg > ss ? pg : ss;
  // Li_g in place: up to four teams (half-warps for CTAs of up to 64 threads, else warps)
  // each take their groups
  if (nth <= 64) {
    const int team = tid >> 4, nteams = nth >> 4;
    for (int g = team; g < sc.n_groups; g += nteams)
      chol_inv_inplace<2>(w.G + g * gstr, w.gn[g], w.prow + team * rb);
  } else {
    for (int g = wid; g < sc.n_groups; g += nw) chol_inv_inplace<0>(w.G + g * gstr, w.gn[g], w.prow + (wid & 3) * rb);
  }
  __syncthreads();
  // F_g[k][j] = sum_{l <= j} E_g[k][l] Li_g[j][l]
  for (int g = 0; g < sc.n_groups; ++g) {
    const int n = w.gn[g], cnt = sc.cpl_n[g] * n;
    const Real* Lb = w.G + g * gstr;
    const Real* Eb = w.E + g * cm * ldg;
    Real* Fb = w.H + g * cm * ldg;
    for (int e = tid; e < cnt; e += nth) {
      const int k = e / n, j = e - k * n;
      Fb[k * ldg + j] = dot2c(Eb + k * ldg, Lb + tri(j, 0), j + 1);
    }
  }
  __syncthreads();
  // S' = S - sum_g F_g F_g^T: group by group (a separator row may couple to two groups),
  // one coupled row pair (k1 >= k2 of the group's coupling list) per thread
  for (int g = 0; g < sc.n_groups; ++g) {
    const int nc = sc.cpl_n[g], n = w.gn[g];
    if (n == 0) continue;                    // no active contact rows: F_g is empty
    const Real* Fb = w.H + g * cm * ldg;
    for (int e = tid; e < nc * nc; e += nth) {
      const int k1 = e / nc, k2 = e - k1 * nc;
      if (k2 > k1) continue;
      const int a = sc.cpl_row[g][k1], b = sc.cpl_row[g][k2];
      w.S[a >= b ? tri(a, b) : tri(b, a)] -= dot2c(Fb + k1 * ldg, Fb + k2 * ldg, n);
    }
    __syncthreads();
  }
  // Lsi = L_s^-1 in place over S, the whole CTA
  if (ss > 0) chol_inv_inplace4(w.S, ss, w.prow);
}

// v <- A^-1 v with the inverse-form block-arrowhead factor (row-parallel phases)
template <class Real> __device__ void arrow_solve(const DevScene& sc, WS<Real>& w, Real* v) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int gstr = tri_size(sc.pg), ss = sc.ss, ldg = sc.ldg, cm = sc.cmax, mc = w.ints[1];
  Real* y = w.tmp;
  Real* z = w.tmp2;
  // y_g = Li_g b_g
  for (int r = tid; r < mc; r += nth) {
    const int g = w.rgrp[r], r0 = w.g0[g], i = r - r0;
    y[r] = dot2c(w.G + g * gstr + tri(i, 0), v + r0, i + 1);
  }
  __syncthreads();
  // b_s' = b_s - sum_g F_g y_g
  for (int a = tid; a < ss; a += nth) {
    Real acc = v[mc + a];
    for (int pa = 0; pa < sc.sep_n[a]; ++pa) {
      const int g = sc.sep_g[a][pa];
      acc -= dot2c(w.H + g * cm * ldg + sc.sep_k[a][pa] * ldg, y + w.g0[g], w.gn[g]);
    }
    z[a] = acc;
  }
  __syncthreads();
  // y_s = Lsi b_s'
  for (int a = tid; a < ss; a += nth) y[mc + a] = dot2c(w.S + tri(a, 0), z, a + 1);
  __syncthreads();
  // x_s = Lsi^T y_s
  for (int a = tid; a < ss; a += nth) v[mc + a] = dot2col(w.S, a, a, ss, y + mc);
  __syncthreads();
  // r_g = y_g - F_g^T x_s
  for (int r = tid; r < mc; r += nth) {
    const int g = w.rgrp[r], i = r - w.g0[g];
    const Real* Fb = w.H + g * cm * ldg;
    Real s0 = y[r], s1 = Real(0);
    const int nc = sc.cpl_n[g];
    int k = 0;
    for (; k + 1 < nc; k += 2) {
      s0 -= Fb[k * ldg + i] * v[mc + sc.cpl_row[g][k]];
      s1 -= Fb[(k + 1) * ldg + i] * v[mc + sc.cpl_row[g][k + 1]];
    }
    if (k < nc) s0 -= Fb[k * ldg + i] * v[mc + sc.cpl_row[g][k]];
    z[r] = s0 + s1;
  }
  __syncthreads();
  // x_g = Li_g^T r_g
  for (int r = tid; r < mc; r += nth) {
    const int g = w.rgrp[r], r0 = w.g0[g], i = r - r0, n = w.gn[g];
    v[r] = dot2col(w.G + g * gstr, i, i, n, z + r0);
  }
  __syncthreads();
}

// out_b = sum over rows touching body b of J_row,b^T x_row  (6 per body)
template <class Real> __device__ void jt_apply(const DevScene& sc, WS<Real>& w, const Real* x, Real* out) {
  const int ssd = sc.ss > 0 ? sc.ss : 1;
  for (int b = threadIdx.x; b < sc.nb; b += blockDim.x) {
    Real jt[6] = {0, 0, 0, 0, 0, 0};
    int g = w.bgrp[b];
    if (g >= 0)
      for (int i = w.g0[g]; i < w.g0[g] + w.gn[g]; ++i)
        for (int k = 0; k < 6; ++k) jt[k] += w.J[12 * i + k] * x[i];
    for (int t = 0; t < w.bsepn[b]; ++t) {
      int i = w.bsep[b * ssd + t];
      int side = w.meta[4 * i + 1] == b ? 0 : 6;
      for (int k = 0; k < 6; ++k) jt[k] += w.J[12 * i + side + k] * x[i];
    }
    for (int k = 0; k < 6; ++k) out[6 * b + k] = jt[k];
  }
}

// compensated variant of jt_apply (exact products, exact partial sums)
template <class Real> __device__ void jt_apply_acc(const DevScene& sc, WS<Real>& w, const Real* x, Real* out) {
  const int ssd = sc.ss > 0 ? sc.ss : 1;
  for (int b = threadIdx.x; b < sc.nb; b += blockDim.x) {
    acc2<Real> jt[6];
    int g = w.bgrp[b];
    if (g >= 0)
      for (int i = w.g0[g]; i < w.g0[g] + w.gn[g]; ++i)
        for (int k = 0; k < 6; ++k) jt[k].add_prod(w.J[12 * i + k], x[i]);
    for (int t = 0; t < w.bsepn[b]; ++t) {
      int i = w.bsep[b * ssd + t];
      int side = w.meta[4 * i + 1] == b ? 0 : 6;
      for (int k = 0; k < 6; ++k) jt[k].add_prod(w.J[12 * i + side + k], x[i]);
    }
    for (int k = 0; k < 6; ++k) out[6 * b + k] = jt[k].value();
  }
}

// M^-1 v per body (6 per body)
template <class Real> __device__ __forceinline__ void minv6(const DevScene& sc, const WS<Real>& w, int b, const Real* v,
                                                            Real* o) {
  Real mi = Real(1) / Real(sc.mass[b]);
  o[0] = v[0] * mi; o[1] = v[1] * mi; o[2] = v[2] * mi;
  vec3<Real> a = mat3<Real>(w.Iwi + 9 * b, v3(v[3], v[4], v[5]));
  o[3] = a.x; o[4] = a.y; o[5] = a.z;
}

// Schur solve with iterative refinement: x = A^-1 b with the arrowhead factor, then
// `sweeps` corrections x += A^-1 (b - A x), where A x = h J (M^-1 J^T x) + (C + delta) x
// (+ the radial friction blocks) is formed matrix-free from J.  b is kept in `b`,
// the solution is returned in `x`; t6 (6 per body) and r (rows) are scratch.
template <class Real>
__device__ void schur_solve(const DevScene& sc, WS<Real>& w, const Real* b, Real* x, Real* t6, Real* r, double h,
                            int sweeps, Real stop_rel = Real(0)) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0];
  const Real hR = Real(h);
  // pass -1 solves for x itself (its correction from x = 0 is A^-1 b), so that one inlined
  // copy of the arrowhead solve serves the first solve and the sweeps
  for (int i = tid; i < m; i += nth) { x[i] = Real(0); r[i] = b[i]; }
  __syncthreads();
  const Real delta = w.scal[2];
  for (int sweep = -1; sweep < sweeps; ++sweep) {
    if (sweep >= 0) {
      jt_apply(sc, w, x, t6);
      __syncthreads();
      for (int bb = tid; bb < sc.nb; bb += nth) {
        Real o[6];
        minv6(sc, w, bb, t6 + 6 * bb, o);
        for (int k = 0; k < 6; ++k) t6[6 * bb + k] = o[k];
      }
      __syncthreads();
      for (int i = tid; i < m; i += nth) {
        const Real* Ji = w.J + 12 * i;
        int b0 = w.meta[4 * i + 1], b1 = w.meta[4 * i + 2];
        acc2<Real> ax;
        for (int k = 0; k < 6; ++k) ax.add_prod(Ji[k], t6[6 * b0 + k]);
        if (b1 >= 0) for (int k = 0; k < 6; ++k) ax.add_prod(Ji[6 + k], t6[6 * b1 + k]);
        acc2<Real> res;                   // r = b - A x, compensated throughout
        res.add(b[i]);
        res.add_prod(-hR, ax.s);
        res.add_prod(-hR, ax.c);
        res.add_prod(-(w.C[i] + delta), x[i]);
        int t = w.meta[4 * i] & 15, sub = w.meta[4 * i] >> 4;
        if (t == ROW_FRIC) {
          const Real* rd = w.srad + 3 * w.ref[i];
          if (sub == 1) { res.add_prod(-rd[0], x[i]); res.add_prod(-rd[1], x[i + 1]); }
          else { res.add_prod(-rd[1], x[i - 1]); res.add_prod(-rd[2], x[i]); }
        }
        r[i] = res.value();
      }
      __syncthreads();
    }
    arrow_solve(sc, w, r);
    Real cmax = Real(0), xmax = Real(0);
    for (int i = tid; i < m; i += nth) {
      x[i] += r[i];
      cmax = fmax(cmax, fabs(r[i]));
      xmax = fmax(xmax, fabs(x[i]));
    }
    __syncthreads();
    // optional early stop once the correction no longer changes x at working precision
    if (sweep >= 0 && stop_rel > Real(0)) {
      block_max2(w, cmax, xmax);
      if (cmax <= stop_rel * xmax) break;
    }
  }
}

// ---------------------------------------------------------------------------
// matrix-free Schur operator and preconditioned conjugate residual (Sec. III-C)
// ---------------------------------------------------------------------------
// out = A v, A = h J M^-1 J^T + C + delta I (+ the radial friction blocks), from the rows:
// t6 = J^T v per body component (a thread per component, over the rows touching the
// body), then per row h J_i M^-1 t6 plus the diagonal and radial terms.  ACC: exact
// products and compensated sums throughout (the adjoint's solve).  Returns this thread's
// part of v . out; the caller reduces it (the rows are written by their owning threads).
template <class Real, bool ACC>
__device__ Real schur_apply(const DevScene& sc, WS<Real>& w, const Real* v, Real* out, Real* t6, double h) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0];
  const int ssd = sc.ss > 0 ? sc.ss : 1;
  for (int task = tid; task < 6 * sc.nb; task += nth) {
    const int b = task / 6, k = task - 6 * (task / 6);
    acc2<Real> ca;
    Real acc = Real(0);
    const int g = w.bgrp[b];
    if (g >= 0)
      for (int i = w.g0[g]; i < w.g0[g] + w.gn[g]; ++i) {
        if (ACC) ca.add_prod(w.J[12 * i + k], v[i]);
        else acc += w.J[12 * i + k] * v[i];
      }
    for (int t = 0; t < w.bsepn[b]; ++t) {
      const int i = w.bsep[b * ssd + t];
      const Real jv = w.J[12 * i + (w.meta[4 * i + 1] == b ? 0 : 6) + k];
      if (ACC) ca.add_prod(jv, v[i]);
      else acc += jv * v[i];
    }
    t6[task] = ACC ? ca.value() : acc;
  }
  __syncthreads();
  const Real hR = Real(h), delta = w.scal[2];
  Real part = Real(0);
  for (int i = tid; i < m; i += nth) {
    const Real* Ji = w.J + 12 * i;
    acc2<Real> ca;
    Real ax = Real(0);
    for (int side = 0; side < 2; ++side) {
      const int b = w.meta[4 * i + 1 + side];
      if (b < 0) continue;
      Real o[6];
      minv6(sc, w, b, t6 + 6 * b, o);
      for (int q = 0; q < 6; ++q) {
        if (ACC) ca.add_prod(Ji[6 * side + q], o[q]);
        else ax += Ji[6 * side + q] * o[q];
      }
    }
    Real y;
    const int t = w.meta[4 * i] & 15, sub = w.meta[4 * i] >> 4;
    if (ACC) {
      acc2<Real> ya;
      ya.add_prod(hR, ca.s);
      ya.add_prod(hR, ca.c);
      ya.add_prod(w.C[i] + delta, v[i]);
      if (t == ROW_FRIC) {
        const Real* rd = w.srad + 3 * w.ref[i];
        if (sub == 1) { ya.add_prod(rd[0], v[i]); ya.add_prod(rd[1], v[i + 1]); }
        else { ya.add_prod(rd[1], v[i - 1]); ya.add_prod(rd[2], v[i]); }
      }
      y = ya.value();
    } else {
      y = hR * ax + (w.C[i] + delta) * v[i];
      if (t == ROW_FRIC) {
        const Real* rd = w.srad + 3 * w.ref[i];
        y += sub == 1 ? rd[0] * v[i] + rd[1] * v[i + 1] : rd[1] * v[i - 1] + rd[2] * v[i];
      }
    }
    out[i] = y;
    part += v[i] * y;
  }
  return part;
}

// Jacobi preconditioner: the inverse diagonal of A, stored per row by the row's thread
template <class Real> __device__ void pcr_jacobi(const DevScene& sc, WS<Real>& w, double h) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0];
  const Real hR = Real(h), delta = w.scal[2];
  Real* pd = w.pcr + 6 * sc.m_max;
  for (int i = tid; i < m; i += nth) {
    const Real* Ji = w.J + 12 * i;
    Real Yi[12];
    minv_row(sc, w, i, Yi);
    Real d = hR * (rowdot(Ji, 0, Yi, 0) + rowdot(Ji, 6, Yi, 6)) + w.C[i] + delta;
    if ((w.meta[4 * i] & 15) == ROW_FRIC) d += w.srad[3 * w.ref[i] + ((w.meta[4 * i] >> 4) == 1 ? 0 : 2)];
    pd[i] = Real(1) / d;
  }
}

// Block-Jacobi preconditioner: each contact group's block and the (unreduced) separator
// block of A, as assembled, factored in place to their inverse Cholesky factors (G, S)
template <class Real> __device__ void factor_blocks(const DevScene& sc, WS<Real>& w) {
  const int tid = threadIdx.x, nth = blockDim.x, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  const int pg = sc.pg, ss = sc.ss, gstr = tri_size(pg), rb = pg > ss ? pg : ss;
  if (nth <= 64) {
    const int team = tid >> 4, nteams = nth >> 4;
    for (int g = team; g < sc.n_groups; g += nteams)
      chol_inv_inplace<2>(w.G + g * gstr, w.gn[g], w.prow + team * rb);
  } else {
    for (int g = wid; g < sc.n_groups; g += nw) chol_inv_inplace<0>(w.G + g * gstr, w.gn[g], w.prow + (wid & 3) * rb);
  }
  __syncthreads();
  if (ss > 0) chol_inv_inplace4(w.S, ss, w.prow);
}

// out = P v.  Jacobi: per row, by the row's thread (no synchronisation).  Block Jacobi:
// L^-T L^-1 v per block (reads other rows of v: synchronises on entry and between the two
// triangular products); out is written by the rows' threads.
template <class Real> __device__ void pcr_precond(const DevScene& sc, WS<Real>& w, const Real* v, Real* out) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0], mc = w.ints[1];
  if (sc.pc == PC_JACOBI) {
    const Real* pd = w.pcr + 6 * sc.m_max;
    for (int i = tid; i < m; i += nth) out[i] = pd[i] * v[i];
    return;
  }
  const int gstr = tri_size(sc.pg), ss = sc.ss;
  Real* y = w.tmp;
  __syncthreads();
  for (int r = tid; r < m; r += nth) {
    Real acc = Real(0);
    if (r < mc) {
      const int g = w.rgrp[r], r0 = w.g0[g], i = r - r0;
      const Real* Li = w.G + g * gstr + tri(i, 0);
      for (int l = 0; l <= i; ++l) acc += Li[l] * v[r0 + l];
    } else {
      const int a = r - mc;
      const Real* La = w.S + tri(a, 0);
      for (int b = 0; b <= a; ++b) acc += La[b] * v[mc + b];
    }
    y[r] = acc;
  }
  __syncthreads();
  for (int r = tid; r < m; r += nth) {
    Real acc = Real(0);
    if (r < mc) {
      const int g = w.rgrp[r], r0 = w.g0[g], i = r - r0, n = w.gn[g];
      const Real* Lb = w.G + g * gstr;
      for (int l = i; l < n; ++l) acc += Lb[tri(l, i)] * y[r0 + l];
    } else {
      const int a = r - mc;
      for (int b = a; b < ss; ++b) acc += w.S[tri(b, a)] * y[mc + b];
    }
    out[r] = acc;
  }
}

// Preconditioned conjugate residual on A x = b from x = 0 (A SPD, P SPD):
//   r = b, z = P r, p = z;  per iteration
//   alpha = (z, A z) / (A p, P A p);  x += alpha p;  r -= alpha A p;  z -= alpha P A p
//   beta = (z', A z') / (z, A z);  p = z' + beta p;  A p = A z' + beta A p
// one operator product and one preconditioner application per iteration; x_k minimises
// |L^T (b - A x)| (P = L L^T) over K_k(P A, P b).  At most `iters` iterations; with rtol > 0
// it stops after the first iteration with |r| <= rtol |b| and sets *conv.  Breakdown (a
// denominator that is not positive: the exact solution reached) stops it too.  Every
// decision is taken on block-reduced values, so all threads leave together.  t6: 6 nb
// scratch.  Returns the iterations taken.
template <class Real, bool ACC>
__device__ int pcr_solve(const DevScene& sc, WS<Real>& w, const Real* b, Real* x, int iters, Real rtol, Real* t6,
                         double h, int* conv) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0], M = sc.m_max;
  Real *r = w.pcr, *z = r + M, *p = z + M, *Ap = p + M, *Az = Ap + M, *q = Az + M;
  Real bb = Real(0);
  for (int i = tid; i < m; i += nth) { x[i] = Real(0); r[i] = b[i]; bb += b[i] * b[i]; }
  pcr_precond(sc, w, r, z);
  __syncthreads();
  Real rho = schur_apply<Real, ACC>(sc, w, z, Az, t6, h);
  for (int i = tid; i < m; i += nth) { p[i] = z[i]; Ap[i] = Az[i]; }
  block_sum2(w, rho, bb);
  *conv = 0;
  if (!(bb > Real(0))) { *conv = 1; return 0; }
  const Real target = rtol * rtol * bb;
  int k = 0;
  for (; k < iters; ++k) {
    pcr_precond(sc, w, Ap, q);
    Real den = Real(0);
    for (int i = tid; i < m; i += nth) den += Ap[i] * q[i];
    den = block_sum(w, den);
    if (!(den > Real(0)) || !(rho > Real(0))) break;
    const Real alpha = rho / den;
    Real rr = Real(0);
    for (int i = tid; i < m; i += nth) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      z[i] -= alpha * q[i];
      rr += r[i] * r[i];
    }
    __syncthreads();
    Real rho1 = schur_apply<Real, ACC>(sc, w, z, Az, t6, h);
    block_sum2(w, rho1, rr);
    const Real beta = rho1 / rho;
    rho = rho1;
    for (int i = tid; i < m; i += nth) { p[i] = z[i] + beta * p[i]; Ap[i] = Az[i] + beta * Ap[i]; }
    if (rtol > Real(0) && rr <= target) { *conv = 1; ++k; break; }
  }
  __syncthreads();
  return k;
}

// The adjoint's PCR solve, restarted on the true residual: x = 0, r = b; then up to 8
// times: PCR on A dx = r (asking for |r'| <= max(rtol |b| / |r|, floor) |r|, floor 1e-4 in
// FP32: what one FP32 run's recurrence reliably attains), x += dx, and the true residual
// r = b - A x formed with the compensated product.  It stops when |r| <= rtol |b|, when a
// correction no longer changes x at working precision (max |dx| <= 2^-23 max |x| in FP32,
// 2^-52 in FP64), or after `iters` PCR iterations in all.  The Schur matrix's condition
// number (~1e5-1e6 with contact compliance) turns a residual of rtol into a solution error
// of up to cond x rtol, hence the FP32 default rtol of 1e-10, far below what one FP32 run
// reaches.  dx, rt: m-row scratch.  Returns the PCR iterations; *conv = 1 when either
// stopping test was met.
template <class Real>
__device__ int pcr_solve_refined(const DevScene& sc, WS<Real>& w, const Real* b, Real* x, int iters, Real rtol,
                                 Real* t6, Real* dx, Real* rt, double h, int* conv) {
  const int tid = threadIdx.x, nth = blockDim.x, m = w.ints[0];
  const Real floor = sizeof(Real) == 4 ? Real(1e-4) : Real(0);
  const Real ulp = sizeof(Real) == 4 ? Real(1.1920929e-7) : Real(2.220446049250313e-16);
  Real bb = Real(0);
  for (int i = tid; i < m; i += nth) { x[i] = Real(0); rt[i] = b[i]; bb += b[i] * b[i]; }
  bb = block_sum(w, bb);
  Real rr = bb;
  Real* Ax = w.pcr + 4 * sc.m_max;     // free between PCR runs
  int its = 0;
  *conv = 0;
  for (int restart = 0; restart < 8; ++restart) {
    if (!(rr > rtol * rtol * bb)) { *conv = 1; break; }
    if (its >= iters) break;
    int c2 = 0;
    Real inner = rtol * ssqrt(bb / rr);
    if (inner < floor) inner = floor;
    its += pcr_solve<Real, true>(sc, w, rt, dx, iters - its, inner, t6, h, &c2);
    Real dmax = Real(0), xmax = Real(0);
    for (int i = tid; i < m; i += nth) {
      x[i] += dx[i];
      dmax = fmax(dmax, fabs(dx[i]));
      xmax = fmax(xmax, fabs(x[i]));
    }
    __syncthreads();
    schur_apply<Real, true>(sc, w, x, Ax, t6, h);
    Real r2 = Real(0);
    for (int i = tid; i < m; i += nth) {
      acc2<Real> r;
      r.add(b[i]);
      r.add(-Ax[i]);
      rt[i] = r.value();
      r2 += rt[i] * rt[i];
    }
    rr = block_sum(w, r2);
    dmax = block_max(w, dmax);
    xmax = block_max(w, xmax);
    if (restart > 0 && dmax <= ulp * xmax) { *conv = 1; break; }
  }
  if (!(rr > rtol * rtol * bb)) *conv = 1;
  return its;
}

// ---------------------------------------------------------------------------
// forward step kernel
// ---------------------------------------------------------------------------
// The scene lives in shared memory during a launch: kernels index its per-body and
// per-row tables with thread-dependent indices, which the constant (parameter) cache
// would serialise across a warp.
__device__ __forceinline__ void scene_to_shared(const DevScene& src, DevScene& dst) {
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevScene) / sizeof(int)); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// One world's step; `item` is the launch's work index (the CTA index of a one-CTA-per-
// world launch, or the index a persistent CTA took from the queue).
template <class Real>
__device__ __forceinline__ void step_world(const DevScene& sc, WS<Real>& w, const StepArgs& a, int item) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int world = a.list ? a.list[item] : a.world0 + item;
  if (world < 0 || world >= a.n_worlds) return;
  const TapeLayout tl = tape_layout(sc);
  Real* tpw = nullptr;    // this world's tape record (nullptr: the step records nothing)
  if (a.tape) {
    const int slot = a.list ? (a.list_slot ? a.list_slot[item] : -1) : 0;
    if (slot >= 0 && (!a.list || slot < a.tape_slots))
      tpw = reinterpret_cast<Real*>(a.tape) + ((size_t)slot * a.n_worlds + world) * tl.total;
  }
  const int ld = a.ld, nb = sc.nb;
  const Real* sin = reinterpret_cast<const Real*>(a.state_in);
  const Real* ctl = reinterpret_cast<const Real*>(a.controls);
  const double h = a.h;
  // this world's inputs (structure of arrays, world index fastest)
  Src<Real> sq = {sin + world, (size_t)ld}, su = {sin + (size_t)7 * nb * ld + world, (size_t)ld};
  Src<Real> sb = {ctl ? ctl + world : sin, ctl ? (size_t)ld : (size_t)0};
  world_setup<Real>(sc, w, sq, su, sb, h, tpw ? tpw + tl.off_ct : nullptr);
  const int m = w.ints[0];
  // warm start: lambda from the previous step on the active rows, into the trial buffers;
  // the loop's evaluation takes it as its first trial
  for (int i = tid; i < 6 * nb; i += nth) w.ut[i] = w.uk[i];
  for (int i = tid; i < m; i += nth) w.lt[i] = sin[(size_t)(13 * nb + w.meta[4 * i + 3]) * ld + world];
  __syncthreads();
  clamp_cone(sc, w, w.lt);
  __syncthreads();
  double* trace = a.trace ? a.trace + (size_t)world * (sc.budget + 2) : nullptr;
  Real merit = Real(0);
  Real best = Real(INFINITY);
  int best_k = -1, k = 0, conv = 0;
  const Real tol2 = Real(sc.tol) * Real(sc.tol);
  const int n_alpha = sc.ls ? 4 : 1;
  // phase 0: the warm start; 1: a Newton trial; 2: the returned iterate when it is not the
  // last one evaluated (the best iterate from k_min on, or the NaN iterate)
  int phase = 0;
  bool nan0 = false;
  uint32_t status = 0;
  Real mret = merit;
  Real alpha = Real(1);
  int ai = 0;
  for (;;) {
    // the loop's one evaluation: of the trial iterate, the warm start or the returned
    // iterate; step control: the full step (Sec. III-C) or backtracking on the merit
    const Real mt = evaluate(sc, w, w.ut, w.lt, h);
    if (phase == 1 && !(mt < merit) && ai + 1 < n_alpha) {
      ++ai;
      alpha *= Real(0.5);
      for (int i = tid; i < 6 * nb; i += nth) w.ut[i] = w.uk[i] + alpha * w.du[i];
      for (int i = tid; i < m; i += nth) w.lt[i] = w.lk[i] + alpha * w.dl[i];
      __syncthreads();
      clamp_cone(sc, w, w.lt);
      __syncthreads();
      continue;
    }
    for (int i = tid; i < 6 * nb; i += nth) w.uk[i] = w.ut[i];
    for (int i = tid; i < m; i += nth) w.lk[i] = w.lt[i];
    if (phase == 2) {
      mret = mt;
    } else {
      merit = mt;
      if (trace && tid == 0) trace[phase == 0 ? 0 : k + 1] = (double)merit;
      // A NaN merit at the warm start (a non-finite input, or an input that has blown up)
      // makes every Newton step NaN: the iterate is set to NaN at once instead of after
      // the whole budget of NaN iterations, and the step returns it with status bits 1 and 2.
      if (phase == 0) nan0 = !(merit == merit);
      else ++k;
    }
    __syncthreads();
    bool fin = phase == 2 || nan0 || k >= sc.budget;
    if (phase != 2) {
      phase = 1;
      if (!fin) {
        if (k >= sc.kmin && merit < best) {
          best = merit; best_k = k;
          for (int i = tid; i < 6 * nb; i += nth) w.ub[i] = w.uk[i];
          for (int i = tid; i < m; i += nth) w.lb[i] = w.lk[i];
        }
        if (merit < tol2) { conv = 1; fin = true; }
      }
      if (fin) {
        // the returned iterate: the last one (evaluated: the workspace holds its rows), or
        // the best from k_min on, or the NaN iterate, which go through the evaluation first
        mret = merit;
        if (!conv) {
          status |= 1u;
          if (nan0 || (!(k >= sc.kmin && merit < best) && best_k >= 0)) {
            const Real qnan = Real(NAN);
            for (int i = tid; i < 6 * nb; i += nth) w.ut[i] = nan0 ? qnan : w.ub[i];
            for (int i = tid; i < m; i += nth) w.lt[i] = nan0 ? qnan : w.lb[i];
            __syncthreads();
            phase = 2;
            continue;
          }
        }
      }
    }
    // a recording direct-mode step factors the returned iterate for the tape at the loop's
    // own assembly and factorisation below; otherwise the loop ends here
    if (fin && !(tpw && sc.lin == LIN_DIRECT)) break;
    // Schur step, Eq. (12): (h J M^-1 J^T + C + delta) dl = J M^-1 r_dyn - rhat, by the
    // block-arrowhead factor or by PCR (the preconditioner formed at this iterate)
    if (sc.lin == LIN_DIRECT) {
      assemble(sc, w, h);
      factor(sc, w, h);
      if (fin) break;
    } else if (sc.pc == PC_BLOCK) {
      assemble(sc, w, h);
      factor_blocks(sc, w);
    } else {
      pcr_jacobi(sc, w, h);
    }
    for (int i = tid; i < m; i += nth) {
      const Real* Ji = w.J + 12 * i;
      int b0 = w.meta[4 * i + 1], b1 = w.meta[4 * i + 2];
      acc2<Real> jm;
      for (int q = 0; q < 6; ++q) jm.add_prod(Ji[q], w.mr[6 * b0 + q]);
      if (b1 >= 0) for (int q = 0; q < 6; ++q) jm.add_prod(Ji[6 + q], w.mr[6 * b1 + q]);
      jm.add(-w.rhat[i]);
      // unrefined direct solve: the right-hand side goes straight to dl, solved in place
      if (sc.lin == LIN_DIRECT && sc.refine == 0) w.dl[i] = jm.value();
      else w.rhs[i] = jm.value();
    }
    __syncthreads();
    if (sc.lin == LIN_DIRECT) {
      if (sc.refine == 0) arrow_solve(sc, w, w.dl);
      else schur_solve(sc, w, w.rhs, w.dl, w.du, w.lt, h, sc.refine);
    } else {
      int pconv;
      pcr_solve<Real, false>(sc, w, w.rhs, w.dl, sc.pcr_iters, Real(0), w.du, h, &pconv);
    }
    // Eq. (13): du = M^-1 (h J^T dl - r_dyn)
    jt_apply(sc, w, w.dl, w.du);
    __syncthreads();
    for (int b = tid; b < nb; b += nth) {
      Real t[6];
      for (int q = 0; q < 6; ++q) t[q] = Real(h) * w.du[6 * b + q] - w.rdyn[6 * b + q];
      minv6(sc, w, b, t, w.du + 6 * b);
    }
    __syncthreads();
    // the full-step trial
    ai = 0;
    alpha = Real(1);
    for (int i = tid; i < 6 * nb; i += nth) w.ut[i] = w.uk[i] + alpha * w.du[i];
    for (int i = tid; i < m; i += nth) w.lt[i] = w.lk[i] + alpha * w.dl[i];
    __syncthreads();
    clamp_cone(sc, w, w.lt);
    __syncthreads();
  }
  if (!(mret == mret) || !(fabs((double)mret) < 1e300)) status |= 2u;
  status |= (uint32_t)w.ints[7];
  if (tpw) {
    // the returned iterate with (direct mode) its Schur factor, formed by the loop's last
    // pass; PCR records no matrix (the adjoint forms its operator and preconditioner at
    // the taped iterate)
    Real* tp = tpw;
    for (int i = tid; i < 7 * nb; i += nth) tp[tl.off_qm + i] = w.qm[i];
    for (int i = tid; i < 6 * nb; i += nth) { tp[tl.off_um + i] = w.um[i]; tp[tl.off_u + i] = w.uk[i]; }
    for (int i = tid; i < sc.n_servo; i += nth) tp[tl.off_ubar + i] = w.ubar[i];
    for (int i = tid; i < sc.m_max; i += nth) tp[tl.off_lam + i] = Real(0);
    __syncthreads();
    for (int i = tid; i < m; i += nth) tp[tl.off_lam + w.meta[4 * i + 3]] = w.lk[i];
    if (sc.lin == LIN_DIRECT) {
      for (int i = tid; i < sc.n_groups * tri_size(sc.pg); i += nth) tp[tl.off_G + i] = w.G[i];
      for (int i = tid; i < sc.n_groups * sc.cmax * sc.ldg; i += nth) tp[tl.off_H + i] = w.H[i];
      for (int i = tid; i < tri_size(sc.ss); i += nth) tp[tl.off_S + i] = w.S[i];
    }
  }
  // outputs: q+ (normalised quaternions), u+, lambda+, impulses h lambda, contact ids
  Real* so = reinterpret_cast<Real*>(a.state_out);
  Real* imp = reinterpret_cast<Real*>(a.impulses);
  for (int b = tid; b < nb; b += nth) {
    Real qp[7];
    kin_body<Real, Real>(w.qm + 7 * b, w.uk + 6 * b, h, qp);
    Real nq = ssqrt(qp[3] * qp[3] + qp[4] * qp[4] + qp[5] * qp[5] + qp[6] * qp[6]);
    for (int c = 3; c < 7; ++c) qp[c] /= nq;
    for (int c = 0; c < 7; ++c) so[(size_t)(7 * b + c) * ld + world] = qp[c];
    for (int c = 0; c < 6; ++c) so[(size_t)(7 * nb + 6 * b + c) * ld + world] = w.uk[6 * b + c];
  }
  for (int i = tid; i < sc.m_max; i += nth) {
    so[(size_t)(13 * nb + i) * ld + world] = Real(0);
    if (imp) imp[(size_t)i * ld + world] = Real(0);
  }
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    int li = w.meta[4 * i + 3];
    so[(size_t)(13 * nb + li) * ld + world] = w.lk[i];
    if (imp) imp[(size_t)li * ld + world] = Real(h) * w.lk[i];
  }
  if (a.ids)
    for (int sl = tid; sl < sc.n_slots; sl += nth) a.ids[(size_t)sl * ld + world] = w.sact[sl] ? w.sid[sl] : -1;
  if (tid == 0) {
    if (a.status) a.status[world] = status;
    if (a.cost) a.cost[world] = k;
    if (a.iters) a.iters[world] = k | (m << 16);
  }
}

// At most 128 threads per world, registers capped for 3 such CTAs per SM (164 in FP32,
// no spills; 6 CTAs of 64 threads, the robot world's FP32 setting, fit as well).  A cap
// for 7 CTAs of 64 threads (128 registers; the robot world's FP32 working set fits 7 per
// SM) made the 8192-world step slower, 7.12 ms against 6.70 ms: the capped code spills
// and instruction-fetch stalls grow with the extra CTA (1.5 -> 2.6 per issue).
template <class Real>
__global__ void __launch_bounds__(128, 3) step_kernel(const DevScene scp, const StepArgs a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ __align__(16) DevScene ssc;
  scene_to_shared(scp, ssc);
  WS<Real> w = ws_carve<Real>(smem, ssc);
  if (!a.queue) {
    step_world<Real>(ssc, w, a, blockIdx.x);
    return;
  }
  // persistent: take work items until the queue is exhausted (no CTA waits on another)
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) w.ints[15] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = w.ints[15];
    if (it >= a.n_items) break;
    step_world<Real>(ssc, w, a, a.order ? a.order[it] : it);
  }
}

// Heaviest-first order of the worlds by their previous step's Newton iterations (a
// counting sort over 0..63, one CTA): worlds that took the most iterations start first,
// so the last wave is short.  Worlds of equal count may come in any order; a world's
// result does not depend on when it runs.
static __global__ void lpt_order_kernel(const int32_t* cost, int n, int32_t* order) {
  __shared__ int bins[64], start[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int c = cost[i];
    c = c < 0 ? 0 : (c > 63 ? 63 : c);
    atomicAdd(&bins[c], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 63; c >= 0; --c) { start[c] = acc; acc += bins[c]; }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int c = cost[i];
    c = c < 0 ? 0 : (c > 63 ? 63 : c);
    order[atomicAdd(&start[c], 1)] = i;
  }
}

// ---------------------------------------------------------------------------
// adjoint kernel
// ---------------------------------------------------------------------------
// Body part of Psi: g_q . q+(q-) + w_u . (M(q-)(u* - u-) - h f(q-, u-)), along (b, dc).
template <class Real>
__device__ Real body_vjp(const DevScene& sc, const WS<Real>& w, int b, int dc, const Real* gq, const Real* wu, double h) {
  typedef dual<Real> D;
  D qm[7], qp[7];
  for (int c = 0; c < 7; ++c) qm[c] = D(w.qm[7 * b + c], c == dc ? Real(1) : Real(0));
  kin_body<D, Real>(qm, w.uk + 6 * b, h, qp);
  D acc(Real(0));
  for (int c = 0; c < 7; ++c) acc = acc + D(gq[7 * b + c]) * qp[c];
  // angular part depends on q- through I_w(q-) = R diag(I) R^T
  vec3<D> dw = v3(D(w.uk[6 * b + 3] - w.um[6 * b + 3]), D(w.uk[6 * b + 4] - w.um[6 * b + 4]), D(w.uk[6 * b + 5] - w.um[6 * b + 5]));
  vec3<D> om = v3(D(w.um[6 * b + 3]), D(w.um[6 * b + 4]), D(w.um[6 * b + 5]));
  auto Iw_apply = [&](vec3<D> v) {
    vec3<D> vb = v3(D(Real(0)), D(Real(0)), D(Real(0)));
    // R^T v via rotating by the conjugate quaternion
    D qc[4] = {qm[3], D(Real(0)) - qm[4], D(Real(0)) - qm[5], D(Real(0)) - qm[6]};
    vb = qrot(qc, v);
    vb = v3(vb.x * D(Real(sc.inertia[b][0])), vb.y * D(Real(sc.inertia[b][1])), vb.z * D(Real(sc.inertia[b][2])));
    return qrot(qm + 3, vb);
  };
  vec3<D> Idw = Iw_apply(dw);
  vec3<D> gy = cross3(om, Iw_apply(om));        // f_ang = -gy
  vec3<D> ra = Idw + scale(gy, D(Real(h)));     // angular r_dyn minus the lambda terms
  acc = acc + D(wu[6 * b + 3]) * ra.x + D(wu[6 * b + 4]) * ra.y + D(wu[6 * b + 5]) * ra.z;
  return acc.d;
}

}  // namespace ost
#include "ostrich_adjoint.cuh"
namespace ost {

// One world's adjoint (Sec. III-D) in mode MODE (ADJ_PAPER or ADJ_EXACT).
template <class Real, int MODE>
__global__ void __launch_bounds__(128, 3) adjoint_kernel(const DevScene scp, const AdjArgs a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ __align__(16) DevScene ssc;
  __shared__ int bgl[NB_CAP * GROUPS_PER_BODY], bgn[NB_CAP], item0[NB_CAP + 1];
  __shared__ int ncon[NB_CAP], jpre[NB_CAP + 1], cpre[NB_CAP + 1];
  scene_to_shared(scp, ssc);
  const DevScene& sc = ssc;
  WS<Real> w = ws_carve<Real>(smem, sc);
  ExWS<Real> ex = {};
  if (MODE == ADJ_EXACT) ex = ex_carve<Real>(smem + ws_bytes<Real>(sc), sc);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int world = a.list ? a.list[blockIdx.x] : a.world0 + blockIdx.x;
  if (world < 0 || world >= a.n_worlds) return;
  const int slot = a.list ? (a.list_slot ? a.list_slot[blockIdx.x] : -1) : 0;
  if (slot < 0 || (a.list && slot >= a.tape_slots)) return;
  const int ld = a.ld, nb = sc.nb;
  const double h = a.h;
  const Real hR = Real(h);
  const TapeLayout tl = tape_layout(sc);
  const Real* tp = reinterpret_cast<const Real*>(a.tape) + ((size_t)slot * a.n_worlds + world) * tl.total;
  if (sc.lin == LIN_DIRECT) {
    // the taped factor, copied to shared memory in the background of the setup and the
    // evaluation (neither touches G, H or S); awaited before the solve
    for (int i = tid; i < sc.n_groups * tri_size(sc.pg); i += nth) cp_async_elem(w.G + i, tp + tl.off_G + i);
    for (int i = tid; i < sc.n_groups * sc.cmax * sc.ldg; i += nth) cp_async_elem(w.H + i, tp + tl.off_H + i);
    for (int i = tid; i < tri_size(sc.ss); i += nth) cp_async_elem(w.S + i, tp + tl.off_S + i);
    cp_async_commit();
  }
  Src<Real> sq = {tp + tl.off_qm, 1}, su = {tp + tl.off_um, 1}, sb = {tp + tl.off_ubar, 1};
  world_setup<Real>(sc, w, sq, su, sb, h, (Real*)nullptr, tp + tl.off_ct);   // the step's contact set
  const int m = w.ints[0], mc = w.ints[1];
  for (int i = tid; i < 6 * nb; i += nth) w.uk[i] = tp[tl.off_u + i];
  for (int i = tid; i < m; i += nth) w.lk[i] = tp[tl.off_lam + w.meta[4 * i + 3]];
  __syncthreads();
  evaluate(sc, w, w.uk, w.lk, h, false);   // J (with E at u*), C, delta, poses at q+
  if (tid == 0) {
    body_groups(sc, w, bgl, bgn);
    int acc = 0;
    for (int b = 0; b < nb; ++b) { item0[b] = acc; acc += 7 * (bgn[b] + 1); }
    item0[nb] = acc;
    // work order of the pull-back items by cost: joint groups, contact groups, body terms
    int aj = 0, ac = 0;
    for (int b = 0; b < nb; ++b) {
      int nc = 0;
      while (nc < bgn[b] && bgl[b * GROUPS_PER_BODY + nc] < sc.n_slots) ++nc;
      ncon[b] = nc;
      jpre[b] = aj; aj += 7 * (bgn[b] - nc);
      cpre[b] = ac; ac += 7 * nc;
    }
    jpre[nb] = aj; cpre[nb] = ac;
  }
  if (sc.lin == LIN_DIRECT) {
    cp_async_wait_all();     // this thread's copies of the taped factor; the barrier below
                             // (before the solve) makes every thread's visible
  } else if (MODE == ADJ_EXACT) {
    // PCR mode tapes no factor: the exact mode's GMRES preconditioner is the direct factor,
    // formed here at the taped iterate
    assemble(sc, w, h);
    factor(sc, w, h);
  } else if (sc.pc == PC_BLOCK) {
    // the PCR operator and preconditioner of the forward pass, at the taped iterate
    assemble(sc, w, h);
    factor_blocks(sc, w);
  } else {
    pcr_jacobi(sc, w, h);
  }
  // incoming cotangent: normalisation Jacobian of the output quaternions, then g
  Real* gq = w.lb;      // the best-iterate buffer is free in the adjoint; m_max >= 7 nb
  Real* gu = w.du;
  const Real* din = reinterpret_cast<const Real*>(a.dL_dnext);
  for (int b = tid; b < nb; b += nth) {
    Real qp[7];
    kin_body<Real, Real>(w.qm + 7 * b, w.uk + 6 * b, h, qp);
    Real nq = ssqrt(qp[3] * qp[3] + qp[4] * qp[4] + qp[5] * qp[5] + qp[6] * qp[6]);
    Real qh[4] = {qp[3] / nq, qp[4] / nq, qp[5] / nq, qp[6] / nq};
    Real gin[4];
    for (int c = 0; c < 4; ++c) gin[c] = din[(size_t)(7 * b + 3 + c) * ld + world];
    Real dp = qh[0] * gin[0] + qh[1] * gin[1] + qh[2] * gin[2] + qh[3] * gin[3];
    for (int c = 0; c < 3; ++c) gq[7 * b + c] = din[(size_t)(7 * b + c) * ld + world];
    for (int c = 0; c < 4; ++c) gq[7 * b + 3 + c] = (gin[c] - qh[c] * dp) / nq;
    for (int c = 0; c < 6; ++c) gu[6 * b + c] = din[(size_t)(7 * nb + 6 * b + c) * ld + world];
    // g = grad_u L + h G(q-)^T grad_q L; G^T for the quaternion block is 1/2 vec(g (x) q-*)
    const Real* q = w.qm + 7 * b + 3;
    const Real* g4 = gq + 7 * b + 3;
    Real vx = -g4[0] * q[1] + g4[1] * q[0] - g4[2] * q[3] + g4[3] * q[2];
    Real vy = -g4[0] * q[2] + g4[1] * q[3] + g4[2] * q[0] - g4[3] * q[1];
    Real vz = -g4[0] * q[3] - g4[1] * q[2] + g4[2] * q[1] + g4[3] * q[0];
    gu[6 * b] += hR * gq[7 * b]; gu[6 * b + 1] += hR * gq[7 * b + 1]; gu[6 * b + 2] += hR * gq[7 * b + 2];
    gu[6 * b + 3] += hR * Real(0.5) * vx; gu[6 * b + 4] += hR * Real(0.5) * vy; gu[6 * b + 5] += hR * Real(0.5) * vz;
    Real mg[6];
    minv6(sc, w, b, gu + 6 * b, mg);
    for (int c = 0; c < 6; ++c) w.mr[6 * b + c] = mg[c];
  }
  __syncthreads();
  Real* wl = w.dl;
  Real* wu = w.ub;
  if (MODE == ADJ_PAPER) {
    // Eq. (18): A w_lambda = -h J M^-1 g, with the forward factor (the refinement's
    // matrix-free product takes delta as the evaluation at the iterate formed it, scal[2]);
    // the right-hand side is formed with exact products: its rounding would otherwise
    // reach the null space of J^T, where A's eigenvalue is only kappa
    for (int i = tid; i < m; i += nth) {
      const Real* Ji = w.J + 12 * i;
      int b0 = w.meta[4 * i + 1], b1 = w.meta[4 * i + 2];
      acc2<Real> jm;
      for (int k = 0; k < 6; ++k) jm.add_prod(Ji[k], w.mr[6 * b0 + k]);
      if (b1 >= 0) for (int k = 0; k < 6; ++k) jm.add_prod(Ji[6 + k], w.mr[6 * b1 + k]);
      w.rhs[i] = -hR * jm.value();
    }
    __syncthreads();
    if (sc.lin == LIN_DIRECT) {
      // refined until a correction no longer changes w_lambda at working precision (at
      // most refine_adj sweeps)
      schur_solve(sc, w, w.rhs, wl, w.f, w.lt, h, sc.refine_adj, Real(sizeof(Real) == 4 ? 1.2e-7 : 0.0));
    } else {
      // a single PCR solve with the forward pass's operator and preconditioner (Sec. III-D)
      int pconv = 0;
      const int its = pcr_solve_refined<Real>(sc, w, w.rhs, wl, sc.pcr_iters_adj, Real(sc.pcr_rtol_adj), w.f, w.lt,
                                              w.tmp2, h, &pconv);
      if (tid == 0 && a.krylov) a.krylov[world] = its | (pconv ? 0 : (1 << 16));
    }
    // Eq. (19): w_u = -M^-1 (g + J^T w_lambda)
    jt_apply_acc(sc, w, wl, w.f);     // f is free now
    __syncthreads();
    for (int b = tid; b < nb; b += nth) {
      Real t[6], o[6];
      for (int c = 0; c < 6; ++c) t[c] = gu[6 * b + c] + w.f[6 * b + c];
      minv6(sc, w, b, t, o);
      for (int c = 0; c < 6; ++c) wu[6 * b + c] = -o[c];
    }
    __syncthreads();
  } else {
    // exact IFT: local Jacobians of every group at the returned iterate, then GMRES on
    // J_F^T [w_u; w_lambda] = [-g; 0] preconditioned by the paper's matrix
    exact_slot_terms(sc, w, ex, h);
    __syncthreads();
    for (int task = tid; task < 6 * nb; task += nth) exact_task(sc, w, ex, bgl, bgn, task / 6, task % 6, h);
    for (int i = tid; i < 6 * nb; i += nth) ex.r[i] = -gu[i];
    for (int i = tid; i < m; i += nth) ex.r[6 * nb + i] = Real(0);
    __syncthreads();
    Real msum = Real(0);
    for (int b = 0; b < nb; ++b) msum += Real(sc.mass[b]);
    const Real sigma = msum / (Real(nb) * hR);
    int conv = 0;
    const int its = exact_gmres(sc, w, ex, h, sigma, Real(sizeof(Real) == 4 ? 1e-6 : 1e-13), &conv);
    for (int i = tid; i < 6 * nb; i += nth) wu[i] = ex.x[i];
    for (int i = tid; i < m; i += nth) wl[i] = ex.x[6 * nb + i];
    if (tid == 0 && a.krylov) a.krylov[world] = its | (conv ? 0 : (1 << 16));
    __syncthreads();
  }
  // Eq. (17) with xi = theta, the physical parameters: explicit partials of the rows
  // that hold them, contracted with the adjoint.  Servo gain k_p: the servo row of
  // Eq. (8) holds lambda_c / k_p, so d/dk_p = -lambda_c / k_p^2.  Body mass m_b: the
  // linear rows of Eq. (10), m_b (v - v-) - h m_b g, so d/dm_b = (v - v-) - h g e_z.
  // Principal moment I_k: the angular rows, I_w (w - w-) + h w- x (I_w w-) with
  // I_w = R diag(I) R^T at q-, so d/dI_k = r_k (r_k . (w - w-)) + h (r_k . w-) (w- x r_k),
  // r_k the k-th column of R(q-).  Friction coefficient mu (exact mode; the paper's
  // frozen W holds it): the friction rows of Eq. (7) through W.
  if (a.dL_dkp) {
    Real* dkp = reinterpret_cast<Real*>(a.dL_dkp);
    for (int i = mc + 5 * sc.nj + tid; i < m; i += nth) {
      // d alpha / d k_p: -1/k_p^2 (velocity target), -h/(k_d + h k_p)^2 (position target)
      const int j = w.ref[i];
      const Real al = Real(servo_alpha(sc, j, h));
      const Real dal = sc.smode[j] == SERVO_POSITION ? -hR * al * al : -al * al;
      dkp[(size_t)(i - mc - 5 * sc.nj) * ld + world] = wl[i] * w.lk[i] * dal;
    }
  }
  if (a.dL_dmass) {
    Real* dm = reinterpret_cast<Real*>(a.dL_dmass);
    for (int b = tid; b < nb; b += nth) {
      Real acc = 0;
      for (int k = 0; k < 3; ++k) acc += wu[6 * b + k] * (w.uk[6 * b + k] - w.um[6 * b + k]);
      acc += wu[6 * b + 2] * (-hR * Real(sc.g));
      dm[(size_t)b * ld + world] = acc;
    }
  }
  if (a.dL_dinertia) {
    Real* di = reinterpret_cast<Real*>(a.dL_dinertia);
    for (int b = tid; b < nb; b += nth) {
      Real R[9];
      qmat(w.qm + 7 * b + 3, R);                 // R(q-); w.R holds R(q+) after the evaluation
      const vec3<Real> wm = v3(w.um[6 * b + 3], w.um[6 * b + 4], w.um[6 * b + 5]);
      const vec3<Real> dw = v3(w.uk[6 * b + 3] - wm.x, w.uk[6 * b + 4] - wm.y, w.uk[6 * b + 5] - wm.z);
      const vec3<Real> ww = v3(wu[6 * b + 3], wu[6 * b + 4], wu[6 * b + 5]);
      for (int k = 0; k < 3; ++k) {
        const vec3<Real> rk = v3(R[k], R[3 + k], R[6 + k]);
        const vec3<Real> c = cross3(wm, rk);
        const Real s1 = dot3(rk, dw), s2 = hR * dot3(rk, wm);
        di[(size_t)(3 * b + k) * ld + world] =
            ww.x * (rk.x * s1 + c.x * s2) + ww.y * (rk.y * s1 + c.y * s2) + ww.z * (rk.z * s1 + c.z * s2);
      }
    }
  }
  if (a.dL_dmu) {
    Real part = Real(0);
    if (MODE == ADJ_EXACT) {
      typedef dual<Real> D;
      for (int sl = tid; sl < sc.n_slots; sl += nth) {
        if (!w.sact[sl]) continue;
        const int i = w.srow[sl], b = sc.slot_body[sl];
        CGroup<Real> g;
        contact_group<Real, Real>(sc, w, sl, b, w.qm + 7 * b, w.uk + 6 * b, h, g);
        D rf[2];
        friction_rows<D, Real>(sc, D(g.vel[1]), D(g.vel[2]), D(w.lk[i]), w.lk[i + 1], w.lk[i + 2],
                               hR * w.swhat[sl], D(Real(sc.mu), Real(1)), rf);
        part += wl[i + 1] * rf[0].d + wl[i + 2] * rf[1].d;
      }
    }
    const Real tot = block_sum(w, part);
    if (tid == 0) reinterpret_cast<Real*>(a.dL_dmu)[world] = tot;
  }
  // dL/du- = -M w_u - h (df/du-)^T w_u ;  dL/dubar = -w_lambda of the servo rows
  Real* dout = reinterpret_cast<Real*>(a.dL_dstate);
  for (int b = tid; b < nb; b += nth) {
    Real mb = Real(sc.mass[b]);
    for (int c = 0; c < 3; ++c) dout[(size_t)(7 * nb + 6 * b + c) * ld + world] = -mb * wu[6 * b + c];
    vec3<Real> wa = v3(wu[6 * b + 3], wu[6 * b + 4], wu[6 * b + 5]);
    vec3<Real> om = v3(w.um[6 * b + 3], w.um[6 * b + 4], w.um[6 * b + 5]);
    vec3<Real> Iwa = mat3<Real>(w.Iw + 9 * b, wa);
    vec3<Real> t1 = mat3<Real>(w.Iw + 9 * b, cross3(om, wa));
    vec3<Real> t2 = cross3(mat3<Real>(w.Iw + 9 * b, om), wa);
    vec3<Real> d = v3(-Iwa.x - hR * (t1.x - t2.x), -Iwa.y - hR * (t1.y - t2.y), -Iwa.z - hR * (t1.z - t2.z));
    dout[(size_t)(7 * nb + 6 * b + 3) * ld + world] = d.x;
    dout[(size_t)(7 * nb + 6 * b + 4) * ld + world] = d.y;
    dout[(size_t)(7 * nb + 6 * b + 5) * ld + world] = d.z;
  }
  for (int i = tid; i < sc.m_max; i += nth) dout[(size_t)(13 * nb + i) * ld + world] = Real(0);
  Real* dctl = reinterpret_cast<Real*>(a.dL_dcontrols);
  if (dctl)   // d b_c / d target: -1 (velocity target), -1/h (position target)
    for (int i = mc + 5 * sc.nj + tid; i < m; i += nth)
      dctl[(size_t)(i - mc - 5 * sc.nj) * ld + world] = sc.smode[w.ref[i]] == SERVO_POSITION ? -wl[i] / hR : -wl[i];
  // dL/dq-: one work item per (body b, coordinate c of its q-, group touching b or the
  // body's own terms), each a dual-number evaluation along that coordinate; the items of a
  // coordinate are summed in a fixed order
  const bool trunc = MODE == ADJ_PAPER && sc.pullback == 1;
  Real* item = w.G;     // the factor (G, E, H, S, one carved run) is no longer needed;
                        // sum_b 7 (groups_b + 1) <= 14 m_max items
  // taken in cost order (every joint item, then every contact item, then the body terms)
  // so that the threads' loads even out; each item is stored at its place in the per-body
  // layout, which fixes the order of the sums below
  const int n_items = item0[nb], nj_items = jpre[nb], nc_items = cpre[nb];
  for (int e = tid; e < n_items; e += nth) {
    int b = 0, c, k;
    if (e < nj_items) {
      while (e >= jpre[b + 1]) ++b;
      const int nj = bgn[b] - ncon[b], r = e - jpre[b];
      c = r / nj;
      k = 1 + ncon[b] + (r - c * nj);
    } else if (e < nj_items + nc_items) {
      const int e2 = e - nj_items;
      while (e2 >= cpre[b + 1]) ++b;
      const int nc = ncon[b], r = e2 - cpre[b];
      c = r / nc;
      k = 1 + (r - c * nc);
    } else {
      const int e3 = e - nj_items - nc_items;
      b = e3 / 7;
      c = e3 - 7 * b;
      k = 0;
    }
    item[item0[b] + c * (bgn[b] + 1) + k] =
        k == 0 ? body_vjp(sc, w, b, c, gq, wu, h)
               : group_vjp_q<Real, MODE>(sc, w, ex, bgl[b * GROUPS_PER_BODY + k - 1], b, c, wl, wu, trunc, h);
  }
  __syncthreads();
  for (int e = tid; e < nb * 7; e += nth) {
    const int b = e / 7, c = e % 7;
    acc2<Real> acc;        // the terms cancel strongly: compensated sum
    const int base = item0[b] + c * (bgn[b] + 1);
    for (int k = 0; k <= bgn[b]; ++k) acc.add(item[base + k]);
    dout[(size_t)(7 * b + c) * ld + world] = acc.value();
  }
}

// ---------------------------------------------------------------------------
// launchers (called by the C ABI)
// ---------------------------------------------------------------------------
// The dynamic shared-memory limit of a kernel is raised once per device and size; a
// launch inside a stream capture then issues nothing but the launch itself.
template <class K> cudaError_t ensure_smem(K kernel, size_t smem, int* done_dev, size_t* done_size) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && done_size[dev] >= smem && done_dev[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // all of the unified L1 as shared memory: the working sets live there, global traffic is small
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && dev < 64) { done_dev[dev] = 1; if (smem > done_size[dev]) done_size[dev] = smem; }
  return e;
}

template <class Real>
cudaError_t launch_step(const DevScene& sc, const StepArgs& a, int threads, cudaStream_t st) {
  static int done_dev[64] = {0};
  static size_t done_size[64] = {0};
  auto kernel = step_kernel<Real>;
  size_t smem = ws_bytes<Real>(sc);
  cudaError_t e = ensure_smem(kernel, smem, done_dev, done_size);
  if (e != cudaSuccess) return e;
  int n = a.list ? a.n_list : a.n_worlds - a.world0;
  if (n <= 0) return cudaSuccess;
  if (a.queue) {
    // persistent: as many CTAs as fit on the device at once, fed from the queue
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess)
      return e;
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm < n ? sms * per_sm : n;
    if ((e = cudaMemsetAsync(a.queue, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (a.order && a.cost) {
      lpt_order_kernel<<<1, 1024, 0, st>>>(a.cost + a.world0, n, const_cast<int32_t*>(a.order));
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    StepArgs b = a;
    b.n_items = n;
    kernel<<<grid, threads, smem, st>>>(sc, b);
    return cudaGetLastError();
  }
  kernel<<<n, threads, smem, st>>>(sc, a);
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_adjoint(const DevScene& sc, const AdjArgs& a, int threads, cudaStream_t st) {
  static int done_dev[2][64] = {{0}};
  static size_t done_size[2][64] = {{0}};
  const int mode = a.mode == ADJ_EXACT ? ADJ_EXACT : ADJ_PAPER;
  auto kernel = mode == ADJ_EXACT ? adjoint_kernel<Real, ADJ_EXACT> : adjoint_kernel<Real, ADJ_PAPER>;
  const size_t smem = adj_smem_bytes<Real>(sc, mode);
  cudaError_t e = ensure_smem(kernel, smem, done_dev[mode], done_size[mode]);
  if (e != cudaSuccess) return e;
  int n = a.list ? a.n_list : a.n_worlds - a.world0;
  if (n <= 0) return cudaSuccess;
  kernel<<<n, threads, smem, st>>>(sc, a);
  return cudaGetLastError();
}


// Bytes the carve of one world actually consumes from a 16-byte aligned base; the
// context refuses a scene for which this exceeds ws_bytes (checked on the host).
template <class Real> size_t ws_used(const DevScene& s) {
  alignas(16) static char probe[16];
  char* base = probe;
  WS<Real> w = ws_carve<Real>(base, s);
  return (size_t)(reinterpret_cast<char*>(w.pcr ? w.pcr + 7 * s.m_max : w.scal + 8) - base);
}

template cudaError_t launch_step<OST_REAL>(const DevScene&, const StepArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint<OST_REAL>(const DevScene&, const AdjArgs&, int, cudaStream_t);
template size_t ws_bytes<OST_REAL>(const DevScene&);
template size_t ws_used<OST_REAL>(const DevScene&);
template size_t adj_smem_bytes<OST_REAL>(const DevScene&, int);

}  // namespace ost
