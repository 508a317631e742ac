// IFT adjoint of the Ostrich step (Sec. III-D), organised by constraint groups.
//
// A group is the set of rows one geometric object produces: a contact slot gives its
// normal row and its two friction rows (Eqs. (4), (7)), a revolute joint its three
// anchor rows, its two axis-alignment rows (Eq. (3)) and its velocity servo (Eq. (8)).
// All rows of a group depend on q-, u+ and the multipliers only through the poses and
// velocities of the group's (at most two) bodies, so one forward-mode dual evaluation
// of a group along one coordinate of one body gives the derivatives of all its rows.
//
// Two modes:
//   paper  Eqs. (18)-(19) with the forward Schur matrix at the returned iterate, W and
//          the FB scalings frozen (Sec. III-B, III-D), solved with the taped factor;
//   exact  the implicit-function theorem with the full Jacobian of the residual in
//          (u+, lambda+): W's dependence on the slip velocities and on lambda_n, the
//          velocity dependence of the friction and servo rows' Jacobians, and the
//          geometric stiffness -h sum_i lambda_i dJ_i^T/du.  The transposed system
//          J_F^T w = [-g; 0] is solved by GMRES in the world's shared memory, right-
//          preconditioned by the paper's matrix (the taped factor).
// The vector-Jacobian products of Eq. (17) then contract w with the partial derivatives
// of the residual in q-, u-, the servo targets and the physical parameters.
#pragma once
// Included by ostrich_kernels.cuh after the step kernel (it uses WS, evaluate() and the
// factor solves defined there).

namespace ost {

constexpr int ADJ_PAPER = 0;
constexpr int ADJ_EXACT = 1;
constexpr int KRYLOV = 20;       // GMRES restart length of the exact mode
constexpr int KRYLOV_CYCLES = 3; // at most 60 Krylov iterations
constexpr int GROUPS_PER_BODY = SLOT_CAP / 2 + NJ_CAP;

// ---------------------------------------------------------------------------
// group evaluators in any scalar type S (Real or dual<Real>)
// ---------------------------------------------------------------------------
template <class S> struct CGroup {
  vec3<S> dir[3];   // n, t1, t2 (world frame)
  vec3<S> ang[3];   // angular parts of the three Jacobian rows, through E^T
  S cn;             // signed distance n . x - d
  S vel[3];         // J_k u
};

// Contact slot sl of body b at q- (qm7) and u+ (u6), both in S; the frame is the slot's
// (a box edge's normal follows the rim centre at q-), the point the rim's deepest point
// at q+ or the box corner; the same geometry as evaluate().
template <class S, class Real>
__device__ __forceinline__ void contact_group(const DevScene& sc, const WS<Real>& w, int sl, int b, const S* qm7,
                                              const S* u6, double h, CGroup<S>& o) {
  const int local = sl - sc.slot_base[b];
  S qp[7];
  kin_body<S, S>(qm7, u6, h, qp);
  vec3<S> n;
  S d;
  const Real ns[3] = {w.sn[3 * sl], w.sn[3 * sl + 1], w.sn[3 * sl + 2]};
  slot_frame2<S, Real>(sc, b, local, w.sftype[sl], qm7, ns, w.sd[sl], w.sedge + 2 * sl, n, d);
  vec3<S> t1, t2;
  tangent_basis(n, t1, t2);
  const vec3<S> p = v3(qp[0], qp[1], qp[2]);
  const vec3<S> x = slot_point<S>(sc, b, local, p, qp + 3, n);
  const vec3<S> lev = x - p;
  const vec3<S> wk = v3(u6[3], u6[4], u6[5]);
  const vec3<S> ul = v3(u6[0], u6[1], u6[2]);
  o.dir[0] = n; o.dir[1] = t1; o.dir[2] = t2;
  const MapE<S> Ek(wk, h);
  for (int k = 0; k < 3; ++k) {
    o.ang[k] = Ek(cross3(lev, o.dir[k]));
    o.vel[k] = dot3(o.dir[k], ul) + dot3(o.ang[k], wk);
  }
  o.cn = dot3(n, x) - d;
}

// The contact rows of slot sl with q- in S and u+ held (real): what the q- pull-back of
// Eq. (17) takes from them -- the signed distance cn, the row velocities vel_k = J_k u+ and
// the products jw_k = J_k . w_u -- with the angular parts' E applied to the constant
// vectors instead of to each row, (E a) . v = a . (E^T v); the same geometry as
// contact_group.
template <class S, class Real>
__device__ __forceinline__ void contact_rows_dot(const DevScene& sc, const WS<Real>& w, int sl, int b, const S* qm7,
                                                 const Real* u6, double h, vec3<Real> wlin, vec3<Real> wang, S& cn,
                                                 S* vel, S* jw) {
  const int local = sl - sc.slot_base[b];
  S qp[7];
  kin_body<S, Real>(qm7, u6, h, qp);
  vec3<S> n;
  S d;
  const Real ns[3] = {w.sn[3 * sl], w.sn[3 * sl + 1], w.sn[3 * sl + 2]};
  slot_frame2<S, Real>(sc, b, local, w.sftype[sl], qm7, ns, w.sd[sl], w.sedge + 2 * sl, n, d);
  vec3<S> t1, t2;
  tangent_basis(n, t1, t2);
  const vec3<S> p = v3(qp[0], qp[1], qp[2]);
  const vec3<S> x = slot_point<S>(sc, b, local, p, qp + 3, n);
  const vec3<S> lev = x - p;
  const vec3<Real> wk = v3(u6[3], u6[4], u6[5]), ul = v3(u6[0], u6[1], u6[2]);
  const MapE<Real> Ek(wk, h);
  const vec3<Real> ew = Ek.T_(wk), ea = Ek.T_(wang);
  const vec3<S> dir[3] = {n, t1, t2};
  for (int k = 0; k < 3; ++k) {
    const vec3<S> a = cross3(lev, dir[k]);
    vel[k] = dotm(dir[k], ul) + dotm(a, ew);
    jw[k] = dotm(dir[k], wlin) + dotm(a, ea);
  }
  cn = dot3(n, x) - d;
}

// Friction weight W of Eq. (7) (the FB reading, cancellation-free numerator) and the
// friction residuals v_k + (W + kappa) lambda_fk, in S; lambda enters as S so that the
// same code differentiates along lambda_n.
template <class S, class Real>
__device__ __forceinline__ S friction_rows(const DevScene& sc, S v1, S v2, S ln, Real l1, Real l2, Real hw, S mu,
                                           S* rf) {
  const Real eps = Real(sc.eps), kap = Real(sc.kappa);
  const S vt = ssqrt(v1 * v1 + v2 * v2 + S(eps * eps));
  const Real lfn = ssqrt(l1 * l1 + l2 * l2 + eps * eps);
  const S lnp = sval(ln) > Real(0) ? ln : S(Real(0));
  const S g = (mu * lnp - S(lfn)) * hw;
  const S sg = ssqrt(vt * vt + g * g + S(eps * eps));
  const S num = sval(g) > Real(0) ? (vt * vt + S(eps * eps)) / (sg + g) : sg - g;
  S den = mu * lnp;
  if (sval(den) < Real(1e-12)) den = S(Real(1e-12));
  const S W = num / den;
  rf[0] = v1 + (W + S(kap)) * l1;
  rf[1] = v2 + (W + S(kap)) * l2;
  return W;
}

template <class S> struct JGroup {
  vec3<S> lin_p[5], ang_p[5], lin_c[5], ang_c[5];   // through E
  S c[5];
  vec3<S> sl_p, sa_p, sl_c, sa_c;   // servo row: linear and angular parts (angular through E)
  S sv;                             // servo row: joint rate J_c u
};

// Joint j between parent and child at q- and u+ (in S): the five position rows and the
// servo row, as evaluate() forms them (same geometry helpers).
template <class S>
__device__ __forceinline__ void joint_group(const DevScene& sc, int j, const S* qmp, const S* up, const S* qmc,
                                            const S* uc, double h, JGroup<S>& o) {
  S qpp[7], qpc[7];
  kin_body<S, S>(qmp, up, h, qpp);
  kin_body<S, S>(qmc, uc, h, qpc);
  const QuatRot<S> rotp(qpp + 3), rotc(qpc + 3);
  const vec3<S> pp = v3(qpp[0], qpp[1], qpp[2]), pc = v3(qpc[0], qpc[1], qpc[2]);
  const vec3<S> wp = v3(up[3], up[4], up[5]), wc = v3(uc[3], uc[4], uc[5]);
  const MapE<S> Ep(wp, h), Ec(wc, h);
  joint_rows_each<S>(sc, j, pp, rotp, pc, rotc, [&](int k, vec3<S> lp, vec3<S> ap, vec3<S> lc, vec3<S> ac, S c) {
    o.lin_p[k] = lp; o.lin_c[k] = lc; o.c[k] = c;
    o.ang_p[k] = Ep(ap);
    o.ang_c[k] = Ec(ac);
  });
  SRow<S> sr;
  servo_row_geom<S>(sc, j, pp, rotp, pc, rotc, sr);
  o.sl_p = sr.lin_p; o.sl_c = sr.lin_c;
  o.sa_p = Ep(sr.ang_p);
  o.sa_c = Ec(sr.ang_c);
  o.sv = dot3(o.sl_p, v3(up[0], up[1], up[2])) + dot3(o.sa_p, wp) + dot3(o.sl_c, v3(uc[0], uc[1], uc[2])) +
         dot3(o.sa_c, wc);
}

// The joint coordinate at q- (in S), for a position servo's bias (x(q-) - target)/h.
template <class S>
__device__ __forceinline__ S joint_coord_qm(const DevScene& sc, int j, const S* qmp, const S* qmc) {
  return joint_coord<S>(sc, j, v3(qmp[0], qmp[1], qmp[2]), QuatRot<S>(qmp + 3), v3(qmc[0], qmc[1], qmc[2]),
                        QuatRot<S>(qmc + 3));
}

// ---------------------------------------------------------------------------
// shared-memory region of the exact mode (after the world's WS region)
// ---------------------------------------------------------------------------
template <class Real> struct ExWS {
  Real *K;      // geometric stiffness, nb x nb blocks of 6 x 6: K[(b * nb + c) * 36 + r * 6 + k]
                // = d(r_dyn of body b, component r) / d(u+ of body c, component k), lambda part
  Real *G;      // exact row derivatives d r_i / d u+ (12 per active row, both sides)
  Real *cfn;    // d (friction row k of slot s) / d lambda_n, 2 per slot
  Real *fsc;    // normal-row derivative scale fa / max(fa, 1e-12), 1 per slot
  Real *V, *Hh, *cs, *sn, *gg, *y, *x, *r, *z, *t6, *wred, *scal;
};

template <class Real> __host__ __device__ inline int ex_n(const DevScene& s) { return 6 * s.nb + s.m_max; }

template <class Real> __host__ __device__ ExWS<Real> ex_carve(char* base, const DevScene& s) {
  ExWS<Real> e;
  char* p = base;
  const int nb = s.nb, n = ex_n<Real>(s), ns = s.n_slots > 0 ? s.n_slots : 1;
  e.K = carve<Real>(p, nb * nb * 36);
  e.G = carve<Real>(p, 12 * s.m_max);
  e.cfn = carve<Real>(p, 2 * ns);
  e.fsc = carve<Real>(p, ns);
  e.V = carve<Real>(p, (KRYLOV + 1) * n);
  e.Hh = carve<Real>(p, (KRYLOV + 1) * KRYLOV);
  e.cs = carve<Real>(p, KRYLOV); e.sn = carve<Real>(p, KRYLOV);
  e.gg = carve<Real>(p, KRYLOV + 1); e.y = carve<Real>(p, KRYLOV);
  e.x = carve<Real>(p, n); e.r = carve<Real>(p, n); e.z = carve<Real>(p, n);
  e.t6 = carve<Real>(p, 6 * nb);
  e.wred = carve<Real>(p, 4 * (KRYLOV + 2));
  e.scal = carve<Real>(p, 8);
  return e;
}

template <class Real> __host__ __device__ size_t ex_bytes(const DevScene& s) {
  char* base = reinterpret_cast<char*>(uintptr_t(16));
  ExWS<Real> e = ex_carve<Real>(base, s);
  return (size_t)(reinterpret_cast<char*>(e.scal + 8) - base);
}

// Shared memory of one world in the adjoint kernel of a mode.
template <class Real> __host__ __device__ size_t adj_smem_bytes(const DevScene& s, int mode) {
  size_t b = ws_bytes<Real>(s);
  if (mode == ADJ_EXACT) b = (b + ex_bytes<Real>(s) + 15) & ~(size_t)15;
  return b;
}

// Groups touching each body: slot indices (active slots of the body) then n_slots + j for
// its joints, in a fixed order; built by one thread.
template <class Real> __device__ void body_groups(const DevScene& sc, const WS<Real>& w, int* bgl, int* bgn) {
  for (int b = 0; b < sc.nb; ++b) {
    int k = 0;
    for (int sl = sc.slot_base[b]; sl < sc.slot_base[b] + sc.slot_count[b]; ++sl)
      if (w.sact[sl]) bgl[b * GROUPS_PER_BODY + k++] = sl;
    for (int j = 0; j < sc.nj; ++j)
      if (sc.jp[j] == b || sc.jc[j] == b) bgl[b * GROUPS_PER_BODY + k++] = sc.n_slots + j;
    bgn[b] = k;
  }
}

// Row index of the servo row of joint j (or -1) in the world's active-row order.
template <class Real> __device__ __forceinline__ int servo_row(const DevScene& sc, const WS<Real>& w, int j) {
  return sc.servo_of[j] >= 0 ? w.ints[1] + 5 * sc.nj + sc.servo_of[j] : -1;
}

// ---------------------------------------------------------------------------
// Eq. (17): the q- pull-back of one group along one coordinate (body db, component dc)
// of q-: the derivative of  sum_rows w_row * rlin_row - h lambda_row J_row . w_u  where
// rlin is the row function with u+ and lambda+ held (paper: the velocity of a friction
// row; exact: the whole friction residual, W included; normal rows: c/h, scaled by
// fa / max(fa, 1e-12) in the exact mode as the row is).
// ---------------------------------------------------------------------------
template <class Real, int MODE>
__device__ Real group_vjp_q(const DevScene& sc, const WS<Real>& w, const ExWS<Real>& ex, int grp, int db, int dc,
                            const Real* wl, const Real* wu, bool trunc, double h) {
  typedef dual<Real> D;
  const Real hR = Real(h);
  if (grp < sc.n_slots) {
    const int sl = grp, b = sc.slot_body[sl], i = w.srow[sl];
    if (trunc) {
      // truncated pull-back: frame and material point frozen at the converged state,
      // first-order rigid motion of the contact point in the normal row only
      D qm[7], qp[7];
      for (int c = 0; c < 7; ++c) qm[c] = D(w.qm[7 * b + c], c == dc ? Real(1) : Real(0));
      kin_body<D, Real>(qm, w.uk + 6 * b, h, qp);
      Real qpv[7];
      for (int c = 0; c < 7; ++c) qpv[c] = qp[c].v;
      const vec3<Real> n = v3(w.sn[3 * sl], w.sn[3 * sl + 1], w.sn[3 * sl + 2]);
      const vec3<Real> pv = v3(qpv[0], qpv[1], qpv[2]);
      const int local = sl - sc.slot_base[b];
      const vec3<Real> xs = slot_point<Real>(sc, b, local, pv, qpv + 3, n);
      Real Rs[9];
      qmat(qpv + 3, Rs);
      const vec3<Real> rho = mat3T<Real>(Rs, xs - pv);
      const vec3<D> x = v3(qp[0], qp[1], qp[2]) + qrot(qp + 3, lift<D>(rho));
      const D c = dot3(lift<D>(n), x) - D(w.sd[sl]);
      return (wl[i] * c / D(hR)).d;
    }
    D qm[7];
    for (int c = 0; c < 7; ++c) qm[c] = D(w.qm[7 * b + c], c == dc ? Real(1) : Real(0));
    D cn, vel[3], jw[3];
    contact_rows_dot<D, Real>(sc, w, sl, b, qm, w.uk + 6 * b, h, v3(wu[6 * b], wu[6 * b + 1], wu[6 * b + 2]),
                              v3(wu[6 * b + 3], wu[6 * b + 4], wu[6 * b + 5]), cn, vel, jw);
    D acc(Real(0));
    // normal row
    const Real fs = MODE == ADJ_EXACT ? ex.fsc[sl] : Real(1);
    acc = acc + D(wl[i] * fs) * cn / D(hR);
    // friction rows
    if (MODE == ADJ_EXACT) {
      D rf[2];
      friction_rows<D, Real>(sc, vel[1], vel[2], D(w.lk[i]), w.lk[i + 1], w.lk[i + 2], hR * w.swhat[sl],
                             D(Real(sc.mu)), rf);
      acc = acc + D(wl[i + 1]) * rf[0] + D(wl[i + 2]) * rf[1];
    } else {
      acc = acc + D(wl[i + 1]) * vel[1] + D(wl[i + 2]) * vel[2];
    }
    // force terms -h lambda J . w_u of the three rows
    for (int k = 0; k < 3; ++k) acc = acc - D(hR * w.lk[i + k]) * jw[k];
    return acc.d;
  }
  const int j = grp - sc.n_slots, bp = sc.jp[j], bc = sc.jc[j];
  D qmp[7], qmc[7], qpp[7], qpc[7];
  for (int c = 0; c < 7; ++c) {
    qmp[c] = D(w.qm[7 * bp + c], (bp == db && c == dc) ? Real(1) : Real(0));
    qmc[c] = D(w.qm[7 * bc + c], (bc == db && c == dc) ? Real(1) : Real(0));
  }
  // the joint's rows as joint_group forms them, each contracted as soon as it is formed
  kin_body<D, Real>(qmp, w.uk + 6 * bp, h, qpp);
  kin_body<D, Real>(qmc, w.uk + 6 * bc, h, qpc);
  const QuatRot<D> rotp(qpp + 3), rotc(qpc + 3);
  const vec3<D> pp = v3(qpp[0], qpp[1], qpp[2]), pc = v3(qpc[0], qpc[1], qpc[2]);
  // u+ and the adjoint w_u are constants along q-: kept in the working precision
  const vec3<Real> wp = v3(w.uk[6 * bp + 3], w.uk[6 * bp + 4], w.uk[6 * bp + 5]);
  const vec3<Real> wc = v3(w.uk[6 * bc + 3], w.uk[6 * bc + 4], w.uk[6 * bc + 5]);
  const vec3<Real> wpl = v3(wu[6 * bp], wu[6 * bp + 1], wu[6 * bp + 2]);
  const vec3<Real> wpa = v3(wu[6 * bp + 3], wu[6 * bp + 4], wu[6 * bp + 5]);
  const vec3<Real> wcl = v3(wu[6 * bc], wu[6 * bc + 1], wu[6 * bc + 2]);
  const vec3<Real> wca = v3(wu[6 * bc + 3], wu[6 * bc + 4], wu[6 * bc + 5]);
  const int i0 = w.ints[1] + 5 * j;
  D acc(Real(0));
  // the rows' angular parts enter through E (u+ is constant along q-), only in products
  // with constant vectors: (E a) . v = a . (E^T v), E^T v formed once per joint
  const MapE<Real> Ep(wp, h), Ec(wc, h);
  const vec3<Real> epa = Ep.T_(wpa), eca = Ec.T_(wca);
  joint_rows_each<D>(sc, j, pp, rotp, pc, rotc, [&](int k, vec3<D> lp, vec3<D> ap, vec3<D> lc, vec3<D> ac, D c) {
    const D Jw = dotm(lp, wpl) + dotm(ap, epa) + dotm(lc, wcl) + dotm(ac, eca);
    acc = acc + D(wl[i0 + k]) * c / D(hR) - D(hR * w.lk[i0 + k]) * Jw;
  });
  const int is = servo_row(sc, w, j);
  if (is >= 0) {
    SRow<D> sr;
    servo_row_geom<D>(sc, j, pp, rotp, pc, rotc, sr);
    const vec3<Real> epw = Ep.T_(wp), ecw = Ec.T_(wc);
    const D sv = dotm(sr.lin_p, v3(w.uk[6 * bp], w.uk[6 * bp + 1], w.uk[6 * bp + 2])) + dotm(sr.ang_p, epw) +
                 dotm(sr.lin_c, v3(w.uk[6 * bc], w.uk[6 * bc + 1], w.uk[6 * bc + 2])) + dotm(sr.ang_c, ecw);
    const D Jw = dotm(sr.lin_p, wpl) + dotm(sr.ang_p, epa) + dotm(sr.lin_c, wcl) + dotm(sr.ang_c, eca);
    acc = acc + D(wl[is]) * sv - D(hR * w.lk[is]) * Jw;
    // a position target's bias (x(q-) - target)/h holds q- directly
    if (sc.smode[j] == SERVO_POSITION) acc = acc + D(wl[is]) * joint_coord_qm<D>(sc, j, qmp, qmc) / D(hR);
  }
  return acc.d;
}

// ---------------------------------------------------------------------------
// exact mode: local Jacobians at the returned iterate
// ---------------------------------------------------------------------------
// Task (body b2, velocity component c): every group touching b2 is evaluated with u+ of
// b2 perturbed along c.  The task writes column c of body b2 in G (the rows' exact
// derivatives) and in every K block (b, b2): each (row, column) entry belongs to one task.
template <class Real>
__device__ void exact_task(const DevScene& sc, const WS<Real>& w, const ExWS<Real>& ex, const int* bgl,
                           const int* bgn, int b2, int c, double h) {
  typedef dual<Real> D;
  const Real hR = Real(h);
  const int nb = sc.nb;
  for (int b = 0; b < nb; ++b)
    for (int r = 0; r < 6; ++r) ex.K[(b * nb + b2) * 36 + r * 6 + c] = Real(0);
  for (int k = 0; k < bgn[b2]; ++k) {
    const int grp = bgl[b2 * GROUPS_PER_BODY + k];
    if (grp < sc.n_slots) {
      const int sl = grp, i = w.srow[sl];
      D qm[7], u[6];
      for (int q = 0; q < 7; ++q) qm[q] = D(w.qm[7 * b2 + q]);
      for (int q = 0; q < 6; ++q) u[q] = D(w.uk[6 * b2 + q], q == c ? Real(1) : Real(0));
      CGroup<D> g;
      contact_group<D, Real>(sc, w, sl, b2, qm, u, h, g);
      D rf[2];
      friction_rows<D, Real>(sc, g.vel[1], g.vel[2], D(w.lk[i]), w.lk[i + 1], w.lk[i + 2], hR * w.swhat[sl],
                             D(Real(sc.mu)), rf);
      ex.G[12 * i + c] = ex.fsc[sl] * g.cn.d / hR;
      ex.G[12 * (i + 1) + c] = rf[0].d;
      ex.G[12 * (i + 2) + c] = rf[1].d;
      for (int q = 0; q < 3; ++q) {
        const Real s = -hR * w.lk[i + q];
        Real* Kc = ex.K + (b2 * nb + b2) * 36 + c;
        const vec3<D>& dr = g.dir[q];
        const vec3<D>& an = g.ang[q];
        Kc[0] += s * dr.x.d; Kc[6] += s * dr.y.d; Kc[12] += s * dr.z.d;
        Kc[18] += s * an.x.d; Kc[24] += s * an.y.d; Kc[30] += s * an.z.d;
      }
    } else {
      const int j = grp - sc.n_slots, bp = sc.jp[j], bc = sc.jc[j];
      D qmp[7], qmc[7], up[6], uc[6];
      for (int q = 0; q < 7; ++q) { qmp[q] = D(w.qm[7 * bp + q]); qmc[q] = D(w.qm[7 * bc + q]); }
      for (int q = 0; q < 6; ++q) {
        up[q] = D(w.uk[6 * bp + q], (bp == b2 && q == c) ? Real(1) : Real(0));
        uc[q] = D(w.uk[6 * bc + q], (bc == b2 && q == c) ? Real(1) : Real(0));
      }
      JGroup<D> g;
      joint_group<D>(sc, j, qmp, up, qmc, uc, h, g);
      const int i0 = w.ints[1] + 5 * j;
      const int side = bp == b2 ? 0 : 6;
      Real* Kp = ex.K + (bp * nb + b2) * 36 + c;
      Real* Kch = ex.K + (bc * nb + b2) * 36 + c;
      for (int k = 0; k < 5; ++k) {
        ex.G[12 * (i0 + k) + side + c] = g.c[k].d / hR;
        const Real s = -hR * w.lk[i0 + k];
        Kp[0] += s * g.lin_p[k].x.d; Kp[6] += s * g.lin_p[k].y.d; Kp[12] += s * g.lin_p[k].z.d;
        Kp[18] += s * g.ang_p[k].x.d; Kp[24] += s * g.ang_p[k].y.d; Kp[30] += s * g.ang_p[k].z.d;
        Kch[0] += s * g.lin_c[k].x.d; Kch[6] += s * g.lin_c[k].y.d; Kch[12] += s * g.lin_c[k].z.d;
        Kch[18] += s * g.ang_c[k].x.d; Kch[24] += s * g.ang_c[k].y.d; Kch[30] += s * g.ang_c[k].z.d;
      }
      const int is = servo_row(sc, w, j);
      if (is >= 0) {
        ex.G[12 * is + side + c] = g.sv.d;
        const Real s = -hR * w.lk[is];
        Kp[0] += s * g.sl_p.x.d; Kp[6] += s * g.sl_p.y.d; Kp[12] += s * g.sl_p.z.d;
        Kp[18] += s * g.sa_p.x.d; Kp[24] += s * g.sa_p.y.d; Kp[30] += s * g.sa_p.z.d;
        Kch[0] += s * g.sl_c.x.d; Kch[6] += s * g.sl_c.y.d; Kch[12] += s * g.sl_c.z.d;
        Kch[18] += s * g.sa_c.x.d; Kch[24] += s * g.sa_c.y.d; Kch[30] += s * g.sa_c.z.d;
      }
    }
  }
}

// Per active slot: the normal row's derivative scale fa / max(fa, 1e-12) and the friction
// rows' derivatives along lambda_n (through W), at the returned iterate.
template <class Real> __device__ void exact_slot_terms(const DevScene& sc, const WS<Real>& w, const ExWS<Real>& ex,
                                                       double h) {
  typedef dual<Real> D;
  const Real hR = Real(h), eps = Real(sc.eps), kap = Real(sc.kappa);
  for (int sl = threadIdx.x; sl < sc.n_slots; sl += blockDim.x) {
    if (!w.sact[sl]) continue;
    const int i = w.srow[sl], b = sc.slot_body[sl];
    Real u[6], qm[7];
    for (int q = 0; q < 6; ++q) u[q] = w.uk[6 * b + q];
    for (int q = 0; q < 7; ++q) qm[q] = w.qm[7 * b + q];
    CGroup<Real> g;
    contact_group<Real, Real>(sc, w, sl, b, qm, u, h, g);
    const Real hw = hR * w.swhat[sl], ln = w.lk[i];
    const Real a = g.cn / hR + kap * ln, bb = hw * ln;
    const Real s = ssqrt(a * a + bb * bb + eps * eps);
    const Real fa = a > Real(0) ? (bb * bb + eps * eps) / (s * (s + a)) : Real(1) - a / s;
    ex.fsc[sl] = fa / (fa > Real(1e-12) ? fa : Real(1e-12));
    D rf[2];
    friction_rows<D, Real>(sc, D(g.vel[1]), D(g.vel[2]), D(ln, Real(1)), w.lk[i + 1], w.lk[i + 2], hw,
                           D(Real(sc.mu)), rf);
    ex.cfn[2 * sl] = rf[0].d;
    ex.cfn[2 * sl + 1] = rf[1].d;
  }
}

// ---------------------------------------------------------------------------
// exact mode: products with J_F^T and with the preconditioner
// ---------------------------------------------------------------------------
// out = J_F^T v for v = [v_u (6 nb); v_lambda (m)], sigma-weighted lambda block:
//   out_u = (M + K)^T v_u + G^T v_lambda
//   out_l = sigma (-h J v_u + C_x^T v_lambda)
// with C_x the exact lambda-derivatives of the rows (the paper's diagonal and radial
// friction blocks plus, per contact, the friction rows' lambda_n column).  Compensated
// sums: the two terms of out_l nearly cancel at the solution.
template <class Real>
__device__ void exact_apply(const DevScene& sc, const WS<Real>& w, const ExWS<Real>& ex, const Real* v, Real* out,
                            double h, Real sigma) {
  const int tid = threadIdx.x, nth = blockDim.x, nb = sc.nb, m = w.ints[0];
  const Real hR = Real(h);
  const Real* vu = v;
  const Real* vl = v + 6 * nb;
  const int ssd = sc.ss > 0 ? sc.ss : 1;
  for (int task = tid; task < 6 * nb; task += nth) {
    const int b = task / 6, k = task - 6 * b;
    acc2<Real> a;
    // M^T v_u (M symmetric: mass and world inertia at q-)
    if (k < 3) a.add_prod(Real(sc.mass[b]), vu[6 * b + k]);
    else for (int q = 0; q < 3; ++q) a.add_prod(w.Iw[9 * b + 3 * (k - 3) + q], vu[6 * b + 3 + q]);
    // K^T v_u: column (b, k) of K over all row blocks
    for (int bb = 0; bb < nb; ++bb)
      for (int r = 0; r < 6; ++r) a.add_prod(ex.K[(bb * nb + b) * 36 + r * 6 + k], vu[6 * bb + r]);
    // G^T v_lambda over the rows touching body b
    const int g = w.bgrp[b];
    if (g >= 0)
      for (int i = w.g0[g]; i < w.g0[g] + w.gn[g]; ++i) a.add_prod(ex.G[12 * i + k], vl[i]);
    for (int t = 0; t < w.bsepn[b]; ++t) {
      const int i = w.bsep[b * ssd + t];
      const int side = w.meta[4 * i + 1] == b ? 0 : 6;
      a.add_prod(ex.G[12 * i + side + k], vl[i]);
    }
    out[task] = a.value();
  }
  for (int i = tid; i < m; i += nth) {
    const Real* Ji = w.J + 12 * i;
    const int b0 = w.meta[4 * i + 1], b1 = w.meta[4 * i + 2];
    acc2<Real> a;
    for (int q = 0; q < 6; ++q) a.add_prod(-hR * Ji[q], vu[6 * b0 + q]);
    if (b1 >= 0) for (int q = 0; q < 6; ++q) a.add_prod(-hR * Ji[6 + q], vu[6 * b1 + q]);
    const int t = w.meta[4 * i] & 15, sub = w.meta[4 * i] >> 4;
    // normal rows: d(phi/scl)/dlambda_n = (fa kappa + fb h what)/scl; evaluate() keeps
    // kappa + fb h what/scl, equal unless the scale is clamped (fa < 1e-12)
    const Real cii = t == ROW_NORMAL ? w.C[i] + (ex.fsc[w.ref[i]] - Real(1)) * Real(sc.kappa) : w.C[i];
    a.add_prod(cii, vl[i]);
    if (t == ROW_FRIC) {
      const Real* rd = w.srad + 3 * w.ref[i];
      if (sub == 1) a.add_prod(rd[1], vl[i + 1]);
      else a.add_prod(rd[1], vl[i - 1]);
      a.add_prod(sub == 1 ? rd[0] : rd[2], vl[i]);
    } else if (t == ROW_NORMAL) {
      // column lambda_n of the two friction rows, transposed
      const int sl = w.ref[i];
      a.add_prod(ex.cfn[2 * sl], vl[i + 1]);
      a.add_prod(ex.cfn[2 * sl + 1], vl[i + 2]);
    }
    out[6 * nb + i] = sigma * a.value();
  }
}

// z = P^-T v with P the paper's Newton matrix [[M, -h J^T], [J, C + delta]] (radial
// friction blocks in C), through the taped factor of A = h J M^-1 J^T + C + delta:
//   z_lambda = A^-1 (v_lambda / sigma + h J M^-1 v_u),  z_u = M^-1 (v_u - J^T z_lambda).
// z may not alias v.  Uses w.mr, w.rhs and ex.t6 as scratch.
template <class Real>
__device__ void exact_precond(const DevScene& sc, WS<Real>& w, const ExWS<Real>& ex, const Real* v, Real* z, double h,
                              Real sigma) {
  const int tid = threadIdx.x, nth = blockDim.x, nb = sc.nb, m = w.ints[0];
  const Real hR = Real(h);
  for (int b = tid; b < nb; b += nth) minv6(sc, w, b, v + 6 * b, w.mr + 6 * b);
  __syncthreads();
  for (int i = tid; i < m; i += nth) {
    const Real* Ji = w.J + 12 * i;
    const int b0 = w.meta[4 * i + 1], b1 = w.meta[4 * i + 2];
    acc2<Real> a;
    for (int q = 0; q < 6; ++q) a.add_prod(hR * Ji[q], w.mr[6 * b0 + q]);
    if (b1 >= 0) for (int q = 0; q < 6; ++q) a.add_prod(hR * Ji[6 + q], w.mr[6 * b1 + q]);
    a.add(v[6 * nb + i] / sigma);
    z[6 * nb + i] = a.value();
  }
  __syncthreads();
  arrow_solve(sc, w, z + 6 * nb);
  jt_apply_acc(sc, w, z + 6 * nb, ex.t6);
  __syncthreads();
  for (int b = tid; b < nb; b += nth) {
    Real t[6];
    for (int q = 0; q < 6; ++q) t[q] = v[6 * b + q] - ex.t6[6 * b + q];
    minv6(sc, w, b, t, z + 6 * b);
  }
  __syncthreads();
}

// Several dot products of one vector with the rows of V at once, deterministic block
// reduction: out[i] = sum_e a[e] V[i][e] for i < cnt (cnt <= KRYLOV + 1).
template <class Real>
__device__ void multi_dot(const ExWS<Real>& ex, const Real* a, const Real* V, int ldv, int cnt, int n, Real* out) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  for (int i = 0; i < cnt; ++i) {
    Real p = Real(0);
    for (int e = tid; e < n; e += blockDim.x) p += a[e] * V[i * ldv + e];
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) ex.wred[wid * (KRYLOV + 2) + i] = p;
  }
  __syncthreads();
  for (int i = tid; i < cnt; i += blockDim.x) {
    Real s = Real(0);
    for (int q = 0; q < nw; ++q) s += ex.wred[q * (KRYLOV + 2) + i];
    out[i] = s;
  }
  __syncthreads();
}

// Euclidean norm of a length-n vector (every thread gets it).
template <class Real> __device__ Real block_norm(const ExWS<Real>& ex, const Real* a, int n) {
  multi_dot(ex, a, a, n, 1, n, ex.scal);
  const Real v = ssqrt(ex.scal[0]);
  __syncthreads();
  return v;
}

// GMRES(KRYLOV) with restarts for J_F^T w = b (b = [-g; 0] in ex.r on entry), right-
// preconditioned by P^-T; the solution is returned in ex.x.  Starts from the paper
// mode's solution P^-T b.  Returns the Krylov iterations run; *conv_out says whether the
// weighted residual fell below rel_tol times that of the starting point's right-hand side.
template <class Real>
__device__ int exact_gmres(const DevScene& sc, WS<Real>& w, const ExWS<Real>& ex, double h, Real sigma, Real rel_tol,
                           int* conv_out) {
  const int tid = threadIdx.x, nth = blockDim.x, n = 6 * sc.nb + w.ints[0];
  Real* V = ex.V;
  Real* bsave = ex.V + KRYLOV * n;      // row KRYLOV of V keeps b (Arnoldi fills rows 0..KRYLOV-1)
  for (int e = tid; e < n; e += nth) bsave[e] = ex.r[e];
  __syncthreads();
  exact_precond(sc, w, ex, bsave, ex.x, h, sigma);           // x0 = P^-T b, the paper mode's solution
  const Real bn = block_norm(ex, bsave, n);
  int total = 0, conv = 0;
  if (!(bn > Real(0))) { *conv_out = 1; return 0; }
  const Real stop = rel_tol * bn;
  for (int cycle = 0; cycle < KRYLOV_CYCLES && !conv; ++cycle) {
    exact_apply(sc, w, ex, ex.x, ex.z, h, sigma);             // r = b - A x
    __syncthreads();
    for (int e = tid; e < n; e += nth) ex.r[e] = bsave[e] - ex.z[e];
    __syncthreads();
    const Real beta = block_norm(ex, ex.r, n);
    if (!(beta > stop)) { conv = 1; break; }
    for (int e = tid; e < n; e += nth) V[e] = ex.r[e] / beta;
    if (tid == 0) { ex.gg[0] = beta; for (int i = 1; i <= KRYLOV; ++i) ex.gg[i] = Real(0); }
    __syncthreads();
    int k = 0;
    for (;;) {
      exact_precond(sc, w, ex, V + k * n, ex.z, h, sigma);    // z = P^-T v_k
      exact_apply(sc, w, ex, ex.z, ex.r, h, sigma);           // r = A z
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {                  // classical Gram-Schmidt, twice
        multi_dot(ex, ex.r, V, n, k + 1, n, ex.y);
        for (int e = tid; e < n; e += nth) {
          Real s = ex.r[e];
          for (int i = 0; i <= k; ++i) s -= ex.y[i] * V[i * n + e];
          ex.r[e] = s;
        }
        if (tid == 0)
          for (int i = 0; i <= k; ++i) ex.Hh[i * KRYLOV + k] = (pass ? ex.Hh[i * KRYLOV + k] : Real(0)) + ex.y[i];
        __syncthreads();
      }
      const Real hn = block_norm(ex, ex.r, n);
      const bool last = k + 1 >= KRYLOV;
      if (!last && hn > Real(0))
        for (int e = tid; e < n; e += nth) V[(k + 1) * n + e] = ex.r[e] / hn;
      if (tid == 0) {
        for (int i = 0; i < k; ++i) {                         // previous Givens rotations
          const Real a = ex.Hh[i * KRYLOV + k], b = ex.Hh[(i + 1) * KRYLOV + k];
          ex.Hh[i * KRYLOV + k] = ex.cs[i] * a + ex.sn[i] * b;
          ex.Hh[(i + 1) * KRYLOV + k] = -ex.sn[i] * a + ex.cs[i] * b;
        }
        const Real a = ex.Hh[k * KRYLOV + k], b = hn;
        const Real rr = ssqrt(a * a + b * b);
        const Real c = rr > Real(0) ? a / rr : Real(1), s = rr > Real(0) ? b / rr : Real(0);
        ex.cs[k] = c; ex.sn[k] = s;
        ex.Hh[k * KRYLOV + k] = rr;
        const Real gk = ex.gg[k];
        ex.gg[k] = c * gk;
        ex.gg[k + 1] = -s * gk;
        w.ints[8] = (fabs((double)ex.gg[k + 1]) <= (double)stop || !(hn > Real(0)) || last) ? 1 : 0;
      }
      __syncthreads();
      ++total;
      ++k;
      if (w.ints[8]) break;
    }
    if (tid == 0) {                                           // y = H^-1 g, k x k upper triangular
      for (int i = k - 1; i >= 0; --i) {
        Real s = ex.gg[i];
        for (int q = i + 1; q < k; ++q) s -= ex.Hh[i * KRYLOV + q] * ex.y[q];
        const Real d = ex.Hh[i * KRYLOV + i];
        ex.y[i] = d != Real(0) ? s / d : Real(0);
      }
      w.ints[9] = fabs((double)ex.gg[k]) <= (double)stop ? 1 : 0;
    }
    __syncthreads();
    for (int e = tid; e < n; e += nth) {                      // x += P^-T (V y)
      Real s = Real(0);
      for (int i = 0; i < k; ++i) s += ex.y[i] * V[i * n + e];
      ex.r[e] = s;
    }
    __syncthreads();
    exact_precond(sc, w, ex, ex.r, ex.z, h, sigma);
    for (int e = tid; e < n; e += nth) ex.x[e] += ex.z[e];
    __syncthreads();
    conv = w.ints[9];
  }
  *conv_out = conv;
  return total;
}

}  // namespace ost
