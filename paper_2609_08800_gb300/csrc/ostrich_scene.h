// Device-side scene description and shared-memory layout of the Ostrich step kernels.
// Product code only (the CPU oracle has its own, independent format).
#pragma once
#include <stdint.h>

namespace ost {

constexpr int NB_CAP = 8;      // bodies per world
constexpr int NJ_CAP = 8;      // revolute joints per world
constexpr int SLOT_CAP = 64;   // contact slots per world
constexpr int SEP_CAP = 5 * NJ_CAP + NJ_CAP;   // separator rows per world

enum { SHAPE_NONE = 0, SHAPE_BOX = 1, SHAPE_WHEEL = 2 };
enum { ENV_PLANE = 0, ENV_BOX = 1, ENV_HEIGHTMAP = 2 };
enum { ROW_JOINT = 0, ROW_SERVO = 1, ROW_NORMAL = 2, ROW_FRIC = 3 };
enum { JOINT_REVOLUTE = 0, JOINT_PRISMATIC = 1 };
enum { SERVO_VELOCITY = 0, SERVO_POSITION = 1 };
enum { LIN_DIRECT = 0, LIN_PCR = 1 };     // Schur solve: block-arrowhead factor / PCR
enum { PC_JACOBI = 0, PC_BLOCK = 1 };     // PCR preconditioner

// Everything a kernel needs to know about the scene and the solver settings.
// Passed by value as a kernel parameter.
struct DevScene {
  int nb, nj, n_servo, n_slots, m_max, n_state, env, nf;
  double mu, g;
  double box[5];                 // x0, x1, y0, y1, H
  int hn; double hsp, hox, hoy;  // heightmap grid
  const float* heights;          // device pointer, hn*hn, or null
  // bodies
  double mass[NB_CAP], inertia[NB_CAP][3], half[NB_CAP][3], radius[NB_CAP], hw[NB_CAP];
  int shape[NB_CAP], slot_base[NB_CAP], slot_count[NB_CAP];
  unsigned char slot_body[SLOT_CAP];
  // joints
  int jp[NJ_CAP], jc[NJ_CAP], servo_of[NJ_CAP];
  double ap[NJ_CAP][3], ac[NJ_CAP][3], axp[NJ_CAP][3], axc[NJ_CAP][3], p1[NJ_CAP][3], p2[NJ_CAP][3], kp[NJ_CAP];
  double kd[NJ_CAP];
  int jtype[NJ_CAP];   // JOINT_REVOLUTE / JOINT_PRISMATIC
  int smode[NJ_CAP];   // SERVO_VELOCITY / SERVO_POSITION
  // solver settings
  int budget, kmin, ls, pullback;
  double tol, delta_rel, kappa, eps, margin;
  int refine;     // iterative-refinement sweeps after each forward (Newton-step) Schur solve
  int refine_adj; // iterative-refinement sweeps after the adjoint's Schur solve
  // linear solver of Eq. (12): LIN_DIRECT, or LIN_PCR (matrix-free preconditioned conjugate
  // residual with preconditioner pc; pcr_iters iterations per Newton step; the adjoint's
  // solve stops at |r| <= pcr_rtol_adj |b| or after pcr_iters_adj iterations)
  int lin, pc, pcr_iters, pcr_iters_adj;
  double pcr_rtol_adj;
  // layout caps derived from the scene
  int n_groups;   // bodies that carry contact slots (leaf blocks of the Schur matrix)
  int pg;         // largest leaf block (3 x slots of one body)
  int ss;         // separator rows (5 per joint + servos)
  int group_body[NB_CAP];
  // static coupling between groups and separator rows (the separator rows are always
  // present): group g couples to separator rows cpl_row[g][0 .. cpl_n[g]); separator row
  // a belongs to the lists of sep_n[a] <= 2 groups, at (sep_g[a][i], sep_k[a][i])
  int ldg, lds, cmax;                    // odd row lengths of the coupling blocks (ldg); cmax coupling rows
  int cpl_n[NB_CAP];
  unsigned char cpl_row[NB_CAP][SEP_CAP];
  unsigned char sep_n[SEP_CAP], sep_g[SEP_CAP][2], sep_k[SEP_CAP][2];
};

// Packed lower-triangular storage of the symmetric Schur blocks and their inverse
// factors: element (i, j), j <= i, of an n x n block sits at tri(i, j); a block takes
// tri_size(n) entries and its row i is contiguous.
__host__ __device__ inline int tri(int i, int j) { return ((i * (i + 1)) >> 1) + j; }
__host__ __device__ inline int tri_size(int n) { return (n * (n + 1)) >> 1; }

// Derived layout of a filled scene: groups, block sizes, the static coupling lists.
inline void finish_scene(DevScene& s) {
  s.n_groups = 0; s.pg = 0;
  for (int b = 0; b < s.nb; ++b)
    if (s.slot_count[b] > 0) {
      s.group_body[s.n_groups++] = b;
      if (3 * s.slot_count[b] > s.pg) s.pg = 3 * s.slot_count[b];
    }
  s.ss = 5 * s.nj + s.n_servo;
  s.ldg = s.pg | 1;
  s.lds = s.ss | 1;
  int gof[NB_CAP];
  for (int b = 0; b < NB_CAP; ++b) gof[b] = -1;
  for (int g = 0; g < s.n_groups; ++g) { gof[s.group_body[g]] = g; s.cpl_n[g] = 0; }
  for (int a = 0; a < s.ss; ++a) {
    int j = a < 5 * s.nj ? a / 5 : -1;
    if (j < 0) {                          // servo row: find its joint
      int k = a - 5 * s.nj, cnt = -1;
      for (j = 0; j < s.nj; ++j) if (s.servo_of[j] >= 0 && ++cnt == k) break;
    }
    s.sep_n[a] = 0;
    int bodies[2] = {s.jp[j], s.jc[j]};
    for (int t = 0; t < 2; ++t) {
      int g = gof[bodies[t]];
      if (g < 0) continue;
      int k = s.cpl_n[g]++;
      s.cpl_row[g][k] = (unsigned char)a;
      s.sep_g[a][s.sep_n[a]] = (unsigned char)g;
      s.sep_k[a][s.sep_n[a]] = (unsigned char)k;
      s.sep_n[a]++;
    }
  }
  s.cmax = 0;
  for (int g = 0; g < s.n_groups; ++g) if (s.cpl_n[g] > s.cmax) s.cmax = s.cpl_n[g];
}



// Arguments of one launch of the step / adjoint kernels.
// World selection: without a list, CTA b steps world world0 + b and records into the
// tape slot that `tape` points at.  With a list (device arrays of gridDim entries), CTA
// b steps world list[b] and records into slot list_slot[b] of the tape that starts at
// `tape` (slot stride n_worlds records; -1: no record); out-of-range entries are skipped.
// The list form launches n_list CTAs.
struct StepArgs {
  const void* state_in; const void* controls; void* state_out; void* impulses;
  int32_t* ids; uint32_t* status; int32_t* iters; void* tape;
  int ld, n_worlds, world0; double h;
  double* trace = nullptr;   // optional diagnostic: merit of each iterate, (budget + 2) per world
  const int32_t* list = nullptr; const int32_t* list_slot = nullptr; int n_list = 0, tape_slots = 0;
  // persistent schedule (queue != nullptr): gridDim CTAs take the work items 0 .. n_items-1
  // from the counter *queue (zero at launch) in the order order[] (or 0, 1, ...); each
  // world's Newton iteration count goes to cost[] for the next step's order
  int* queue = nullptr; const int32_t* order = nullptr; int32_t* cost = nullptr; int n_items = 0;
};
struct AdjArgs {
  const void* tape; const void* dL_dnext; void* dL_dstate; void* dL_dcontrols;
  int ld, n_worlds, world0; double h;
  const int32_t* list = nullptr; const int32_t* list_slot = nullptr; int n_list = 0, tape_slots = 0;
  // optional physical-parameter gradients: dL/dk_p per servo (n_servo x ld), dL/dm per
  // body (nb x ld), dL/dI per body-frame principal moment (3 nb x ld), or null
  void* dL_dkp = nullptr; void* dL_dmass = nullptr; void* dL_dinertia = nullptr;
  void* dL_dmu = nullptr;       // optional: dL/dmu per world (n_worlds entries)
  int mode = 0;                 // 0: the paper's adjoint (frozen W), 1: exact IFT
  int32_t* krylov = nullptr;    // optional: per world Krylov iterations (GMRES, or the PCR solve) | 1 << 16 if not converged
};

// Tape record of one world for one step: inputs, the contact slot table the step's
// activation produced, returned iterate and the Schur factor (block-arrowhead, in inverse
// form).  All counts in Real elements.
struct TapeLayout {
  int off_qm, off_um, off_ubar, off_ct, off_u, off_lam, off_G, off_H, off_S, total;
};
constexpr int CT_PER_SLOT = 9;   // active, id, feature type (bit-exact), normal (3), offset, edge (2)

inline __host__ __device__ TapeLayout tape_layout(const DevScene& s) {
  TapeLayout t;
  int o = 0;
  t.off_qm = o; o += 7 * s.nb;
  t.off_um = o; o += 6 * s.nb;
  t.off_ubar = o; o += s.n_servo > 0 ? s.n_servo : 1;
  t.off_ct = o; o += CT_PER_SLOT * s.n_slots;        // the step's contact slot table
  t.off_u = o; o += 6 * s.nb;
  t.off_lam = o; o += s.m_max;
  t.off_G = o; o += s.n_groups * tri_size(s.pg);    // inverse Cholesky factors L_g^-1 of the groups (packed)
  t.off_H = o; o += s.n_groups * s.cmax * s.ldg;     // F_g = E_g L_g^-T (coupled separator rows)
  t.off_S = o; o += tri_size(s.ss);                  // inverse Cholesky factor of the reduced separator (packed)
  o = (o + 3) & ~3;   // 16-byte multiple per world for FP32
  t.total = o;
  return t;
}

}  // namespace ost
