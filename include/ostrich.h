/*
 * ostrich.h -- C ABI of libostrich: the per-timestep non-smooth Newton solve of
 * many independent rigid-body worlds and its implicit-function-theorem adjoint,
 * for NVIDIA GB300 (sm_103a).
 *
 * The problem follows the paper's statement (Sec. III-C, III-D): one step is the
 * implicit map s+ = s+(s-, a) defined by the stacked residual r(s+, s-, a) = 0 of
 * Eqs. (9)-(11) (backward-Euler kinematics Eq. (1), implicit dynamics Eq. (2),
 * joint rows Eq. (3), Fischer-Burmeister normal contact Eq. (4), friction Eq. (7),
 * implicit velocity or position servos Eq. (8)); the adjoint maps dL/ds+ to dL/ds- and dL/da
 * through Eqs. (16)-(19) with the Schur factor of the forward step.
 *
 * Layout.  Every state, control, impulse and gradient array is a device pointer
 * owned by the caller, structure of arrays with the world index fastest: component
 * c of world w sits at ptr[c * ld + w], ld >= n_worlds (ld is fixed at create).
 *   state   = [q: 7 per body (p, quaternion w x y z)] [u: 6 per body (v, w_world)]
 *             [lambda: 5 per joint, 1 per servo, 3 per contact slot]        (n_state)
 *   controls: one target per servo: joint rate (rad/s, m/s) or joint position
 *             (rad, m) by the servo's mode                                   (n_servo)
 *   impulses: h * lambda in the lambda layout, zero on inactive rows          (m_max)
 *   contact ids: per slot (body << 24 | rim_or_corner << 20 | feature), -1 if inactive
 * Element type is float for OSTRICH_F32 contexts and double for OSTRICH_F64.
 *
 * Errors.  Functions return an ostrich_status and never abort or print; the text of
 * the last error of a context is available from ostrich_last_error.  Work is queued
 * asynchronously on the given stream; per-world outcome bits are written to
 * world_status (1: not converged, best iterate returned; 2: non-finite; 4: contact
 * overflow).  Calls on one context must not overlap on the device when they use the
 * same tape slot.
 */
#ifndef OSTRICH_H
#define OSTRICH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ostrich_ctx ostrich_ctx;

typedef enum {
  OSTRICH_OK = 0,
  OSTRICH_EINVAL = 1,   /* bad argument, size or layout */
  OSTRICH_ENOMEM = 2,   /* device allocation failed */
  OSTRICH_ECUDA = 3,    /* a CUDA call failed (see ostrich_last_error) */
  OSTRICH_ETAPE = 4     /* adjoint on a tape slot that holds no recorded step */
} ostrich_status;

enum { OSTRICH_F32 = 0, OSTRICH_F64 = 1 };
enum { OSTRICH_ENV_PLANE = 0, OSTRICH_ENV_BOX = 1, OSTRICH_ENV_HEIGHTMAP = 2 };
enum { OSTRICH_SHAPE_NONE = 0, OSTRICH_SHAPE_BOX = 1, OSTRICH_SHAPE_WHEEL = 2 };
enum { OSTRICH_PULLBACK_FULL = 0, OSTRICH_PULLBACK_TRUNCATED = 1 };
enum { OSTRICH_ADJ_PAPER = 0, OSTRICH_ADJ_EXACT = 1 };
/* Linear solver of the Schur system Eq. (12) (ostrich_set_linear_solver) and the PCR
 * preconditioner. */
enum { OSTRICH_LIN_DIRECT = 0, OSTRICH_LIN_PCR = 1 };
enum { OSTRICH_PC_JACOBI = 0, OSTRICH_PC_BLOCK = 1 };

#define OSTRICH_MAX_BODIES 8
#define OSTRICH_MAX_JOINTS 8

/* Rigid body: mass, principal inertia (body frame), collision shape (box corners
 * or a wheel cylinder whose axle is the body y axis). */
typedef struct {
  double mass, inertia[3];
  int shape;
  double half_extents[3];
  double radius, half_width;
} ostrich_body_desc;

/* Joint between two bodies (Eq. (3), five rows, no compliance).  type
 * OSTRICH_JOINT_REVOLUTE: 3 anchor rows + 2 axis-alignment rows (perp1/perp2_parent
 * against axis_child); OSTRICH_JOINT_PRISMATIC: the child anchor held on the parent's
 * axis line (2 rows along perp1/perp2_parent), 2 axis-alignment rows and a twist lock
 * (perp2_parent against the child's perp1, the same coordinates in the child frame).
 * kp > 0 adds a servo row on the joint coordinate (Eq. (8)): servo_mode
 * OSTRICH_SERVO_VELOCITY tracks a target rate (compliance 1/kp); OSTRICH_SERVO_POSITION
 * tracks a target angle / slide (compliance 1/(kd + h kp), bias (x(q-) - target)/h, x the
 * angle about axis_parent from perp1_parent to the child's perp1, or the slide
 * axis . (child anchor - parent anchor)).  Zero-initialised fields give a revolute
 * joint with a velocity servo. */
enum { OSTRICH_JOINT_REVOLUTE = 0, OSTRICH_JOINT_PRISMATIC = 1 };
enum { OSTRICH_SERVO_VELOCITY = 0, OSTRICH_SERVO_POSITION = 1 };
typedef struct {
  int parent, child;
  double anchor_parent[3], anchor_child[3];
  double axis_parent[3], axis_child[3];
  double perp1_parent[3], perp2_parent[3];
  double kp;
  int type, servo_mode;
  double kd;
} ostrich_joint_desc;

/* Scene shared by all worlds of a context.  heights: host pointer to hm_n*hm_n
 * FP32 heights (copied at create), or NULL. */
typedef struct {
  int n_bodies, n_joints, env;
  double mu, gravity;
  double box[5];                 /* obstacle x0, x1, y0, y1, height */
  int hm_n;
  double hm_spacing, hm_origin[2];
  const float* heights;
  ostrich_body_desc bodies[OSTRICH_MAX_BODIES];
  ostrich_joint_desc joints[OSTRICH_MAX_JOINTS];
} ostrich_scene_desc;

/* Solver settings: Newton budget and best-iterate floor (Sec. III-C), stopping
 * tolerance on sqrt(merit) in m/s, step damping relative to mean diag(h J M^-1 J^T),
 * contact compliance kappa (s/kg), FB smoothing eps (Sec. III-D), activation margin
 * (m), line search (0: full steps, 1: backtracking), position pull-back mode. */
typedef struct {
  int budget, k_min, line_search, pullback;
  double tol, delta_rel, kappa, eps_fb, margin;
} ostrich_solver_cfg;

/* Create a context for n_worlds worlds (arrays strided by ld >= n_worlds), with
 * tape_slots recorded steps of device workspace (library-owned, freed by destroy).
 * EINVAL on sizes beyond the caps, ENOMEM if the tape cannot be allocated. */
ostrich_status ostrich_create(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg, int n_worlds, int ld,
                              int dtype, int tape_slots, ostrich_ctx** out);

/* Layout sizes: out[0] n_state, out[1] m_max, out[2] n_slots, out[3] n_servo. */
ostrich_status ostrich_layout(const ostrich_ctx* ctx, int32_t out[4]);

/* Threads per world (32, 64 or 128) used by both kernels; the autotuner's knob. */
ostrich_status ostrich_set_threads(ostrich_ctx* ctx, int threads);

/* Launch schedule of ostrich_step (an autotuner knob; results do not depend on it):
 * 0 one CTA per world (default); 1 persistent: as many CTAs as fit on the device take
 * worlds from a device work counter, heaviest first by each world's Newton iterations in
 * the previous step (a one-CTA counting sort launched before the step).  The list form
 * always uses one CTA per entry.  ENOMEM if the context's small schedule buffers cannot
 * be allocated. */
ostrich_status ostrich_set_schedule(ostrich_ctx* ctx, int schedule);

/* One forward step of every world (Sec. III-C): state_in -> state_out, with
 * h the time step.  impulses_out, contact_ids_out, world_status and iters_out
 * (per world: Newton iterations | active rows << 16) may be NULL.  tape_slot >= 0
 * records what the adjoint needs in that slot; -1 records nothing.  state_in and
 * state_out may not alias. */
ostrich_status ostrich_step(ostrich_ctx* ctx, const void* state_in, const void* controls, double h, void* state_out,
                            void* impulses_out, int32_t* contact_ids_out, uint32_t* world_status, int32_t* iters_out,
                            int tape_slot, void* stream);

/* Adjoint of the step recorded in tape_slot (Sec. III-D): dL/dstate_next (state
 * layout; lambda entries ignored) -> dL/dstate (lambda entries zero) and
 * dL/dcontrols (may be NULL).  The slot holds the step's inputs, its contact set (the
 * adjoint uses the same set, it does not run the activation again), the returned
 * iterate and, under the direct solver, the Schur factor at that iterate.  h must equal
 * the recorded step's.  ETAPE if the slot holds no step. */
ostrich_status ostrich_adjoint(ostrich_ctx* ctx, int tape_slot, const void* dL_dstate_next, double h,
                               void* dL_dstate, void* dL_dcontrols, void* stream);

/* ostrich_adjoint plus the gradients of the physical parameters (Eq. (17) with xi =
 * theta): dL/dk_p of each servo gain (n_servo x ld, servo order as the controls), dL/dm
 * of each body mass (nb x ld), dL/dI of each body-frame principal moment (3 nb x ld,
 * body-major) and dL/dmu of the friction coefficient (one per world, n_worlds entries),
 * element type as the context's, any may be NULL.  They contract the step's adjoint
 * with the explicit partials of the rows holding the parameter: the servo row of Eq. (8)
 * (-lambda_c / k_p^2), the linear and angular rows of Eq. (10) ((v+ - v-) - h g e_z;
 * r_k (r_k . (w+ - w-)) + h (r_k . w-) (w- x r_k), r_k the k-th column of R(q-)) and the
 * friction rows of Eq. (7) through W (exact mode; the paper's frozen W holds mu, so its
 * mu gradient is 0).  The FB scaling what = J M^-1 J^T, which also holds the mass
 * properties, is a step-start constant here.  Arguments and errors otherwise as
 * ostrich_adjoint. */
ostrich_status ostrich_adjoint_params(ostrich_ctx* ctx, int tape_slot, const void* dL_dstate_next, double h,
                                      void* dL_dstate, void* dL_dcontrols, void* dL_dkp, void* dL_dmass,
                                      void* dL_dinertia, void* dL_dmu, void* stream);

/* Adjoint mode of the context's ostrich_adjoint / _params / _list calls (Sec. III-D):
 * OSTRICH_ADJ_PAPER (default) solves Eqs. (18)-(19) with the forward Schur factor at the
 * returned iterate, W and the FB scalings frozen as the paper prescribes; OSTRICH_ADJ_EXACT
 * solves the implicit-function theorem's transposed system with the full Jacobian of the
 * residual in (u+, lambda+) -- W's dependence on the slip velocities and on lambda_n
 * (Eqs. (6)-(7)), the velocity dependence of the friction and servo rows' Jacobians, and
 * the geometric stiffness d(J^T lambda)/du of Eq. (10) -- by GMRES (restart 20, at most 60
 * iterations) in the world's shared memory, right-preconditioned by the paper's matrix
 * through the taped factor; its q- pull-back is always the full one.  krylov_iters: a
 * device array of n_worlds int32 (or NULL) that receives, per world, the GMRES iterations
 * of the exact mode, with bit 16 set when the relative residual did not reach 1e-6
 * (FP32) / 1e-13 (FP64); under the PCR solver (ostrich_set_linear_solver) the paper mode
 * writes its PCR iterations there the same way.  EINVAL for an unknown mode or when the exact mode's working
 * set (about twice the paper mode's) exceeds the shared memory of one CTA. */
ostrich_status ostrich_set_adjoint_mode(ostrich_ctx* ctx, int mode, int32_t* krylov_iters);

/* Linear solver of the Schur system A dl = rhs of Eq. (12), A = h J M^-1 J^T + C + delta I,
 * in the context's steps and adjoints (Sec. III-C, III-D).
 *   OSTRICH_LIN_DIRECT (default): the block-arrowhead Cholesky factor, formed at every Newton
 *     iterate and recorded on the tape at the returned iterate for the adjoint.
 *   OSTRICH_LIN_PCR: the paper's matrix-free preconditioned conjugate residual: iters
 *     iterations per Newton step from dl = 0, each one product with A formed from the rows
 *     (never assembled) and one application of the preconditioner, precond =
 *     OSTRICH_PC_JACOBI (the inverse diagonal of A) or OSTRICH_PC_BLOCK (the inverse of each
 *     contact group's diagonal block and of the joint/servo block, by in-place Cholesky).
 *     No factor is taped; the paper-mode adjoint forms the same operator and
 *     preconditioner at the taped iterate and solves with PCR, restarted on the true
 *     residual (formed with compensated sums) until |r| <= adj_rtol |rhs|, until a restart
 *     no longer changes the solution at working precision, or after adj_iters PCR iterations
 *     in all (krylov_iters of ostrich_set_adjoint_mode, when given, receives the iterations
 *     per world, bit 16 set if neither test was met).
 *     The exact-mode adjoint forms the direct factor at the taped iterate as its GMRES
 *     preconditioner.
 * iters and adj_iters >= 1; adj_rtol >= 0 (0: 1e-10 for FP32, 1e-12 for FP64; the Schur
 * matrix's condition number, up to ~1e6 with contact compliance, turns a residual of rtol
 * into a solution error of up to cond x rtol).  Both
 * solvers reach the same solution of each step when its Newton iteration converges; PCR
 * with few iterations leaves inexact Newton steps and so needs more of them.  A change of
 * the solver discards what the tape holds (its slots read as unwritten).  EINVAL for an
 * unknown solver or preconditioner, counts below 1, or a PCR working set (7 m_max values
 * more per world) beyond the shared memory of one CTA. */
ostrich_status ostrich_set_linear_solver(ostrich_ctx* ctx, int solver, int precond, int iters, int adj_iters,
                                         double adj_rtol);

/* Step of a selected subset of worlds (Sec. III-C, per world as ostrich_step): CTA b
 * steps world worlds[b] and, when tape_slots is not NULL and tape_slots[b] >= 0,
 * records it in that slot.  worlds and tape_slots are device arrays of n_list
 * int32 entries; the worlds must be distinct.  Entries outside [0, n_worlds) and slots
 * outside [-1, tape_slots of the context) are skipped or record nothing, on the device.
 * Unlike ostrich_step, state_in may equal state_out: a world reads its own column
 * before it writes it and touches no other.  Unlisted worlds are left untouched.  The
 * slots' bookkeeping is the caller's: ostrich_adjoint_list trusts that each listed
 * slot holds that world's step taken with the same h.  This is the batching entry point
 * of a serving loop whose requests stand at different steps of their horizons. */
ostrich_status ostrich_step_list(ostrich_ctx* ctx, const void* state_in, const void* controls, double h,
                                 void* state_out, void* impulses_out, int32_t* contact_ids_out,
                                 uint32_t* world_status, int32_t* iters_out, const int32_t* worlds,
                                 const int32_t* tape_slots, int n_list, void* stream);

/* Adjoint (Sec. III-D, per world as ostrich_adjoint) of a selected subset of worlds:
 * CTA b back-propagates world worlds[b] through the step recorded in tape_slots[b].
 * dL_dstate_next may equal dL_dstate.  Entries out of range are skipped (their
 * outputs untouched).  n_list <= n_worlds; EINVAL otherwise. */
ostrich_status ostrich_adjoint_list(ostrich_ctx* ctx, const void* dL_dstate_next, double h, void* dL_dstate,
                                    void* dL_dcontrols, const int32_t* worlds, const int32_t* tape_slots, int n_list,
                                    void* stream);

/* Diagnostic: when merits is a device pointer of n_worlds * (budget + 2) doubles, the
 * following steps record the merit of the warm start and of every Newton iterate of
 * each world there; NULL switches it off. */
ostrich_status ostrich_debug_trace(ostrich_ctx* ctx, double* merits);

/* Mark every tape slot empty (checkpoint recomputation reuses slots). */
ostrich_status ostrich_tape_clear(ostrich_ctx* ctx);

/* Device bytes of one tape slot (all worlds). */
size_t ostrich_tape_bytes(const ostrich_ctx* ctx);

/* Shared-memory bytes one world's working set takes in either kernel (the dynamic
 * allocation of one CTA); with the registers it bounds the worlds resident per SM. */
size_t ostrich_workspace_bytes(const ostrich_ctx* ctx);

/* Message of the context's last failed call (a NUL-terminated string owned by the
 * context, valid until its next failing call or ostrich_destroy; "" when none failed);
 * for a NULL context a fixed message. */
const char* ostrich_last_error(const ostrich_ctx* ctx);

/* Free the context, its tape and its device buffers (cudaFree; NULL is ignored).  No
 * call may use the context afterwards, and no queued work may still read its tape. */
void ostrich_destroy(ostrich_ctx* ctx);

/* Allocation-free step + adjoint (FP32), for callers that cannot call cudaMalloc: a
 * real-time control loop that must not allocate once running (an allocation can block
 * or fail at an arbitrary moment), or a plugin whose host framework owns all device
 * memory and hands out only the buffers it manages.  The paper has no counterpart; it
 * adds no computation to ostrich_step / ostrich_adjoint.
 *
 * One forward step of n_worlds worlds (as ostrich_step, without impulses, ids or
 * status; one CTA of 64 threads per world) followed at once by the adjoint of that step
 * (as ostrich_adjoint), with the tape in a fixed library array of
 * OSTRICH_NOALLOC_SCRATCH_BYTES instead of a context.  Arrays are caller-owned device
 * pointers in the layout above (ld >= n_worlds; 0 means n_worlds).  No context is
 * needed and nothing is allocated, freed or kept.
 *
 * EINVAL if n_worlds times the scene's per-world tape record exceeds the array (the
 * record is ostrich_tape_bytes / n_worlds of an FP32 context for the same scene: 10432 B
 * for the four-wheel robot over a box, so at most 1608 worlds per call; see
 * ostrich_noalloc_capacity), for heightmap
 * scenes (env OSTRICH_ENV_HEIGHTMAP: the heights would need a device copy), or on the
 * same argument errors as ostrich_create / ostrich_step; ECUDA if a launch fails.
 * The first call on a device resolves the array's device address on that device (with
 * it current) and caches it; make that first call before any stream capture, and do not
 * use the entry point across a cudaDeviceReset (the cached address would be stale).
 * Every call on a device shares the one array and leaves its contents behind; nothing
 * in it needs clearing, as the step writes every entry the adjoint reads.  Calls that
 * overlap on the GPU (different streams, or host threads) race on the array: order
 * them on one stream. */
#define OSTRICH_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Capacity of ostrich_step_adjoint_noalloc for a scene: *max_worlds receives how many
 * worlds one call accepts (the array divided by the scene's FP32 per-world tape record),
 * *record_bytes (may be NULL) that record's size.  Host only, touches no device.  EINVAL
 * for a scene the entry point refuses (heightmap, or a description ostrich_create would
 * refuse) or a NULL max_worlds. */
ostrich_status ostrich_noalloc_capacity(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg,
                                        int32_t* max_worlds, size_t* record_bytes);
ostrich_status ostrich_step_adjoint_noalloc(const ostrich_scene_desc* scene, const ostrich_solver_cfg* cfg,
                                            int n_worlds, int ld, const float* state_in, const float* controls,
                                            double h, float* state_out, const float* dL_dstate_next,
                                            float* dL_dstate, float* dL_dcontrols, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OSTRICH_H */
