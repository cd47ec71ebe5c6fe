/*
 * abasim: batched, differentiable articulated-body simulation on one GPU (C ABI).
 *
 * Computes, for many independent articulated systems at once, time-stepped
 * forward dynamics with Featherstone's Articulated Body Algorithm plus an Euler
 * integrator, and the reverse-mode adjoint of that rollout with only the
 * per-step initial states checkpointed and the intermediates recomputed during
 * backprop (Qiao et al., "Efficient Differentiable Simulation of Articulated
 * Bodies", ICML 2021: problem statement Sec. 2; step modules and adjoint Sec. 3.1,
 * Eq. 3-6; checkpointing Sec. 3.2, Eq. 7; checkpoint interval supplement Sec. B).
 *
 * Layouts.  Every per-system array is structure-of-arrays with the system index
 * fastest and the coordinate index zero-padded to the batch maximum:
 *   q    [nq_max][B]        generalized positions (revolute angle; free joint:
 *                           world position p then unit quaternion x y z w)
 *   qd   [nv_max][B]        generalized velocities (free joint: body-frame
 *                           angular then linear velocity)
 *   tau  [T][nv_max][B]     joint forces; tau^t acts over step t -> t+1
 *   ckpt [ceil(T/k)][nq_max+nv_max][B]   x^t = (q^t, qd^t) for t = 0, k, 2k, ...
 *   traj [T+1][nq_max+nv_max][B]         x^0 .. x^T (optional)
 * Scalars are double for SIM_FP64 and float for SIM_FP32 / SIM_FP32_D64.
 * Per-link arrays (gmass, set_masses) follow the link order of the model
 * description (CSR by system).
 *
 * Ownership.  Every array argument of the step / rollout / backward calls is
 * DEVICE memory owned by the caller, on the device that was current at
 * sim_create.  Those calls allocate nothing; they enqueue kernels on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and return without waiting.
 * Model constants, the per-step tape and the status words are owned by the
 * handle.
 *
 * Errors.  Every call returns SIM_OK (0) or a negative SIM_E* code and stores a
 * message readable with sim_last_error(handle) (sim_last_error(NULL) for a
 * failed sim_create).  Non-finite results are reported per system through
 * sim_status, never by a trap.
 */
#ifndef ABASIM_H
#define ABASIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIM_OK 0
#define SIM_EINVAL (-1)      /* bad model, size or pointer */
#define SIM_ECUDA (-2)       /* a CUDA runtime call failed */
#define SIM_ENOMEM (-3)      /* device allocation or caller workspace too small */
#define SIM_ENONFINITE (-4)  /* sim_status: some system produced NaN/Inf */
/* -5 is reserved for a timed-out wait; no call has one: the kernels never spin on
 * a flag (the two-warp kernels hand data over through hardware named barriers that
 * both warps reach the same number of times). */
#define SIM_EUNSUPPORTED (-6) /* a valid request this build or model cannot run (the
                               * message says which) */

enum sim_precision { SIM_FP64 = 0, SIM_FP32 = 1, SIM_FP32_D64 = 2 };
enum sim_integrator { SIM_SEMI_IMPLICIT_EULER = 0, SIM_EXPLICIT_EULER = 1 };
enum sim_joint { SIM_REVOLUTE = 0, SIM_FREE = 1 };

/* Model description, host memory, copied by sim_create.
 * Links are stored CSR by system (sys_link_offset[n_systems+1]); within a system
 * they are in topological order: parent[l] is the parent's index inside the
 * same system and must be < l, or -1 for the world.  A SIM_FREE joint is allowed
 * only on a system's first link (the floating base).  Per link:
 *   axis[3]     unit rotation axis in the link frame (revolute); sim_create
 *               re-expresses each revolute link in a frame whose z axis is this
 *               axis (no state, input or gradient depends on the link frames)
 *   X_tree[12]  parent frame -> joint frame: rotation E (row major, 9) then the
 *               joint origin r in parent coordinates (3); motion vectors map as
 *               [E w; E (v - r x w)] (the supplement's st_apply)
 *   mass, com[3], I_com[6]  rigid-body inertia: mass, centre of mass in the link
 *               frame, rotational inertia about the COM (xx yy zz xy xz yz)
 *   damping     viscous damping of a revolute joint: the joint force is
 *               tau - damping * qd (NULL: none; ignored for free joints)
 *   contact[4]  a contact sphere rigidly attached to the link: centre in the link
 *               frame (3) and radius (a negative radius: none).  NULL: no contacts.
 *   limits[2]   position limits lo < hi of a revolute joint (-inf / +inf: no limit
 *               on that side).  NULL: no limits.  Finite limits on a free joint are
 *               rejected.
 * gravity[3] is the world-frame gravitational acceleration (e.g. 0 0 -9.81).
 *
 * Contacts and joint limits (Sec. 3.1 "collision resolution", Eq. 8; the
 * projected Gauss-Seidel solver of the supplement, Alg. 1): each sphere is
 * tested against the ground plane z = 0 with gap phi = (world z of its centre) -
 * radius; at most SIM_MAX_CONTACTS spheres per system.  Each limited joint is
 * tested against its range: below it the row is J = +e_j with gap q - lo, above
 * it J = -e_j with gap hi - q; at most SIM_MAX_LIMITS limited joints per system.
 * For the rows with phi < 0, the impulses lambda (world x, y friction, z normal
 * per contact, then one per limit row) solve the mixed LCP a = A lambda + b,
 * A = J M^-1 J^T (J: world velocity Jacobian of the sphere centres, then the
 * limit rows), b = J (qd + dt qdd) + (erp / dt) phi on the normal and limit rows,
 * lambda_z >= 0 complementary to a_z, |lambda_x|, |lambda_y| <= friction *
 * lambda_z, limit impulses >= 0 complementary to their rows, by pgs_iterations
 * Gauss-Seidel sweeps (per contact the normal row, then x, then y; then the limit
 * rows) from lambda = 0; the velocity change M^-1 J^T lambda is added to the
 * step's qd update.
 * friction >= 0, erp in [0, 1], pgs_iterations in [1, SIM_MAX_PGS_ITERATIONS];
 * all three are ignored without contact spheres or limits.  The adjoint
 * differentiates the solver's iterations exactly (the active set is held fixed).
 * sim_step_jvp returns SIM_EUNSUPPORTED for models with contact spheres or
 * limits. */
/* Slot packing (how systems are assigned to the kernels' threads).  By default
 * systems are sorted by link count, longest first, so a warp's 32 systems walk
 * equally many links.  With SIM_KEEP_SYSTEM_ORDER in flags they keep their own
 * order: a warp then holds 32 consecutive systems, so the per-step state,
 * torque, checkpoint and gradient streams (indexed by system) are read and
 * written as whole cache lines, at the price of warps whose systems walk
 * different numbers of links.  Results do not depend on the packing. */
#define SIM_KEEP_SYSTEM_ORDER 1
#define SIM_MAX_CONTACTS 4
#define SIM_MAX_LIMITS 12
#define SIM_MAX_PGS_ITERATIONS 64
typedef struct sim_model_desc {
  int32_t n_systems;
  int32_t precision;   /* enum sim_precision */
  int32_t integrator;  /* enum sim_integrator */
  int32_t flags;       /* 0 or SIM_KEEP_SYSTEM_ORDER */
  double dt;
  double gravity[3];
  const int32_t* sys_link_offset;
  const int32_t* parent;
  const int32_t* joint_type;
  const double* axis;
  const double* X_tree;
  const double* mass;
  const double* com;
  const double* I_com;
  const double* damping;  /* [1] per link or NULL: viscous joint damping b >= 0 */
  const double* contact;  /* [4] per link or NULL: contact sphere centre and radius */
  double friction;        /* Coulomb coefficient of the friction box */
  double erp;             /* fraction of the penetration removed per step */
  int32_t pgs_iterations; /* Gauss-Seidel sweeps of the contact solver */
  int32_t reserved2;
  const double* limits;   /* [2] per link or NULL: revolute joint position limits */
} sim_model_desc;

typedef struct sim_handle sim_handle;

/* Validate and pack a model (Sec. 2: state x = [q, qd], control u = tau), upload
 * its constants to the current device and allocate the per-step tape.  Each
 * system's links are stored in depth-first preorder (children in the model's
 * order); coordinates, masses and every result keep the model's numbering.
 * Returns SIM_EINVAL with a message for an invalid tree, joint, axis, rotation or
 * inertia; SIM_ENOMEM / SIM_ECUDA for device failures.  *out is NULL on error. */
int sim_create(const sim_model_desc* desc, sim_handle** out);

/* Free every device and host resource of the handle.  NULL is ignored. */
void sim_destroy(sim_handle* h);

/* Batch dimensions: number of systems, padded coordinate counts, links. */
int sim_dims(const sim_handle* h, int32_t* n_systems, int32_t* nq_max, int32_t* nv_max,
             int32_t* n_links_total);

/* Bytes of the checkpoint buffer for a T-step rollout with interval k >= 1:
 * ceil(T/k) states (Sec. 3.2; the supplement's memory model n/k * m_ckpt). */
size_t sim_ckpt_bytes(const sim_handle* h, int64_t T, int32_t k);

/* Bytes of caller workspace sim_backward_rollout needs for interval k (the k
 * replayed states of one segment); 0 for k == 1. */
size_t sim_work_bytes(const sim_handle* h, int32_t k);

/* Replace every link mass from a device array [n_links_total] of the handle's
 * scalar type, COM and rotational inertia held fixed.  Stream ordered.  The masses
 * are the model parameters the adjoint differentiates besides the controls (Sec. 3.1:
 * after Eq. 4 the paper notes that the gradients of other parameters follow the
 * same way as those of u^k; here I(m) = [Ic + m cx cx^T, m cx; m cx^T, m 1] with
 * c and Ic fixed), so a caller can set them, roll out, and read dPhi/dm from
 * sim_backward_rollout. */
int sim_set_masses(sim_handle* h, const void* mass, void* stream);

/* One step x -> x' for every system (Sec. 3.1: kinematics, the three ABA passes,
 * integration).  q, qd may alias q_out, qd_out. */
int sim_step_batch(sim_handle* h, const void* q, const void* qd, const void* tau, void* q_out,
                   void* qd_out, void* stream);

/* Size of the library's static step scratch used by sim_step_batch_static. */
#define SIM_STATIC_SCRATCH_BYTES (16u << 20)

/* One step x -> x' like sim_step_batch, for callers that cannot allocate device
 * memory.  Examples: a plug-in inside a host application (a physics or game
 * engine, robotics middleware, a serving process) that owns every device
 * allocation through its own pool and only hands the plug-in a handle and state
 * buffers, so that its memory budget stays exact; or a real-time control loop in
 * which cudaMalloc's implicit synchronisation and unbounded latency are not
 * allowed.  The paper has no counterpart; this is a deployment convenience.
 * Allocates nothing: the per-link tape is a file-scope device array of
 * SIM_STATIC_SCRATCH_BYTES (16 MiB) that every GPU loading the library holds
 * until the process exits; batches whose tape (links x 119 scalars x systems x
 * scalar size) exceeds it are rejected with SIM_ENOMEM and a message.  The first
 * call on each device looks up the array's device address (once, with that
 * device current); make that first call before any stream capture.  The device
 * current at the call must be the handle's (the one current at sim_create), else
 * SIM_EINVAL.  The array is shared by all calls and keeps the last call's
 * contents (every word a step reads is written earlier in the same step, so
 * nothing needs clearing); calls whose kernels overlap on the GPU race on it, so
 * serialize them (one stream, or events).  For a model with contact spheres or
 * joint limits the constraint solver's per-system scratch is the handle's,
 * allocated once by sim_create.  Same layouts, ownership and error codes as
 * sim_step_batch. */
int sim_step_batch_static(sim_handle* h, const void* q, const void* qd, const void* tau,
                          void* q_out, void* qd_out, void* stream);

/* T steps from (q0, qd0) under tau [T][nv_max][B] (Sec. 2: x^{k+1} from x^k and
 * u^k; each step as sim_step_batch).  Writes x^T to (qT, qdT), the checkpoints
 * x^0, x^k, ... to ckpt (if non-NULL; sim_ckpt_bytes(T, k) bytes) and every state
 * to traj (if non-NULL).  Only these step-initial states are kept, never a
 * step's intermediates (Sec. 3.2, Fig. 2: the checkpoint of step k is its initial
 * state; k > 1 is the sparser interval of the supplement's Sec. B).  T == 0
 * copies the input. */
int sim_rollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T,
                int32_t k, void* ckpt, void* qT, void* qdT, void* traj, void* stream);

/* Forward-mode derivative of one step (the Jacobian-vector product the paper's
 * RL sample enhancement needs, Sec. 4: s'(a + da) ~ s'(a) + ds'/da da):
 * (q_out, qd_out) = x' as sim_step_batch, (dq_out, dqd_out) = dx'/dx (dq, dqd)
 * + dx'/dtau dtau.  Any of dq, dqd, dtau may be NULL (zero tangent).  The step
 * runs on dual numbers in the caller's workspace of sim_jvp_work_bytes() bytes.
 * The SIM_FP32_D64 mode runs this call in plain FP32. */
size_t sim_jvp_work_bytes(const sim_handle* h);
int sim_step_jvp(sim_handle* h, const void* q, const void* qd, const void* tau, const void* dq,
                 const void* dqd, const void* dtau, void* q_out, void* qd_out, void* dq_out,
                 void* dqd_out, void* work, size_t work_bytes, void* stream);

/* Adjoint of sim_rollout (Sec. 3.1 Eq. 3-4: R^k = xbar^k pulled back step by step;
 * Sec. 3.2 Eq. 7: each step recomputed from its checkpoint; for k > 1 each
 * segment is replayed forward once into `work` and then differentiated).
 * Seeds: gqT, gqdT = dPhi/dx^T; g_traj (optional, traj layout) adds dPhi/dx^t
 * for t = 0..T.  Outputs (overwritten): gq0, gqd0 = dPhi/dx^0, gtau
 * [T][nv_max][B] = dPhi/dtau, gmass [n_links_total] = dPhi/dm (optional; COM and
 * rotational inertia held fixed).  Padded coordinates come back as 0. */
int sim_backward_rollout(sim_handle* h, const void* ckpt, const void* tau, int64_t T, int32_t k,
                         const void* gqT, const void* gqdT, const void* g_traj, void* gq0,
                         void* gqd0, void* gtau, void* gmass, void* work, size_t work_bytes,
                         void* stream);

/* Copy the per-system status words to host memory flags[n_systems] (bit 0:
 * a non-finite state or gradient was produced since the last sim_clear_status)
 * after synchronizing the device.  Returns SIM_ENONFINITE if any bit is set. */
int sim_status(sim_handle* h, int32_t* flags);
int sim_clear_status(sim_handle* h, void* stream);

/* Launch shape of the batched kernels (the autotuner drives this).  threads:
 * threads per block, a multiple of 32 in [32, 1024] (0 = default 32); each block
 * is one work unit of `threads` consecutive slots.  schedule SIM_SCHED_GRID
 * launches one block per unit; SIM_SCHED_PERSISTENT launches as many blocks as
 * fit on the device at once and each takes units from an atomic ticket until
 * none is left (one persistent launch per rollout). */
#define SIM_SCHED_GRID 0
#define SIM_SCHED_PERSISTENT 1
int sim_set_launch(sim_handle* h, int32_t threads, int32_t schedule);

/* Where the per-step tape lives: SIM_TAPE_AUTO (default) puts it in shared
 * memory when the block's tiles of 32 systems fit the per-block limit, else in
 * the handle's global scratch; SIM_TAPE_GLOBAL / SIM_TAPE_SHARED force one
 * (SHARED fails with SIM_EUNSUPPORTED at launch if it does not fit).
 * SIM_TAPE_PIPELINED runs batches of serial revolute chains with two warps per
 * 32-system tile: in the rollout (any precision, chains of at most 14 links) one
 * warp runs the articulated-inertia recursion of each step while the other runs
 * the velocity, bias-force and acceleration passes; in the adjoint (FP32 storage,
 * checkpoint interval 1) one warp recomputes step t's forward intermediates into
 * one of two shared-memory tapes while the other differentiates step t + 1 from
 * the other tape (when the two tapes fit, about 7 links).  AUTO picks each when it
 * applies; forcing it fails with SIM_EUNSUPPORTED where it does not.
 * SIM_TAPE_ONE_WARP chooses like AUTO among the one-warp-per-tile kernels only
 * (the autotuner times both, as one or two lanes per system).  Models with contact spheres or joint limits always run with the tape
 * in global memory.  Results do not depend on the choice beyond rounding. */
#define SIM_TAPE_AUTO 0
#define SIM_TAPE_GLOBAL 1
#define SIM_TAPE_SHARED 2
#define SIM_TAPE_PIPELINED 3
#define SIM_TAPE_ONE_WARP 4  /* as SIM_TAPE_AUTO, without the pipelined kernels */
/* SIM_TAPE_ALIGNED runs models whose joints are all revolute, with no contact
 * spheres or limits, on the kernels of the world-aligned step: the same ABA step
 * and adjoint (Sec. 3.1) written in link frames that keep the world's
 * orientation with their origin at the joint, so that the inward recursion on
 * the articulated inertias translates them from child to parent instead of
 * rotating and translating them (each body's inertia is rotated into world axes
 * once per step, off that serial chain).  Tape and adjoint record in shared
 * memory when a block's tiles fit, else in the handle's global scratch (whose
 * lines each pass prefetches sim_set_prefetch links ahead).  Links are stored in
 * depth-first preorder; the values a branching link hands to or collects from
 * its later children live on a per-system stack (in shared memory with an
 * on-chip tape, else in a handle buffer) as deep as the nesting of branchings.
 * AUTO picks these kernels for such
 * models, except where the pipelined kernels apply (serial chains short enough
 * for their on-chip tapes) and where a system's state and input streams exceed a
 * block's shared memory; forcing them on another model fails with
 * SIM_EUNSUPPORTED.  The FP64 state accumulation of SIM_FP32_D64 rollouts is not
 * available on them (AUTO then takes the one-warp kernels). */
#define SIM_TAPE_ALIGNED 5
/* SIM_TAPE_ALIGNED_PIPELINED is SIM_TAPE_ALIGNED with the adjoint (checkpoint
 * interval 1) on two warps per 32-system tile: one recomputes step t's forward
 * intermediates (Sec. 3.2, Eq. 7) into one of two tapes while the other runs the
 * adjoint of step t + 1 from the other tape (on chip when a tile's tapes fit a
 * block, else in global memory).  AUTO uses this adjoint wherever it uses the
 * world-aligned kernels with k = 1. */
#define SIM_TAPE_ALIGNED_PIPELINED 6
int sim_set_tape_space(sim_handle* h, int32_t space);

/* The storage mode the last sim_rollout (or step) and sim_backward_rollout
 * launches of this handle ran with: 0 tape in global memory, 1 tape global with
 * state and input streams on chip, 2 tape on chip, 3 the pipelined two-warp
 * kernels, 4 the world-aligned kernels with the tape on chip, 5 the world-aligned
 * kernels with the tape in global memory, 6 / 7 the pipelined world-aligned adjoint
 * with its tapes on chip / in global memory.  Either pointer may be NULL.  No
 * device work. */
int sim_last_storage(const sim_handle* h, int32_t* rollout_mode, int32_t* backward_mode);

/* Prefetch distance of the world-aligned kernels when their tape is in global
 * memory: while link l computes, each pass asks for the cache lines of the link
 * links_ahead further along its walk (and the next step's input lines), so a
 * warp's tape reads find L1 instead of waiting on L2 / HBM once per link.
 * 0 switches prefetching off; default 2; at most 16.  A tuning control (the
 * autotuner may set it); results do not depend on it. */
int sim_set_prefetch(sim_handle* h, int32_t links_ahead);

/* How sim_backward_rollout rebuilds the states inside a checkpoint segment when
 * k > 1.  SIM_REPLAY_SEGMENT (default): replay the segment once into the caller
 * workspace, then differentiate it backwards (≈ one extra forward step per step).
 * SIM_REPLAY_QUADRATIC: the supplement's scheme (Sec. B) — every state x^t is
 * recomputed from the segment's checkpoint, (k+1)k/2 forward steps per segment,
 * giving its (k+1)/2 · t_forward + t_backward time per step.  Same gradients. */
#define SIM_REPLAY_SEGMENT 0
#define SIM_REPLAY_QUADRATIC 1
int sim_set_replay(sim_handle* h, int32_t mode);

/* Running-state precision of sim_rollout in SIM_FP32_D64 mode (the mixed mode's
 * FP64 D-solves leave the step-to-step state sums in FP32; the paper does not say
 * which).  fp64 = 1: sim_rollout keeps q and qd in FP64 (device memory the handle
 * allocates here, (nq_max + nv_max) * n_systems doubles) and accumulates the
 * integrator's sums there; every step's dynamics read the FP32 rounding of that
 * state, and the checkpoints, trajectory and final state are stored as FP32.
 * fp64 = 0 (default): the state is FP32 throughout.  With the flag on,
 * sim_step_batch (a one-step sim_rollout) also sums in FP64, starting from the
 * FP64 widening of its FP32 input, and returns the FP32 rounding.  The
 * backward's segment replay (k > 1) sums in FP32, so its replayed states can
 * differ from the rollout's by FP32 rounding; with k = 1 the adjoint recomputes
 * every step from exactly the FP32 state the rollout evaluated.  Rollouts then
 * use the one-warp kernels.  Returns
 * SIM_EUNSUPPORTED for the other precisions and SIM_ECUDA if the buffer cannot
 * be allocated.  Not thread-safe with a rollout in flight on the handle. */
int sim_set_state_accumulation(sim_handle* h, int32_t fp64);

/* The packing of systems into slots (thread order): sys_of_slot[n_systems]
 * (host memory) receives the system index run by each slot.  Systems are sorted
 * by link count, longest first, so the systems of a warp walk equally many links
 * and the longest work is issued first; results do not depend on it. */
int sim_slot_order(const sim_handle* h, int32_t* sys_of_slot);

/* Message of the last failed call on h (or of the last failed sim_create when h
 * is NULL).  Owned by the library, valid until the next call on h. */
const char* sim_last_error(const sim_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* ABASIM_H */
