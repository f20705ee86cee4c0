/*
 * pbdr.h - C ABI of the GB300 (sm_103a) PBD-R solver.
 *
 * PBD-R ("Physically Accurate Rigid-Body Dynamics in Particle-Based
 * Simulation", arXiv 2603.14634) steps rigid bodies made of equal spheres
 * ("particles") with position-based dynamics.  One substep is Algorithm 1:
 *   - integration:  v~ = v + dt w f_ext(x),  x~ = x + dt v~       (Alg. 1, integration)
 *   - K solver iterations, each:                                    (Alg. 1, solver loop)
 *       ground contact dX_PG and particle-particle contact dX_PP between
 *       particles of different bodies, with Coulomb friction (Sec. III-A),
 *       shape matching dX_SM toward the best rigid fit of the rest shape
 *       (Sec. III-A (3), Sec. III-C),
 *       incremental velocity update V_{i+1} = V_i + dX/dt (Sec. III-B, Eqs. 1-2),
 *       momentum enforcement: uniform dv and rigid w corrections restoring the
 *       linear and angular momentum of the body before shape matching
 *       (Sec. III-C, Eqs. lin_momentum and ang_momentum).
 * Contact candidates are found once per substep on x~ with a hashed uniform
 * grid (pairs closer than Rn = 2.2 r, FP32 predicate; the paper does not
 * specify the search).
 *
 * Conventions
 *   - All functions return PBDR_OK (0) or a negative PBDR_ERR_* code; no C++
 *     exception crosses the ABI.  pbdr_last_error() gives a message for the
 *     calling thread's last failure.
 *   - Host arrays are owned by the caller and copied; the library owns every
 *     device allocation (state, neighbour lists, sort buffers, graphs).
 *   - Particle order on input and output is the caller's order.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that return device results to host buffers synchronise that stream;
 *     pbdr_step is asynchronous.
 *   - A context is bound to one device and is not thread-safe: one thread
 *     drives a context at a time.  Its device buffers are shared by all its
 *     calls, which therefore run in stream order: a caller that switches
 *     streams between calls synchronises the earlier stream first.
 *   - Units are SI; state is FP32.
 */
#ifndef PBDR_H
#define PBDR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define PBDR_OK 0
#define PBDR_ERR_INVALID (-1)      /* bad argument or descriptor */
#define PBDR_ERR_OOM (-2)          /* device allocation failed */
#define PBDR_ERR_BUDGET (-3)       /* request exceeds the context's HBM budget */
#define PBDR_ERR_NBR_OVERFLOW (-4) /* a neighbour list exceeded its capacity */
#define PBDR_ERR_NONFINITE (-5)    /* a non-finite position was produced */
#define PBDR_ERR_TIMEOUT (-6)      /* a bounded device wait gave up */
#define PBDR_ERR_CUDA (-7)         /* a CUDA runtime call failed */
#define PBDR_ERR_UNSUPPORTED (-8)  /* a flag combination the GPU path does not implement */

/* per-scene error bits reported by pbdr_read_state / pbdr_read_states */
#define PBDR_EBIT_NBR_OVERFLOW (1u << 0) /* a neighbour list was truncated */
#define PBDR_EBIT_NONFINITE (1u << 1)    /* a position became NaN or Inf */

/* scene flags (ablations of Sec. V-C and readings of the paper) */
#define PBDR_STD_VELOCITY (1u << 0) /* V = (X - X_init)/dt (standard PBD, Sec. III-A) */
#define PBDR_NO_LINMOM (1u << 1)    /* drop Eq. lin_momentum */
#define PBDR_NO_ANGMOM (1u << 2)    /* drop Eq. ang_momentum */
#define PBDR_CONTACT_AVG (1u << 3)  /* average particle-particle corrections per particle */
#define PBDR_SM_FROM_XI (1u << 4)   /* shape matching on X_i instead of X_i + contacts */

typedef struct pbdr_ctx pbdr_ctx; /* opaque: device state, scene table, plans, graphs */
typedef int32_t pbdr_scene;       /* scene handle, >= 0 */

/* One independent scene (Sec. III notation).  Particles of body b are
 * [body_off[b], body_off[b+1]).  The rest shape of each body is its
 * configuration at creation: q_p = x_p - c_b (Mueller et al. 2005). */
typedef struct {
  int32_t num_particles;   /* N >= 0 */
  int32_t num_bodies;      /* B >= 1 when N > 0 */
  const float *pos;        /* [N*3] host, xyz per particle */
  const float *vel;        /* [N*3] host */
  const float *inv_mass;   /* [N] host, w_p > 0 and finite */
  const int32_t *body_off; /* [B+1] host, body_off[0] = 0, strictly increasing, body_off[B] = N */
  float radius;            /* r > 0, equal for every particle of the scene */
  float friction;          /* mu >= 0 (kinetic coefficient, Table I; static = kinetic) */
  float gravity[3];        /* m/s^2 */
  float plane[4];          /* ground n.x = d: n (unit) = plane[0..2], d = plane[3];
                              particles are kept on the side n.x >= d + r */
  float dt;                /* substep length > 0 */
  int32_t iterations;      /* solver iterations K, 1..1024 */
  uint32_t flags;          /* PBDR_* scene flags */
} pbdr_scene_desc;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context may hold (0 = no cap).  *out receives the handle.
 * Errors: PBDR_ERR_INVALID (bad device or NULL out), PBDR_ERR_CUDA. */
int pbdr_ctx_create(int device, size_t hbm_budget_bytes, pbdr_ctx **out);

/* Frees every device resource of the context.  NULL is accepted. */
int pbdr_ctx_destroy(pbdr_ctx *ctx);

/* Copies a scene into device memory (synchronous: the copies have landed
 * when it returns) and returns its handle.  Computes M_b, c_b and the rest
 * offsets in FP64 on the host.  Slots and table ranges of destroyed scenes
 * are reused; a call that reuses one that was freed while library work was
 * still in flight (see pbdr_destroy_scene) first waits for the device to
 * finish the work already queued, otherwise it does not wait, and work of
 * other scenes may run meanwhile on non-blocking streams.
 * Errors: PBDR_ERR_INVALID (descriptor check failed: sizes, offsets, masses,
 * radius, dt, iterations, plane normal), PBDR_ERR_BUDGET, PBDR_ERR_OOM,
 * PBDR_ERR_UNSUPPORTED (flags). */
int pbdr_create_scene(pbdr_ctx *ctx, const pbdr_scene_desc *desc, pbdr_scene *out);

/* Removes a scene from the context; its handle becomes invalid.  Never
 * waits: it checks (without blocking) whether the work of every earlier call
 * that took a stream has completed, e.g. after a pbdr_read_state(s) of the
 * results; if not, the next pbdr_create_scene that reuses the freed slot or
 * ranges waits for the device. */
int pbdr_destroy_scene(pbdr_ctx *ctx, pbdr_scene scene);

/* Sets a constant external force F (N) at the centre of mass and a constant
 * torque tau (N m) about it on one body (the f_ext of the integration step of Alg. 1, for the
 * pushed-box and box-with-torque tests of Table I).  Each particle receives
 * F/M + alpha x (x - c) with alpha = I^-1 tau, c and I taken at the start of
 * the substep.  Zero F and tau remove the wrench.  Synchronous. */
int pbdr_set_body_wrench(pbdr_ctx *ctx, pbdr_scene scene, int32_t body,
                         const float F[3], const float tau[3]);

/* Advances the n scenes ids[0..n) by `substeps` PBD-R substeps (Algorithm 1)
 * on `stream`, asynchronously.  All scenes of one call are stepped together
 * in the same kernels (batched); scenes are independent.  Results are
 * bit-identical whatever other scenes share the call.
 * Errors: PBDR_ERR_INVALID (bad handle, duplicate id, n < 1, substeps < 0),
 * PBDR_ERR_OOM, PBDR_ERR_CUDA.  Device-side problems (neighbour overflow,
 * non-finite positions) are reported per scene by pbdr_read_state. */
int pbdr_step(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, int32_t substeps,
              void *stream);

/* Copies one scene's state to host buffers pos, vel ([N*3] each, may be
 * NULL) and its error bits to *err_bits (may be NULL; bits are cleared by
 * the read), then synchronises `stream`. */
int pbdr_read_state(pbdr_ctx *ctx, pbdr_scene scene, float *pos, float *vel,
                    uint32_t *err_bits, void *stream);

/* Overwrites one scene's state from host buffers pos, vel ([N*3] each; NULL
 * leaves that part unchanged) on `stream`; the host buffers must stay valid
 * until the stream reaches this point (pbdr_read_state or a stream sync).
 * The rest shape is not changed. */
int pbdr_write_state(pbdr_ctx *ctx, pbdr_scene scene, const float *pos,
                     const float *vel, void *stream);

/* Batched forms: the scenes' particles are concatenated in the order of ids
 * (host buffers [sum N_s * 3]); err_bits is [n] (may be NULL).  One device
 * gather/scatter plus one copy each way.  read synchronises `stream`. */
int pbdr_read_states(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, float *pos,
                     float *vel, uint32_t *err_bits, void *stream);
int pbdr_write_states(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n,
                      const float *pos, const float *vel, void *stream);

/* pbdr_read_states without the final synchronisation: enqueues the gather
 * and the copies on `stream` and returns.  pos, vel and err_bits are valid
 * once the stream has reached this point (an event recorded after the call,
 * or a stream sync); page-locked host buffers keep the copies asynchronous
 * (pageable ones make them wait for the stream).  The device staging area is
 * shared with the other reads and writes of states, so issue those on the
 * same stream or after this read has completed.  A scene read this way
 * counts as in use until the read completes: destroying it earlier makes
 * the next scene that reuses its ranges wait for the device.  Serving uses
 * it to read finished requests between two substeps on one stream. */
int pbdr_read_states_async(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, float *pos,
                           float *vel, uint32_t *err_bits, void *stream);

/* Number of particles and bodies of a scene (either pointer may be NULL). */
int pbdr_scene_info(pbdr_ctx *ctx, pbdr_scene scene, int32_t *num_particles,
                    int32_t *num_bodies);

/* Message of the calling thread's last error ("" if none).  The pointer stays
 * valid until the thread's next pbdr_* call. */
const char *pbdr_last_error(void);

/* ---- inspection (tests and profiling) ---------------------------------- */

/* Runs only the neighbour stage (cell keys, radix sort, cell ranges,
 * neighbour lists) of the scenes ids[0..n) on their CURRENT positions, taken
 * as the predicted positions x~; the state is not modified. */
int pbdr_build_neighbors(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, void *stream);

/* Reads one scene's result of the last neighbour stage, in scene-local
 * numbering: sorted_key[N] (bucket in [0, T_s), T_s = smallest power of two
 * >= 2N) and sorted_id[N] (particle index), sorted by key and by id within a
 * key; off[N+1] and idx (ascending neighbour indices of each particle, CSR).
 * idx_cap bounds idx; *idx_count receives the total.  Any pointer except
 * idx_count may be NULL.  Synchronises `stream`. */
int pbdr_read_neighbors(pbdr_ctx *ctx, pbdr_scene scene, uint32_t *sorted_key,
                        uint32_t *sorted_id, int32_t *off, int32_t *idx,
                        int64_t idx_cap, int64_t *idx_count, void *stream);

/* Execution options (each call drops the cached step plans).
 * PBDR_OPT_PATH: 0 (default) = scenes of up to 8192 particles run in the
 *   scene-resident kernel (one CTA keeps a scene in shared memory for the
 *   whole substep), larger scenes in the streaming kernels; 1 = streaming
 *   kernels for every scene (one launch per stage and per iteration).
 * PBDR_OPT_FUSED_THREADS: threads per CTA of the scene-resident kernel,
 *   0 (default) = per size class, else a multiple of 32 in 32..512. */
#define PBDR_OPT_PATH 1
#define PBDR_OPT_FUSED_THREADS 2
/* PBDR_OPT_GRAPHS: 1 (default) = the first pbdr_step of a scene set captures
 *   one substep into a CUDA graph and every substep replays it (not on the
 *   legacy NULL stream, and not while stage timing is on); 0 = plain launches.
 * PBDR_OPT_AUTOTUNE: 1 (default) = once a scene set has run
 *   PBDR_OPT_TUNE_AFTER substeps (contacts have formed), the scene-resident
 *   kernel's launch shapes are
 *   timed per size class with at least as many scenes as SMs (threads per
 *   CTA, scratch and velocities in shared or global memory, CTAs per SM), on
 *   whole substeps from the same saved state whose effects are undone, and
 *   the fastest is kept (and reused for later sets with the same class
 *   sizes); results do not depend on the shape. */
#define PBDR_OPT_GRAPHS 3
#define PBDR_OPT_AUTOTUNE 4
/* PBDR_OPT_TUNE_AFTER: substeps a scene set runs before its launch shapes are
 *   tuned, >= 1 (default 128): a state close to the one that will be stepped
 *   most (bodies at rest after a drop, say) gives the most useful timings. */
#define PBDR_OPT_TUNE_AFTER 5
int pbdr_set_option(pbdr_ctx *ctx, int32_t option, int64_t value);

/* Tangent-linear (forward-mode) substeps: the derivative of Algorithm 1's
 * map from the state at the start of a substep to the state at its end,
 * along a direction given per particle (dX, dV).  pbdr_step_tangent advances
 * the scenes ids[0..n) by `substeps` substeps of the streaming form (the
 * primal state exactly as pbdr_step with PBDR_OPT_PATH = 1 advances it) and
 * their tangents with them: prediction x~' = x' + dt v', then per iteration
 * the derivative of the contacts with friction (Sec. III-A (1), (2)), of
 * shape matching including the rotation (from the polar decomposition
 * A = R S: dR = R [w]x with (tr(S) I - S) w = axial(R^T dA - dA^T R)), of the
 * velocity update (Sec. III-B) and of the momentum constraint (Sec. III-C,
 * Eqs. lin_momentum / ang_momentum, including the change of the inertia
 * tensor).  The neighbour lists, the contact set and the sticking/sliding
 * branch of every friction term are the primal's (the tangent is the
 * derivative inside those pieces).  Scenes with a body wrench or with
 * PBDR_STD_VELOCITY / PBDR_SM_FROM_XI give PBDR_ERR_UNSUPPORTED.
 * Tangent storage (4 float4 per particle) is allocated on first use; new
 * scenes start with zero tangents.  Asynchronous on `stream`.
 * Errors: PBDR_ERR_INVALID, PBDR_ERR_UNSUPPORTED, PBDR_ERR_OOM,
 * PBDR_ERR_BUDGET, PBDR_ERR_CUDA. */
int pbdr_step_tangent(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, int32_t substeps,
                      void *stream);

/* Sets the tangent of one scene's friction coefficient mu (default 0): the
 * friction terms then carry d(mu pen) = dmu pen + mu d(pen).  Synchronous. */
int pbdr_write_tangent_friction(pbdr_ctx *ctx, pbdr_scene scene, float dmu, void *stream);

/* Sets the tangent of one scene: dpos, dvel host [N*3] in the caller's
 * particle order (NULL = zero).  Stream-ordered on `stream`; the host
 * buffers must stay valid until the stream reaches this point. */
int pbdr_write_tangent(pbdr_ctx *ctx, pbdr_scene scene, const float *dpos, const float *dvel,
                       void *stream);

/* Reads the tangent of one scene into host [N*3] arrays (NULL = skip) and
 * synchronises `stream`.  PBDR_ERR_INVALID before any tangent exists. */
int pbdr_read_tangent(pbdr_ctx *ctx, pbdr_scene scene, float *dpos, float *dvel, void *stream);

/* Reverse mode (adjoint): the gradient of a scalar loss of the final state
 * with respect to the initial state, through `substeps` substeps of the
 * streaming form.  Before the call the adjoint buffers hold dLoss/dX, dLoss/dV
 * of the final state (pbdr_write_adjoint); the scenes hold the initial state.
 * The call runs the substeps forward, keeping device checkpoints every
 * `checkpoint_every` substeps, then sweeps backward: each segment is run
 * forward again from its checkpoint, and each substep once more keeping the
 * state before each solver iteration, whose adjoint is then taken by hand-
 * written kernels (the transpose of the derivative pbdr_step_tangent
 * propagates: contacts with friction, shape matching and the rotation from
 * the polar decomposition, velocity update, momentum constraint).  Contact
 * terms are gathered per particle over the symmetric neighbour lists (no
 * atomics: the result is deterministic).  On return the adjoint buffers hold
 * dLoss/dX, dLoss/dV of the initial state (pbdr_read_adjoint) and the scenes
 * hold the final state.  Device memory: (substeps/checkpoint_every +
 * checkpoint_every + K + 1) saved states of the context (32 B per particle,
 * 32 B per body each).  Same restrictions and errors as pbdr_step_tangent. */
int pbdr_adjoint(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, int32_t substeps,
                 int32_t checkpoint_every, void *stream);

/* Sets the adjoint (dLoss/dX, dLoss/dV, host [N*3], NULL = zero) of one
 * scene's state; stream-ordered like pbdr_write_tangent. */
int pbdr_write_adjoint(pbdr_ctx *ctx, pbdr_scene scene, const float *xbar, const float *vbar,
                       void *stream);

/* Reads one scene's adjoint into host [N*3] arrays (NULL = skip) and
 * synchronises `stream`.  PBDR_ERR_INVALID before any adjoint exists. */
int pbdr_read_adjoint(pbdr_ctx *ctx, pbdr_scene scene, float *xbar, float *vbar, void *stream);

/* dLoss/dmu of one scene after pbdr_adjoint: the friction terms of every
 * particle's corrections over all substeps and iterations, accumulated per
 * particle on the device (no atomics) and summed here in FP64.  Zero after
 * pbdr_write_adjoint.  Synchronises `stream`. */
int pbdr_read_adjoint_friction(pbdr_ctx *ctx, pbdr_scene scene, double *mubar, void *stream);

/* Launch shapes of the scene-resident kernel for the scene set ids[0..n):
 * out[5k..5k+4] = {particle capacity, scenes, threads per CTA, scratch bits
 * (1: velocities in shared memory, 2: per-particle scratch in shared memory),
 * CTAs} for size class k = 0..3 (capacities 1024, 2048, 4096 and 8192
 * particles; cap >= 20). */
int pbdr_plan_config(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, int32_t *out, int32_t cap);

/* Launch statistics of the last pbdr_step call: the number of kernel
 * launches it issued (graph nodes counted individually). */
int pbdr_last_launch_count(pbdr_ctx *ctx, int64_t *launches);

/* Sum of the neighbour-list lengths of the scenes ids[0..n) from the last
 * neighbour stage (the mean list length kbar = total / particles).
 * Synchronises `stream`. */
int pbdr_neighbor_total(pbdr_ctx *ctx, const pbdr_scene *ids, int32_t n, int64_t *total,
                        void *stream);

/* Stage timing.  While enabled, pbdr_step records CUDA events on its stream
 * around each stage of every substep (no CUDA graph is used).  Stages:
 * 0 wrench, 1 integration + cell keys, 2 radix sort, 3 cell ranges +
 * neighbour lists, 4 solver iterations (all K launches) - the streaming
 * form - and 5 the scene-resident kernels (whole substeps).
 * pbdr_read_profile synchronises, returns the summed milliseconds and launch
 * counts per stage (arrays of `nstages` <= 6 entries) and resets them. */
#define PBDR_NUM_STAGES 6
int pbdr_set_profiling(pbdr_ctx *ctx, int enable);
int pbdr_read_profile(pbdr_ctx *ctx, double *stage_ms, int64_t *stage_launches, int32_t nstages);

/* ---- allocation-free neighbour stage ---------------------------------- */

/* The paper has no counterpart to this call.  It is the neighbour stage of
 * one scene (cell keys, stable sort, bucket ranges, neighbour lists, the same
 * definitions as pbdr_build_neighbors) for callers that must not allocate
 * device memory themselves: a host framework that owns all device memory
 * through its own pool or arena, or a control loop whose latency budget an
 * allocation could break.  It calls no cudaMalloc or cudaFree: its
 * intermediates live in one fixed ~3 MB __device__ array of the library,
 * which every GPU that loads the library holds until the process exits.
 *
 *   pos        [n*3] device, FP32 xyz of the scene's particles (taken as x~)
 *   body       [n] device, body index of every particle
 *   n          0..65536 (larger n: PBDR_ERR_INVALID)
 *   radius     particle radius r > 0 (R_n = 2.2 r)
 *   sorted_key [n] device out: bucket in [0, T), T = smallest power of two >= 2n
 *   sorted_id  [n] device out: particle indices sorted by key, ascending within a key
 *   nbr_cnt    [n] device out: full neighbour count of each particle; a count
 *              above cap means the list was cut to its cap lowest indices
 *   nbr        [cap*n] device out: ascending neighbour indices (the lowest
 *              min(count, cap) of them), column-major (slot j of particle p
 *              at nbr[j*n + p])
 *   cap        1..64
 *   stream     cudaStream_t (NULL = legacy default stream); asynchronous
 *
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents: calls that
 * overlap on the GPU (different streams, or different host threads on one
 * device) race and must be ordered by the caller. */
int pbdr_neighbors_noalloc(const float *pos, const int32_t *body, int32_t n, float radius,
                           uint32_t *sorted_key, uint32_t *sorted_id, int32_t *nbr_cnt,
                           int32_t *nbr, int32_t cap, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PBDR_H */
