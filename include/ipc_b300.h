/*
 * ipc_b300.h -- C-ABI of the batched ABD-IPC step library (sm_103a).
 *
 * One implicit time step of the unified affine-body / soft-body IPC method of
 * Taccel (arXiv 2504.12908), run for many independent environments at once:
 *
 *   (y, x)^{n+1} = argmin  E_IP(x) + E_IP(y) + h^2 B(phi(y); x)         (Eq. unified_ipc,
 *                                                                         Eq. unified_ipc_variational)
 *   subject to the kinematic constraints S^x x = s^x, S^y y = s^y        (Sec. 3.4, Eq. unified_ipc_AL)
 *
 * where E_IP is the backward-Euler incremental potential of App. A.2 with a
 * lumped mass matrix and gravity, the elastic potential is neo-Hookean
 * (App. A.1), affine bodies carry 12 reduced DoFs y = [p, a0, a1, a2] with
 * x_j = p + A xbar_j and M^y = J^T M J (Sec. 3.3) plus a stiff orthogonality
 * potential kappa_s V |A^T A - I|_F^2, and B is the area-weighted IPC log
 * barrier b(d) = -(d - dhat)^2 ln(d / dhat) over point-triangle and edge-edge
 * pairs (App. A.3, Eq. ipc_energy).  The minimiser is projected Newton with
 * block-Jacobi PCG, an additive-CCD filtered backtracking line search and
 * augmented-Lagrangian kinematic targets; all of it runs on the GPU.
 *
 * Conventions
 *   - SI units; every host-side floating-point array is double.
 *   - Vertex arrays are row-major [n][3].  Body states are [n_bodies][12] in
 *     the order y = [p_x, p_y, p_z, A(:,0), A(:,1), A(:,2)] (columns of A).
 *     p is the body's centre of mass; the rest placement is p = com, A = I
 *     (ipc_body_com returns com).
 *   - Gel vertex order is the caller's order everywhere in this API; the
 *     library renumbers internally and maps back.
 *   - "Contact vertex ids" (debug calls): gel vertex i -> i; vertex j of body
 *     b -> n_verts + (sum of body_nv[0..b-1]) + j.
 *
 * Ownership and memory
 *   - The caller owns every host buffer; inputs are copied before the call
 *     returns.
 *   - Device memory: the caller allocates ONE device buffer of the size that
 *     ipc_workspace_bytes reports (e.g. a torch uint8 tensor) and keeps it
 *     alive until ipc_destroy.  The library sub-allocates from it and never
 *     calls cudaMalloc.  It allocates a few KB of pinned host memory at
 *     ipc_create_envs for status read-back.
 *   - The CUDA stream belongs to the caller (cudaStream_t passed as void*;
 *     NULL = legacy default stream).  One ipc_ctx must not be used from two
 *     host threads at once.
 *
 * Errors
 *   Every call returns an ipc_status.  IPC_EINVAL: bad argument or malformed
 *   scene (non-positive tet volume, open body surface, index out of range);
 *   IPC_ENOMEM: workspace too small; IPC_ECUDA: a CUDA runtime error (the
 *   message is in ipc_last_error).  ipc_step also reports a status per env:
 *   IPC_ENOTCONV (Newton, line-search or AL iteration cap hit; the env keeps
 *   its last feasible iterate), IPC_EOVERFLOW (more candidate pairs than the
 *   per-env capacity; the env is left at its state before the step).
 */
#ifndef IPC_B300_H
#define IPC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipc_ctx ipc_ctx;

typedef enum {
  IPC_OK = 0,
  IPC_EINVAL = 1,
  IPC_ENOMEM = 2,
  IPC_ENOTCONV = 3,
  IPC_EINTERSECT = 4,
  IPC_EINVERTED = 5,
  IPC_EOVERFLOW = 6,
  IPC_ECUDA = 7
} ipc_status;

/* Solver parameters (App. A.2-A.3; constants the paper omits are readings
 * documented with the library).  ipc_default_params fills the defaults. */
typedef struct {
  double dt;              /* time step h, s                                  */
  double gravity[3];      /* m/s^2                                           */
  double dhat;            /* barrier activation distance, m                  */
  double kappa;           /* barrier stiffness, Pa                           */
  double newton_tol;      /* stop when |p|_inf / h < newton_tol, m/s         */
  double pcg_rel_tol;     /* PCG stops at |r|_2 <= pcg_rel_tol |b|_2         */
  int newton_max;         /* Newton iteration cap per step                   */
  int pcg_max;            /* PCG iteration cap per Newton iteration          */
  int ls_max;             /* line-search halving cap                         */
  int accd_max;           /* ACCD iteration cap per pair                     */
  double accd_s;          /* ACCD minimum gap fraction (0.1)                 */
  double al_kappa;        /* mass-weighted AL penalty factor (1e6)           */
  int al_max;             /* AL multiplier updates per step                  */
  double ee_mollifier;    /* EE mollifier threshold factor (1e-3)            */
  int precision;          /* 0 = FP64 throughout, 1 = mixed (FP32 element
                             Hessians, assembly and PCG mat-vec; FP64
                             distances, CCD, energies, residuals)            */
  int max_pairs_per_env;  /* candidate-pair capacity per env (0 = default)  */
  double friction_mu;     /* lagged IPC friction coefficient mu (App. A.3,
                             D_k = mu lambda_k f0(|u_k|)); 0 = frictionless  */
  double friction_eps_v;  /* static / dynamic threshold eps_v, m/s (1e-3)   */
  int newton_abs_after;   /* eigenvalue filter of the projected element,
                             pair and body Hessians: Newton iterations 1..n
                             of a step set negative eigenvalues to zero,
                             later ones replace them by their absolute
                             values (default 1000000: always zero; 0:
                             always absolute values)                        */
  int rollout_pcg_window; /* ipc_rollout: PCG iterations per loop iteration
                             (even, >= 2): an env whose solve is longer
                             carries it over while the envs whose solves
                             ended take their Newton steps; 0 (default) =
                             every solve of a Newton iteration ends before
                             the next Newton iteration (not in the paper: a
                             scheduling property of this library)          */
  int pcg_fused;          /* 1 (default): a PCG iteration is one persistent
                             kernel (contact terms, SELL mat-vec and update;
                             an env's update items start when its own
                             products are in, in the order the envs become
                             ready); 2: the same kernel taking the update
                             items in env order (each waits for its env;
                             with more than one iteration per launch both
                             run the multi-iteration kernel, env order);
                             0: three kernels (the mat-vecs, then the
                             update).  With friction the fused kernels take
                             the friction records among an env's products.
                             The same arithmetic in every form.            */
  int pcg_iters_per_launch; /* fused kernel: PCG iterations per launch, 1
                             to 16 (default 8).  Above 1 an env's next
                             products wait only for its own update, so
                             envs do not line up on iteration boundaries
                             (not inside a rollout window, which counts
                             single iterations).  The same arithmetic.   */
} ipc_params;

/* One environment: a tetrahedral gel mesh (one or more pads) and affine bodies. */
typedef struct {
  int n_verts;                 /* gel vertices                               */
  int n_tets;                  /* gel tetrahedra                             */
  const double* rest_x;        /* [n_verts][3] rest positions                */
  const int32_t* tets;         /* [n_tets][4], positive volume required      */
  const int32_t* pad_id;       /* [n_verts] pad (contact object) id, or NULL */
  const uint8_t* pinned;       /* [n_verts] 1 = fixed at its position, NULL  */
  const int32_t* attach_body;  /* [n_verts] body index driving the vertex,
                                  -1 = free; NULL = all free                 */
  double E, nu, rho;           /* neo-Hookean parameters, gel density        */
  int n_bodies;
  const int32_t* body_nv;      /* [n_bodies] vertex counts                   */
  const double* body_rest_x;   /* [sum nv][3] rest placement (world)         */
  const int32_t* body_nt;      /* [n_bodies] triangle counts                 */
  const int32_t* body_tris;    /* [sum nt][3] local vertex ids, closed and
                                  outward oriented                           */
  const double* body_rho;      /* [n_bodies] density                         */
  const double* body_kappa_s;  /* [n_bodies] orthogonality stiffness, Pa     */
  const uint8_t* body_driven;  /* [n_bodies] 1 = follows ipc_set_targets     */
  const uint8_t* pad_self_contact; /* [n_pads] (n_pads = 1 + max pad_id): 1 =
                                  the pad's own primitives that share no
                                  vertex pair up too (gel self-contact, the
                                  soft-soft contact of the soft-block
                                  pressing comparison, Fig. sim-compare b);
                                  NULL = no pad self-contacts.  Candidate
                                  search within such a pad is quadratic in
                                  its surface size.                          */
} ipc_scene_desc;

typedef struct {
  int newton_iters;     /* max over the stepped envs                         */
  int pcg_iters;        /* total PCG iterations (batched, all Newton its)     */
  int ls_trials;        /* total line-search energy evaluations              */
  int al_updates;       /* max over envs                                     */
  int max_pairs;        /* max candidate pairs seen in one env               */
  long long newton_env_iters; /* Newton iterations summed over the stepped envs */
  long long al_env_updates;   /* AL multiplier updates summed over the envs    */
  long long ccd_limited;      /* line searches that started below alpha = 1    */
  double alpha_sum;           /* accepted line-search steps, summed            */
  long long accd_iters;       /* ACCD advancement iterations, all pairs        */
  int accd_iters_max;         /* most ACCD iterations taken by one pair        */
  double ms_total;      /* wall time of the call (host clock), ms            */
  long long pair_evals;       /* static candidate pairs evaluated (barrier terms),
                                 summed over Newton iterations and envs      */
  long long swept_pairs;      /* swept candidate pairs of the line searches
                                 (ACCD and line-search energies), summed     */
  long long loop_iters;       /* device loop iterations of the call's graph:
                                 Newton loop (ipc_step) or rollout loop; 0
                                 for host-driven calls                     */
  long long pcg_launches;     /* PCG kernel launches the graph ran (each
                                 runs pcg_iters_per_launch iterations of
                                 every env in PCG at the time, one inside
                                 a rollout window); 0 for host-driven
                                 calls                                     */
  long long act_pair_iters;   /* active contact pairs x PCG iterations,
                                 summed over the solves and envs (the work
                                 of the contact mat-vec)                   */
} ipc_step_stats;

void ipc_default_params(ipc_params* prm);

/* Bytes of device workspace needed for n_envs scenes (array of n_envs
 * descriptors, one per env; they may differ in size). */
ipc_status ipc_workspace_bytes(const ipc_scene_desc* scenes, int n_envs,
                               const ipc_params* prm, size_t* bytes);

/* Build the envs: validates and preprocesses each scene on the host, copies
 * it into dev_workspace (ws_bytes >= ipc_workspace_bytes), sets every env to
 * its rest state (velocities zero, bodies at p = com, A = I; Sec. 4.1
 * "Robot Actions") and driven targets to the rest placement. */
ipc_status ipc_create_envs(const ipc_scene_desc* scenes, int n_envs,
                           const ipc_params* prm, void* dev_workspace,
                           size_t ws_bytes, void* cuda_stream, ipc_ctx** out);

ipc_status ipc_destroy(ipc_ctx* ctx);

/* Last error message of this ctx (empty string if none). */
const char* ipc_last_error(const ipc_ctx* ctx);

/* CUDA-graph execution (a property of this library; results are the same
 * as with plain launches):
 *   mode 0 (default): kernel by kernel; the host polls the device's loop
 *     state (PCG every 16 iterations, Newton and line search every
 *     iteration).
 *   mode 1: each PCG solve (the block-Jacobi PCG of every Newton iteration,
 *     named as the method's main cost in the paper's Limitations) is one
 *     graph: a work-list kernel, then a WHILE node over one launch of the
 *     PCG kernel (pcg_iters_per_launch iterations) whose condition its
 *     last CTA sets on the device.
 *   mode 2: the whole step is one graph: nested WHILE / IF nodes for the
 *     Newton loop, the PCG solve, the line-search gate and the line-search
 *     trials, all conditions set on the device and every loop bounded by
 *     its cap (newton_max, pcg_max, ls_max); ipc_step then needs no host
 *     round trip (see ipc_step).
 * Graphs are captured on the ctx stream at their first use and replayed
 * after that; ipc_autotune and a mode change drop them.  The ctx stream must
 * support capture (a created stream, not the legacy default stream);
 * otherwise ipc_step returns IPC_ECUDA with the reason in ipc_last_error.
 * While per-kernel profiling is on, plain launches are used so that every
 * kernel is timed.  IPC_EINVAL for another mode. */
ipc_status ipc_set_graph_mode(ipc_ctx* ctx, int mode);

/* Launch shapes chosen by ipc_autotune and the timings behind the choice. */
typedef struct {
  int spmv_unroll;        /* SELL slots in flight per lane in the PCG mat-vec: 2, 4 or 8 */
  int pcg_ctas_per_sm;    /* persistent PCG grid: CTAs per SM (x SM count)            */
  float spmv_us[3];       /* mat-vec time per launch for 2, 4, 8 slots, us (mean of a
                             launch over every env and one over every 4th env)     */
  int grid_ctas_per_sm[3];/* grid candidates: half, all and twice the resident CTAs   */
  float grid_us[3];       /* mean mat-vec time per launch for those grids, us          */
  int assemble_block;     /* threads per CTA of the gather assembly: 64, 128 or 256    */
  float assemble_us[3];   /* mean assembly time per launch for 64, 128, 256, us        */
  int pairs_ctas_per_sm;  /* broad phase: CTAs per SM of the candidate-pair search     */
  float pairs_us[3];      /* mean broad-phase time per search for 4, 8, 16 CTAs / SM   */
  int pcg_iter_bound;     /* single-iteration fused PCG kernel (one iteration per
                             launch: inside rollout windows): register bound on (1)
                             or off                                                  */
  float pcg_iter_us[2];   /* mean time per fused iteration with the bound on, off, us
                             (0 when the fused kernel is not in use: pcg_fused = 0
                             or friction on)                                        */
} ipc_tuning;

/* Choose launch shapes by timing `reps` launches of each candidate on this
 * ctx's current state (call it after at least one ipc_step, between steps):
 * the PCG mat-vec's SELL slots in flight per lane and the persistent PCG
 * grid (each on a batch of every env and one of every 4th env: the mean),
 * the fused PCG iteration kernel's register bound (PCG iterations from a
 * fresh start on the last system, every env and every 4th env), the
 * gather assembly's CTA size and the candidate-pair search's grid
 * (every env).  A candidate replaces the default shape
 * only when it is more than 5% faster.  It touches only scratch that the
 * next Newton iteration rebuilds (PCG scratch, the SELL values from the
 * stored element blocks, the candidate pair lists) and clears the contact
 * accumulator afterwards, so later steps give the same results as before
 * apart from the launch shapes.  Captured graphs are dropped and
 * re-captured at their next use.  Not in the paper: a property of this
 * library.  `out` may be NULL. */
ipc_status ipc_autotune(ipc_ctx* ctx, int reps, ipc_tuning* out);

int ipc_num_envs(const ipc_ctx* ctx);

/* Bounds-checked builds (libipc_b300_checks.so, compiled with -DIPC_CHECKS):
 * the kernels test the indices they gather through (SELL columns, tet
 * vertices, pair and active-pair vertices and slots, PCG work items,
 * assembly sources) and, on a violation, skip the access and record the
 * first violation's code (1 SELL column, 2 tet vertex, 3 pair vertex, 4 PCG
 * item, 5 active-pair slot or vertex, 6 assembly source) and index.
 * *checks_built = 1 in such a build (0 otherwise, where *code stays 0);
 * *code = 0 when nothing was recorded since the context was created.
 * Synchronises the ctx stream.  Any pointer may be NULL.  A debugging aid of
 * this library (no counterpart in the paper). */
ipc_status ipc_check_report(ipc_ctx* ctx, int* checks_built, int* code, long long* index);
ipc_status ipc_env_sizes(const ipc_ctx* ctx, int env, int* n_verts, int* n_bodies,
                         int* n_surface_out);

/* Rest centre of mass of a body (the p of its rest placement). */
ipc_status ipc_body_com(const ipc_ctx* ctx, int env, int body, double com[3]);

/* State of one env.  x, v: [n_verts][3]; y, ydot: [n_bodies][12].  Any
 * pointer may be NULL to leave that part unchanged.  set_state synchronises
 * the stream and rejects non-finite values (IPC_EINVAL), inverted tets
 * (IPC_EINVERTED) and touching or interpenetrating surfaces (IPC_EINTERSECT:
 * a candidate pair at distance <= 0, or an edge of one contact object
 * passing through a triangle of another), leaving the previous state in
 * place (Sec. 1: the simulator keeps every state intersection-free).
 * A state read with get_state and set again (in this or another ctx built
 * from the same scene) continues as the original would (checkpoint /
 * resume). */
ipc_status ipc_set_state(ipc_ctx* ctx, int env, const double* x, const double* v,
                         const double* y, const double* ydot);
ipc_status ipc_get_state(ipc_ctx* ctx, int env, double* x, double* v,
                         double* y, double* ydot);

/* Replace env `env` by a new scene of the same topology (equal mesh sizes
 * and connectivity, pinned / attached / driven sets and body vertex counts;
 * material, rest geometry, body shapes and masses may differ) and set it to
 * that scene's rest state with zero velocities (as ipc_create_envs does).
 * This lets a caller reuse an env slot of a resident context for a new
 * request (continuous batching) without creating a context.  Copies only
 * the env's own value tables; synchronises the ctx stream.  IPC_EINVAL
 * (message in ipc_last_error) when the topology differs or the scene is
 * invalid.  Not in the paper: a property of this library. */
ipc_status ipc_reset_env(ipc_ctx* ctx, int env, const ipc_scene_desc* scene);

/* Kinematic targets s^y of the driven bodies of one env for the next step,
 * [n_bodies][12] (rows of free bodies are ignored).  Gel vertices attached
 * to a driven body get the target p + A xbar (xbar = rest offset from the
 * body's com).  Sec. 3.4 / 4.1. */
ipc_status ipc_set_targets(ipc_ctx* ctx, int env, const double* y_target);

/* Same for all envs at once from one host array [n_envs][max_bodies][12]
 * (max_bodies = largest n_bodies over the envs): one host->device copy into
 * a staging buffer, scattered on the device. */
ipc_status ipc_set_targets_all(ipc_ctx* ctx, const double* y_targets);

/* Same as ipc_set_targets_all but from a device buffer (device-to-device
 * copy on the ctx stream; no host synchronisation). */
ipc_status ipc_set_targets_all_device(ipc_ctx* ctx, const double* dev_y_targets);

/* Advance the listed envs by one time step (env_ids NULL = all envs; the
 * argmin of Eq. unified_ipc_variational by projected Newton, App. A.2).
 * per_env_status (may be NULL) receives n statuses, stats the counters.
 * With either of them non-NULL the call synchronises the stream and fills
 * them.  With both NULL in graph mode 2 (ipc_set_graph_mode) the call only
 * enqueues the step's graph on the ctx stream and returns: the step runs
 * on the device without host round trips, and ipc_step_results reads its
 * results later.  Other modes synchronise inside the Newton loop. */
ipc_status ipc_step(ipc_ctx* ctx, const int32_t* env_ids, int n,
                    int32_t* per_env_status, ipc_step_stats* stats);

/* Results of the last ipc_step (the statuses of its envs, in its order,
 * and its counters): synchronises the ctx stream.  Either pointer may be
 * NULL.  A second call after the results were read returns zeroed stats
 * and leaves per_env_status untouched. */
ipc_status ipc_step_results(ipc_ctx* ctx, int32_t* per_env_status, ipc_step_stats* stats);

/* n_steps time steps of each listed env (env_ids NULL = all envs) in one
 * call, each env on its own schedule: the same per-step computation as
 * n_steps calls of ipc_step (App. A.2), but an env whose step converges
 * begins its next step while the slower envs of the batch are still
 * iterating, so a few hard steps no longer hold the whole batch.  Targets
 * of step k of env e come from dev_targets[k][e][max_bodies][12] (device
 * memory, all envs of the context, layout of ipc_set_targets_all; caller
 * owned, read during the rollout, may be NULL without driven bodies).
 * steps_per_env (host, n entries in env_ids' order, or NULL): env i runs
 * min(steps_per_env[i], n_steps) steps (IPC_EINVAL if negative).  An
 * env whose step fails (any status but IPC_OK) stops after that step: its
 * state is what ipc_step would have left.
 *   per_env_status: n statuses (the failing step's, else IPC_OK);
 *   per_env_steps: n counts of the steps taken (n_steps unless one failed);
 *   stats: the counters summed over the rollout's steps (newton_iters,
 *   al_updates, max_pairs, accd_iters_max: maxima over env-steps).
 * With all three NULL the call only enqueues the rollout (one CUDA graph,
 * captured at the first call; no host round trip) on the ctx stream and
 * returns; ipc_rollout_results reads the results.  With profiling on
 * (ipc_profile_enable) the same loop runs as plain launches driven from
 * the host.  Not in the paper: a batching property of this library; the
 * caller gives up per-step host control (targets are fixed in advance). */
ipc_status ipc_rollout(ipc_ctx* ctx, const int32_t* env_ids, int n, int n_steps, const int32_t* steps_per_env,
                       const double* dev_targets, int32_t* per_env_status, int32_t* per_env_steps,
                       ipc_step_stats* stats);

/* Results of the last ipc_rollout (synchronises the ctx stream); any
 * pointer may be NULL. */
ipc_status ipc_rollout_results(ipc_ctx* ctx, int32_t* per_env_status, int32_t* per_env_steps,
                               ipc_step_stats* stats);

/* Per-env counters of the last ipc_step that included `env` (host only; the
 * values were read back at the end of that step).  out[IPC_ENV_STATS]:
 *   0 status, 1 Newton iterations, 2 AL multiplier updates, 3 PCG
 *   iterations (all Newton iterations), 4 line-search energy trials,
 *   5 line searches that started below alpha = 1 (CCD-limited), 6 most ACCD
 *   iterations one pair took, 7 candidate pairs in the last list,
 *   8 ACCD iterations over all pairs, 9 static candidate pairs evaluated
 *   (all Newton iterations), 10 swept candidate pairs (all line searches).
 * Diagnostics of this library (the paper reports no iteration counts). */
#define IPC_ENV_STATS 11
ipc_status ipc_env_stats(const ipc_ctx* ctx, int env, int32_t* out);

/* Coated-surface vertex positions of one env's gel (Sec. 4.1: the surface
 * minus pinned and attached vertices), in increasing gel vertex id order.
 * Writes min(capacity, count) rows of [3]; *n_written = count. */
ipc_status ipc_read_gel_surface(ipc_ctx* ctx, int env, double* out_xyz, int capacity,
                                int* n_written);

/* Coated-surface positions of all envs into one host array, env after env
 * (counts from ipc_env_sizes): gathered on the device, one device->host
 * copy, synchronises the stream. */
ipc_status ipc_read_gel_surface_all(ipc_ctx* ctx, double* out_xyz, size_t capacity_rows,
                                    size_t* rows_written);

/* Same result as ipc_read_gel_surface_all, for callers that cannot allocate
 * device memory when they read results back (a restricted allocator, or a
 * workspace sized without spare room): the device gather is staged through a
 * fixed array of 262144 rows (6 MiB) compiled into the library, which every
 * GPU that loads the library keeps until the process exits.  This is a
 * property of this library; the paper has no counterpart.
 *   - Calls no cudaMalloc / cudaFree; needs no workspace scratch.
 *   - Returns IPC_EINVAL (message in ipc_last_error) when the envs hold more
 *     than 262144 coated-surface rows in total.
 *   - The context's device must be the current device (IPC_EINVAL
 *     otherwise); devices 0..63 are supported.  The first call on a device
 *     looks up the array's device address (cudaGetSymbolAddress) with that
 *     device current; make that first call before any stream capture.
 *   - Every call shares the array: calls that overlap on the GPU (several host
 *     threads or streams) race on it and must be serialised by the caller.
 * Synchronises the ctx stream. */
ipc_status ipc_read_gel_surface_all_noalloc(ipc_ctx* ctx, double* out_xyz, size_t capacity_rows,
                                            size_t* rows_written);

/* ---- tactile outputs (Sec. 4.2) ------------------------------------------
 * Read off the deformed coated surface after a step.  The paper gives no
 * sensor model; the library uses an orthographic sensor on one gel pad:
 * origin on the pad's rest contact face (a corner of the image), unit
 * in-plane axes u and v, unit normal pointing out of the coated face, pixel
 * (r, c) centred at origin + (c + 1/2) pitch u + (r + 1/2) pitch v.  It looks
 * through the gel along +normal: each pixel shows the front-face triangle
 * (a coated boundary triangle of that pad whose rest outward normal has a
 * normal-component above 1/2) with the smallest height h = (x - origin).normal
 * at the pixel centre.  depth = -h (0 at rest, positive where pressed in),
 * linearly interpolated over the triangle; normal = the triangle's deformed
 * outward unit normal; pixels nothing covers: hit 0, depth 0, normal 0. */
typedef struct {
  int env;                /* env index                                       */
  int pad;                /* gel pad id (pad_id of its vertices; 0 if none)  */
  double origin[3];       /* corner of the image on the rest contact face, m  */
  double axis_u[3];       /* unit, along image columns                       */
  double axis_v[3];       /* unit, along image rows                          */
  double normal[3];       /* unit, out of the coated face                    */
  double pitch;           /* pixel size, m                                   */
} ipc_sensor;

/* Global rows of gel vertices (user vertex ids of one env) for the device
 * calls below.  Host only.  IPC_EINVAL for an id outside the env. */
ipc_status ipc_gel_vertex_rows(const ipc_ctx* ctx, int env, int n, const int32_t* verts, int32_t* rows_out);

/* Front-face triangles of a sensor as global row triples [n][3] (host only,
 * from the rest mesh; call once per sensor).  rows_out may be NULL to count;
 * *n_out receives the count; IPC_EOVERFLOW if it exceeds capacity. */
ipc_status ipc_sensor_triangles(const ipc_ctx* ctx, const ipc_sensor* sensor, int32_t* rows_out, int capacity,
                                int* n_out);

/* Depth / normal / hit maps of n_sensors sensors, all height x width, from
 * the ctx's current positions, on the ctx stream (asynchronous).  Device
 * buffers, caller-owned: frames [n_sensors][13] (origin, axis_u, axis_v,
 * normal, pitch), tri_off [n_sensors + 1] (prefix offsets into tri_rows),
 * tri_rows [n_tri_total][3] (from ipc_sensor_triangles), keys scratch
 * [n_sensors][height][width] (uint64), depth [n_sensors][height][width]
 * (double), normal [..][3] (double, may be NULL), hit (uint8, may be NULL).
 * A pixel's winner is the smallest (FP32 height, triangle index) key, so the
 * result does not depend on thread order; depth and normal are FP64. */
ipc_status ipc_tactile_maps_device(ipc_ctx* ctx, int n_sensors, int height, int width, const double* frames,
                                   const int32_t* tri_off, const int32_t* tri_rows, int n_tri_total,
                                   unsigned long long* keys, double* depth, double* normal, uint8_t* hit);

/* Marker positions p = sum_u alpha_u x_u and flows p - rest (Sec. 4.2,
 * Markers) for n markers on coated triangles, from the ctx's current
 * positions, on the ctx stream.  Device buffers: rows [n][3] global rows
 * (ipc_gel_vertex_rows), bary [n][3], rest [n][3] (may be NULL), pos [n][3],
 * flow [n][3] (may be NULL; needs rest). */
ipc_status ipc_markers_device(ipc_ctx* ctx, int n, const int32_t* rows, const double* bary, const double* rest,
                              double* pos, double* flow);

/* ---- diagnostics (used by the parity tests; not needed to step) -------- */

/* Objective, gradient and Hessian-vector product of one env at its current
 * state, as the first Newton iteration of a step would see it (xtilde =
 * x + h v, targets as set, multipliers zero).  grad/vec/hvec are full DoF
 * vectors [3 n_verts + 12 n_bodies] in caller vertex order; the Hessian is
 * the PSD-projected one with pinned DoFs eliminated (identity rows).  Any
 * output may be NULL. */
ipc_status ipc_debug_eval(ipc_ctx* ctx, int env, double* energy, double* grad,
                          const double* vec, double* hvec);

/* Candidate pairs of one env for caller-given contact-vertex positions
 * cv_x [n_verts + sum body_nv][3] (indexed by contact vertex id; only
 * surface vertices are read): static set (cv_x_end NULL) or swept set from
 * cv_x to cv_x_end.  Rows of out: [kind (0 = PT, 1 = EE), v0, v1, v2, v3]
 * with contact vertex ids (PT: point, triangle; EE: edge of the lower
 * object, edge of the higher).  Order is unspecified.  *n_pairs = count
 * (IPC_EOVERFLOW if above the env's pair capacity). */
ipc_status ipc_debug_pairs(ipc_ctx* ctx, int env, const double* cv_x, const double* cv_x_end,
                           int32_t* out, int capacity, int* n_pairs);

/* First Newton direction of one env from its current state (PCG solve). */
ipc_status ipc_debug_newton_dir(ipc_ctx* ctx, int env, double* p, int* pcg_iters);

/* Failure path of the multi-iteration PCG kernel's bounded waits: assembles
 * env's system from its current state, starts its PCG solve, sets its
 * count of completed update rounds to -1 (so its first products wait for a
 * round that nothing completes) and runs one launch of the kernel.  The
 * waits give up after about a second; the kernel ends the env's step with
 * IPC_ECUDA (*env_status) and resets its counters, and the context stays
 * usable (set_state, then step, as after any failed step).  *ms: the
 * launch's device time.  Synchronises.  IPC_EINVAL when the context does
 * not run the multi-iteration kernel (pcg_fused 0 or pcg_iters_per_launch
 * 1).  A test aid of this library (no counterpart in the paper). */
ipc_status ipc_debug_pcg_wait_out(ipc_ctx* ctx, int env, int* env_status, float* ms);

/* Largest CCD-safe step along dir (ACCD over the swept candidates). */
ipc_status ipc_debug_accd(ipc_ctx* ctx, int env, const double* dir, double* alpha);

/* ---- profiling ---------------------------------------------------------- */
/* Kernel launches are always counted.  With profiling on, every kernel
 * launch of ipc_step is bracketed by CUDA events recorded on the ctx stream
 * and its device time is accumulated per kernel class.  Off by default. */
ipc_status ipc_profile_enable(ipc_ctx* ctx, int on);
ipc_status ipc_profile_reset(ipc_ctx* ctx);
int ipc_profile_count(const ipc_ctx* ctx);  /* number of kernel classes */
/* Class i: its name (static string), launches and accumulated device ms
 * since the last reset (profiling on). */
ipc_status ipc_profile_get(const ipc_ctx* ctx, int i, const char** name, long long* launches, double* ms);
/* Kernels launched through this ctx since creation. */
long long ipc_launch_count(const ipc_ctx* ctx);
/* Sizes of the assembled system of one env: real 3x3 blocks of the sparse
 * matrix (gel and body), stored SELL blocks (with padding), rows, tets. */
ipc_status ipc_system_sizes(const ipc_ctx* ctx, int env, long long* real_blocks, long long* stored_blocks,
                            int* rows, int* tets);

/* FP64 and FP32 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA), each timed with CUDA events over one launch of
 * independent FMA chains on every SM, on `stream` (synchronises it).
 * scratch: device memory of at least SM count x 8 x 256 doubles (written).
 * The denominators of the ALU rooflines of the FP64-bound kernels; touches
 * no clock or power setting.  A property of this library, not the paper. */
ipc_status ipc_fma_peaks(void* scratch, size_t scratch_bytes, double* fp64_tflops, double* fp32_tflops,
                         void* stream);

/* ---- element kernels on caller device buffers (no ctx) ----------------- */
/* All pointers are device pointers; n elements; the call is asynchronous on
 * stream.  Returns IPC_EINVAL for n < 0 or NULL required pointers. */

/* Neo-Hookean tet (App. A.1): x [n][4][3], Dm_inv [n][3][3] (row-major),
 * vol [n]; outputs (NULL to skip) energy [n] = vol Psi (+inf if J <= 0),
 * grad [n][12], hess [n][12][12] = vol B^T Pi(dP/dF) B: project = 1: Pi
 * sets the negative eigenvalues of d2Psi/dF2 to zero, project = 2: Pi
 * replaces them by their absolute values, project = 0: the exact Hessian. */
ipc_status ipc_k_tet(int n, const double* x, const double* Dm_inv, const double* vol,
                     double mu, double lam, double* energy, double* grad, double* hess,
                     int project, void* stream);

/* Weighted barrier of pairs (App. A.3): X [n][4][3], is_ee [n] (0/1),
 * weight [n] (multiplies c(x) b(d)), eps_x [n] (mollifier threshold, EE
 * only); energy [n], grad [n][12], hess [n][12][12] (project = 1: negative
 * eigenvalues set to zero, 2: replaced by their absolute values, 0: the
 * exact Hessian).  project | 8: the Hessian is formed and projected in FP32
 * from the FP64 per-pair factors, as the mixed-precision step does, and
 * written widened to FP64; energy and gradient stay FP64. */
ipc_status ipc_k_barrier(int n, const double* X, const int32_t* is_ee, const double* weight,
                         const double* eps_x, double dhat, double* energy, double* grad,
                         double* hess, int project, void* stream);

/* ACCD time of impact of pairs moving from X0 by P: toi [n] in (0, 1];
 * iters [n] (may be NULL) receives the advancement iterations of each pair. */
ipc_status ipc_k_accd(int n, const double* X0, const double* P, const int32_t* is_ee,
                      double s, int max_iter, double* toi, int32_t* iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IPC_B300_H */
