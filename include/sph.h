/*
 * sph.h -- C ABI of the GB300 (sm_103a) WCSPH(-RANS) time step with the
 * improved bidirectional buffer (Wang & Hu, arXiv 2510.25702).
 *
 * One call of sph_step advances every instance by whole advection steps:
 * cell-linked-list rebuild (Sec. 2.4.1, 2.4.3), region-constrained buffer
 * labelling (Sec. 3.2), dual-criteria time step (Sec. 2.3), kernel
 * correction matrix with the mirror condition (Sec. 2.2, 3.3), ARD viscosity
 * and k-epsilon sweeps (Sec. 2.1, 2.2), acoustic sub-steps with the RKGC
 * momentum sweep, the compensated open-boundary pressure term (Sec. 3.3,
 * final Eq.) and the Riemann continuity sweep (Sec. 2.2), buffer boundary
 * values (Sec. 2.4.2, buffer table of Sec. 4.3), and the buffer update:
 * injection across the generation line (Sec. 2.4.2, 3.1), ID-checked
 * deletion (Sec. 2.4.3, 3.2) and stable compaction with appended copies
 * (Sec. 2.4.2).
 *
 * Conventions
 *  - Every function returns int: 0 (SPH_OK) or a negative SPH_ERR_* code;
 *    nothing throws across this boundary.  sph_error_string() names codes.
 *  - Vectors are [n][3] row-major doubles (z = 0 in 2D); matrices [n][9].
 *  - The library owns all device state.  The caller owns every array it
 *    passes; arrays are copied in (sph_create, sph_write_fields) or out
 *    (sph_read_fields) before the call returns.
 *  - Work is ordered on the context's CUDA stream (sph_alloc.stream, or the
 *    legacy default stream when NULL).  sph_step does not synchronise with
 *    the host except for reading its 4-byte status word at the end;
 *    sph_step_async and sph_set_profile do not wait at all;
 *    sph_read_fields, sph_write_fields and sph_get_stats synchronise.
 *  - Rows read or written by sph_read_fields / sph_write_fields are ordered
 *    by (instance, uid).
 *  - A context is used from one host thread at a time.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_ABI_VERSION 3

/* return codes */
#define SPH_OK 0
#define SPH_ERR_ARG -1       /* invalid argument (message via sph_last_error) */
#define SPH_ERR_CUDA -2      /* a CUDA call failed */
#define SPH_ERR_CAPACITY -3  /* particle capacity exceeded (buffer update not committed), or a
                                particle has more neighbours than its list holds (2.5 x the
                                full-support count; the surplus is dropped from that step) */
#define SPH_ERR_NONFINITE -4 /* a density or velocity became NaN/Inf */
#define SPH_ERR_TIMEOUT -5   /* a bounded device wait ran out */
#define SPH_ERR_OVERLAP -6   /* buffer boxes of one instance intersect */
#define SPH_ERR_STATE -7     /* call not valid in the context's state */
#define SPH_ERR_ALLOC -8     /* device allocation failed */

/* sph_config.precision: arithmetic of the pair sweeps.  Positions,
   velocities, densities, the time integration, the B inversion and the
   time-step reductions are FP64 in both modes. */
#define SPH_PREC_FP64 0
#define SPH_PREC_FP32 1 /* FP32 pair sweeps with FP32 accumulation */

/* sph_config.dt_mode (Sec. 2.3 dual-criteria time stepping) */
#define SPH_DT_DUAL 0   /* advection step + n = ceil(dt_ad/dt_ac) equal sub-steps */
#define SPH_DT_SINGLE 1 /* one sub-step of min(dt_ad, dt_ac) per step */
#define SPH_DT_FIXED 2  /* dt_ad_fixed split into n_ac_fixed sub-steps */

/* buffer types (Sec. 2.4.2; buffer table of Sec. 4.3) */
#define SPH_BUF_VELOCITY 0 /* prescribed velocity, pressure extrapolated */
#define SPH_BUF_PRESSURE 1 /* prescribed pressure p_ob, velocity extrapolated */
#define SPH_TURB_ZERO_GRADIENT 0
#define SPH_TURB_FREESTREAM 1

#define SPH_MAX_THETA 64
#define SPH_MAX_BUFFERS 16 /* per instance */

/* One instance (an independent problem).  h is the smoothing length
   (1.3 dp in the paper, Sec. 2.2); the cell grid covers [domain_lo,
   domain_hi) with cells of 2h (points outside are clamped to the edge
   cells); periodic axes wrap with length domain_hi - domain_lo and need at
   least 3 cells. */
typedef struct sph_config {
  int32_t dim;        /* 2 or 3 */
  int32_t rans;       /* 0 laminar, 1 k-epsilon RANS */
  int32_t precision;  /* SPH_PREC_* */
  int32_t dt_mode;    /* SPH_DT_* */
  int32_t n_ac_fixed; /* sub-steps in SPH_DT_FIXED */
  int32_t kinematic;  /* 1: no physics, only the topology and buffer stages
                         (positions are set by the caller) */
  int32_t periodic[3];
  uint32_t seed;      /* Philox4x32-10 key word 0 of the inlet fluctuation */
  double dp, h, rho0, c0, nu_l;
  double eta;         /* ARD limiter (3 in the paper) */
  double U_ref;       /* reference speed of the advection criterion */
  double dt_ad_fixed;
  double gravity[3];
  double domain_lo[3], domain_hi[3];
  int32_t obc;        /* SPH_OBC_*: open-boundary treatment (0 = the paper's) */
  int32_t density_sum; /* 1: density of fluid particles re-evaluated once per
                          advection step by kernel summation (below) */
  double tvf_alpha;   /* transport-velocity correction (below); 0 = off */
  int32_t wall_function; /* 1: step-wise wall function at the walls (RANS
                            instances; below) */
  int32_t tvf_pbuf;   /* 1: the transport-velocity correction also moves the
                         particles of pressure buffers, across the buffer
                         axis only (below); 0 = fluid particles only */
} sph_config;

/* The two stages of the advection step that Sec. 2.3 names through the
   schemes it cites (without formulas), both switched per instance and both
   taken over the frozen configuration of the step, for fluid particles
   (label 0; the first with tvf_pbuf also for pressure-buffer particles),
   after the correction matrix, viscous and k-epsilon terms
   (which use the volumes m / rho from before them):
   - transport-velocity correction: x_i += -2 tvf_alpha h^2 sum_j V_j grad_i W_ij
     over real and wall neighbours (the background-pressure term of the
     transport-velocity formulation, with the background pressure tied to
     the step so that the shift is a fixed fraction of h^2); with tvf_pbuf
     also for particles labelled in a pressure buffer, whose motion no
     boundary value prescribes, minus its component along the buffer axis
     n_b (their support is cut at the open face, so the sum points into the
     fluid): the shift then only spreads them across the buffer, and the
     flux through the face stays the momentum equation's;
   - density reinitialisation: rho_i = rho0 sigma_i / sigma_0 with
     sigma_i = W(0) + sum_j W_ij over real and wall neighbours and sigma_0
     the same sum on the perfect lattice of spacing dp.  The summed
     density follows the particle spacing, so a lattice at dp carries zero
     pressure: buffers that impose a background pressure on such an
     instance start it out of balance (give its outlet zero pressure).
   The acoustic sub-steps start from the reinitialised density.
   Step-wise wall function (Sec. 2.3 uses the one of its reference at
   turbulent walls; the standard two-layer wall law): a fluid particle of a
   RANS instance lying y < dp from the wall surface (y = distance to its
   nearest wall dummy - dp/2) takes the friction velocity u_tau of the law
   u_t = u_tau^2 y / nu_l (y+ <= 11.225) or u_t = (u_tau / 0.4187)
   ln(9.793 y u_tau / nu_l), u_t its speed along the wall relative to that
   dummy (the wall normal from its wall kernel-gradient sum); its wall pairs
   carry the viscosity u_tau^2 y / u_t (wall stress rho0 u_tau^2), its k
   production is u_tau^3 / (0.4187 y) (0 in the sublayer) and after the
   k-eps update eps takes the wall value C_mu^(3/4) k^(3/2) / (0.4187 y)
   (2 nu_l k / y^2 in the sublayer).
   Differentiated windows need all three off. */

/* sph_config.obc: the open-boundary treatments compared in Sec. 4.1 (Table
   of the four cases), for ablation.  IMPROVED (case 4, default): B_i with
   the mirror support at pressure-buffer particles, B^_j = B_i at buffer
   neighbours, compensation (2 p_ob / rho_i) B_i sum_j V_j grad W (final Eq.
   of Sec. 3.3).  VIPO (case 1): no kernel correction (B = I).  VIPO_RKGC
   (case 2): B from the truncated support, own B_j at buffer neighbours,
   compensation without B_i.  VIPO_RKGC_MIRROR (case 3): as IMPROVED but the
   compensation without B_i.  MINIMAL_MIRROR: as IMPROVED but B_i from the
   truncated support (the literal reading of B_k = B_i alone).  Adjoint
   windows take IMPROVED only. */
#define SPH_OBC_IMPROVED 0
#define SPH_OBC_VIPO 1
#define SPH_OBC_VIPO_RKGC 2
#define SPH_OBC_VIPO_RKGC_MIRROR 3
#define SPH_OBC_MINIMAL_MIRROR 4

/* Initial particles of one instance.  Pointers are host memory when
   on_device == 0, device memory of the context's GPU when 1.  k, eps, uid
   and wall_vel may be NULL (zeros; uid = 0..n-1). */
typedef struct sph_particles {
  int64_t n;        /* real (fluid + buffer) particles */
  int64_t nw;       /* wall dummies (fixed positions, volume dp^dim) */
  int64_t capacity; /* real-particle capacity of this instance, >= n */
  int32_t on_device;
  int32_t reserved;
  const double *pos;      /* [n][3] */
  const double *vel;      /* [n][3] */
  const double *rho;      /* [n] */
  const double *mass;     /* [n] */
  const double *k;        /* [n] turbulent kinetic energy (RANS) */
  const double *eps;      /* [n] dissipation rate (RANS) */
  const uint32_t *uid;    /* [n] */
  const double *wall_pos; /* [nw][3] */
  const double *wall_vel; /* [nw][3] prescribed wall velocity */
} sph_particles;

/* One bidirectional buffer (Sec. 2.4.1): the aligned box
   0 <= x'_0 < length, |x'_1| <= half[0], |x'_2| <= half[1] in the frame
   x' = F (x - origin), whose rows are n_b (pointing from the open face into
   the domain), t1, t2.  Velocity buffers impose U(s) n_b with U linearly
   interpolated in theta[0..n_theta) across s = x'_1 in [-half[0], half[0]]
   and a Philox relative fluctuation of amplitude noise; pressure buffers
   impose p_ob.  Freestream turbulence sets (k_in, eps_in). */
typedef struct sph_buffer_desc {
  int32_t type;    /* SPH_BUF_* */
  int32_t turb_bc; /* SPH_TURB_* */
  int32_t n_theta; /* 1..SPH_MAX_THETA */
  int32_t reserved;
  double origin[3];
  double frame[9];
  double length;
  double half[2];
  double p_ob;
  double noise;
  double k_in, eps_in;
  double theta[SPH_MAX_THETA];
} sph_buffer_desc;

/* Optional device allocator (e.g. a caching allocator); NULL functions mean
   cudaMalloc / cudaFree.  stream is a cudaStream_t (NULL = legacy stream).
   Every block returned must start on a 256-byte boundary (as cudaMalloc's
   do): the sweeps read 32-byte records with single 256-bit loads.  A block
   that does not is handed back to free and the call fails with
   SPH_ERR_ALLOC. */
typedef struct sph_alloc {
  void *(*alloc)(void *user, size_t bytes, void *stream);
  void (*free)(void *user, void *ptr, void *stream);
  void *user;
  void *stream;
} sph_alloc;

typedef struct sph_stats {
  int64_t n;         /* live real particles, all instances */
  int64_t step;      /* advection steps taken */
  double t;          /* simulated time of instance 0 */
  double dt_ad;      /* last advection step of instance 0 */
  double dt_ac;      /* last acoustic criterion of instance 0 */
  int32_t n_ac;      /* last sub-step count of instance 0 */
  int32_t n_instances;
  int64_t spawned;   /* cumulative injected particles */
  int64_t deleted;   /* cumulative deleted particles */
  int64_t capacity;
  int64_t device_bytes; /* device memory owned by the context */
  int64_t kernel_launches; /* cumulative kernels this context launched */
  int32_t status;    /* device status word: 0 or the first SPH_ERR_* a kernel
                        set (sticky; sph_step returns it too) */
  int32_t reserved;
} sph_stats;

typedef struct sph_ctx sph_ctx;

/* Create a context of n_instances independent problems; cfg and init are
   arrays of n_instances.  All instances of one context share precision
   and dimension.  Returns SPH_ERR_ARG on an invalid configuration,
   SPH_ERR_ALLOC / SPH_ERR_CUDA on device failure; *out is NULL on error. */
int sph_create(const sph_config *cfg, int32_t n_instances, const sph_particles *init,
               const sph_alloc *alloc, sph_ctx **out);

/* Add a buffer to an instance before its first step (Sec. 2.4.1, 3.2).
   *out_id receives the buffer ID (0-based in call order per instance);
   particles inside it carry label ID+1.  SPH_ERR_OVERLAP if its box
   intersects another buffer box of the same instance, SPH_ERR_STATE after
   the first step, SPH_ERR_ARG on a bad frame or profile. */
int sph_add_buffer(sph_ctx *ctx, int32_t instance, const sph_buffer_desc *b, int32_t *out_id);

/* Replace the velocity profile theta of a velocity buffer (any time).  The
   values are staged in pinned host memory and copied on the context's
   stream, in order with the steps enqueued around the call; the call
   returns without waiting (theta may be reused at once). */
int sph_set_profile(sph_ctx *ctx, int32_t instance, int32_t buffer_id, const double *theta,
                    int32_t n_theta);

/* Advance every instance by nsteps advection steps.  Returns the first
   device error (SPH_ERR_CAPACITY, SPH_ERR_NONFINITE, SPH_ERR_TIMEOUT) seen
   in the status word; *t_out (may be NULL) receives instance 0's time. */
int sph_step(sph_ctx *ctx, int32_t nsteps, double *t_out);

/* Enqueue nsteps advection steps on the context's stream and return at once
   (no wait for the GPU).  Device errors are not seen here: sph_get_stats
   reports the status word (sph_stats.status), and sph_step returns it.
   Errors: SPH_ERR_ARG (nsteps < 0), SPH_ERR_CUDA (launch or capture). */
int sph_step_async(sph_ctx *ctx, int32_t nsteps);

/* Field selectors for sph_read_fields / sph_write_fields.  dst[k] (src[k])
   is the array of the k-th set bit in increasing bit order. */
#define SPH_F_POS (1u << 0)    /* double [n][3] */
#define SPH_F_VEL (1u << 1)    /* double [n][3] */
#define SPH_F_RHO (1u << 2)    /* double [n] */
#define SPH_F_MASS (1u << 3)   /* double [n] */
#define SPH_F_DRHO (1u << 4)   /* double [n] density rate of the last sub-step */
#define SPH_F_P (1u << 5)      /* double [n] pressure */
#define SPH_F_K (1u << 6)      /* double [n] */
#define SPH_F_EPS (1u << 7)    /* double [n] */
#define SPH_F_NUT (1u << 8)    /* double [n] eddy viscosity */
#define SPH_F_LABEL (1u << 9)  /* int32 [n] 0 fluid, b+1 in buffer b */
#define SPH_F_UID (1u << 10)   /* uint32 [n] */
#define SPH_F_B (1u << 11)     /* double [n][9] correction matrix of the last step */
#define SPH_F_ACC_NU (1u << 12) /* double [n][3] viscous acceleration of the last step */
#define SPH_F_INST (1u << 13)  /* int32 [n] instance */
#define SPH_F_KEY (1u << 14)   /* int64 [n] cell index of the current position */
#define SPH_F_ALL_READ 0x7FFFu
#define SPH_F_ALL_WRITE (SPH_F_POS | SPH_F_VEL | SPH_F_RHO | SPH_F_MASS | SPH_F_DRHO | SPH_F_K | SPH_F_EPS)

/* Copy the live particles' selected fields into caller arrays (host when
   dst_on_device == 0, device otherwise) sized for *n_out rows; call with
   dst == NULL to query *n_out only.  Synchronises the stream. */
int sph_read_fields(sph_ctx *ctx, uint32_t mask, void *const *dst, int32_t dst_on_device,
                    int64_t *n_out);

/* Overwrite selected fields of the live particles (rows in the order of
   sph_read_fields; n must equal the live count).  Only SPH_F_ALL_WRITE
   fields may be written.  Synchronises the stream. */
int sph_write_fields(sph_ctx *ctx, uint32_t mask, const void *const *src, int32_t src_on_device,
                     int64_t n);

int sph_get_stats(sph_ctx *ctx, sph_stats *out);

/* Stage timing (tracing aid, no counterpart in the paper).  While enabled,
   sph_step brackets every kernel stage with CUDA events on the context's
   stream and accumulates, per stage, the summed event time (ms) and the
   number of launches.  Stages: 0 sort (with the live count), 1 cells (empty:
   the permute writes the cell offsets), 2 permute, 3 time step (empty when
   stepping: the neighbour-list launch takes it), 4 advection sweep,
   5 momentum sweep, 6 continuity sweep (both: sub-step 1), 7 buffer update,
   8 neighbour list (built once per advection step, before the advection
   sweep), 9 later sub-steps (momentum and continuity of sub-steps 2 ..
   n_ac: in 2D one launch, which ends at once when no instance takes them;
   in 3D one momentum and one continuity launch per sub-step up to the
   context's bound on the sub-step count, each returning at once past every
   instance's count).  enable = 0 stops timing; enable = 2 also clears the totals.
   sph_get_stage_times writes up to max_stages entries. */
#define SPH_N_STAGES 10
int sph_set_profiling(sph_ctx *ctx, int32_t enable);
int sph_get_stage_times(sph_ctx *ctx, double *ms_total, int64_t *launches, int32_t max_stages,
                        int32_t *n_stages);
const char *sph_stage_name(int32_t stage);

/* CUDA-graph stepping (batching pattern; no counterpart in the paper).
   With enable != 0, sph_step replays one captured graph per advection step
   instead of enqueuing its kernels one by one: two graphs are captured on
   first use (the FP64 master arrays alternate between two copies from step
   to step), on a private capture stream, and launched on the context's
   stream.  The first step after enabling runs uncaptured.  Results are
   identical to uncaptured stepping; stage timing is not recorded for
   replayed steps.  enable = 0 returns to uncaptured stepping (the graphs
   are kept).  Errors: SPH_ERR_CUDA if capture or instantiation fails. */
int sph_set_graph(sph_ctx *ctx, int32_t enable);

/* Threads per block of the four pair-sweep kernels, in the order
   SPH_SWEEP_LIST, SPH_SWEEP_ADV, SPH_SWEEP_MOM, SPH_SWEEP_CONT; each 64, 128
   (the default) or 256, else SPH_ERR_ARG.  Drops captured graphs. */
#define SPH_SWEEP_LIST 0
#define SPH_SWEEP_ADV 1
#define SPH_SWEEP_MOM 2
#define SPH_SWEEP_CONT 3
int sph_set_launch(sph_ctx *ctx, const int32_t block[4]);
int sph_get_launch(sph_ctx *ctx, int32_t block[4]);

/* Autotuner of the sweep block sizes (no counterpart in the paper).  Looks
   up the key (GPU name and SM count, dimension, precision, instances, live
   particles, walls, RANS, sub-step bound) in the text file cache_path (may
   be NULL: no cache); on a miss it saves the state and, for each sweep in
   turn (coordinate descent), times `steps` whole advection steps replayed
   from the step's CUDA graphs with that sweep at 64, 128 and 256 threads per
   block (three untimed steps before each trial, the state restored before
   each), applies the fastest choice and appends
   "key b_list b_adv b_mom b_cont" to the file.  The state after
   the call equals the state before it.  block_out (may be NULL) receives
   the four block sizes; *from_cache (may be NULL) 1 on a cache hit. */
int sph_autotune(sph_ctx *ctx, int32_t steps, const char *cache_path, int32_t block_out[4],
                 int32_t *from_cache);

/* Snapshots of the particle state in device memory (checkpointing; no
   counterpart in the paper).  sph_save_state copies the live state (FP64
   masters, pending cell keys, counters, instance table incl. time and step
   counter, uid counters, B and viscous acceleration of the last step) into
   a new device allocation and returns its slot; sph_restore_state copies it
   back (stream-ordered), after which stepping reproduces the steps taken
   from the saved state bit for bit.  Buffer descriptions and profiles are
   not part of a snapshot.  sph_drop_state frees a slot; sph_destroy frees
   all.  Errors: SPH_ERR_ALLOC, SPH_ERR_ARG (unknown slot). */
int sph_save_state(sph_ctx *ctx, int32_t *slot_out);
int sph_restore_state(sph_ctx *ctx, int32_t slot);
int sph_drop_state(sph_ctx *ctx, int32_t slot);

/* Differentiated windows (adjoint; no counterpart in the paper).  A window
   of `steps` advection steps from the current state is differentiated with
   respect to the velocity profile theta of one velocity buffer, for the
   outlet mass flux
       J = sum over the window's steps of dt * sum_{i in S} m_i v_i . n_out / slab,
   S = the particles of `instance` labelled in one of the `outlets` buffers
   when the window starts (followed by uid), n_out = -n_b of that buffer, v
   the velocity after each step's buffer update.  Inside the window every
   instance needs SPH_DT_FIXED (dt is not differentiated), and RANS
   instances hold k, eps and nu_t at their values (frozen turbulence); the
   discrete decisions of each step (cell order, neighbour lists, labels,
   injection and deletion) are those the forward took.
   sph_adjoint_forward sets theta (n_theta values, the profile of
   profile_buffer), advances the window, keeps a state snapshot every
   checkpoint_every steps and the final state, and returns J.
   sph_adjoint_backward recomputes each segment from its snapshot, runs the
   hand-written reverse of every step in reverse order and writes dJ/dtheta
   (n_theta values); the context is left in the state after the window.
   sph_adjoint_release frees the snapshots and work arrays.
   Errors: SPH_ERR_ARG (FP32 context, dt mode, buffer kinds, sizes),
   SPH_ERR_STATE (backward without forward), SPH_ERR_ALLOC, device errors
   of the steps. */
typedef struct sph_adjoint_desc {
  int32_t instance;
  int32_t profile_buffer;  /* a velocity buffer of instance */
  int32_t steps;
  int32_t checkpoint_every;
  int32_t n_outlets;
  int32_t outlets[SPH_MAX_BUFFERS];
  int32_t n_theta;
  double slab;  /* w_s, the slab width that normalises the flux */
  double theta[SPH_MAX_THETA];
} sph_adjoint_desc;
int sph_adjoint_forward(sph_ctx *ctx, const sph_adjoint_desc *d, double *J_out);
int sph_adjoint_backward(sph_ctx *ctx, double *grad_out, int32_t n_theta);
int sph_adjoint_release(sph_ctx *ctx);

/* Neighbour pairs of the configuration at the current positions
   (0 < |r_ij|^2 < (2h)^2 in FP64, Sec. 2.4.1 cell-linked list): rows
   (uid_i, uid_j or wall index, is_wall, instance).  Writes up to max rows
   into out (host memory, [max][4] int64) and the total into *count.
   Test and debug aid; re-sorts the particles by cell. */
int sph_debug_pairs(sph_ctx *ctx, int64_t *out, int64_t max, int64_t *count);

/* The neighbour list that the pair sweeps of a step walk, built from the
   configuration at the current positions by the same kernel, precision and
   launch shape as in sph_step (the frozen configuration of the dual-criteria
   advection step, Sec. 2.3; pairs 0 < |r_ij|^2 < (2h)^2 from the cell-linked
   list, Sec. 2.4.1): rows (uid_i, uid_j or wall index, is_wall, instance),
   one per list entry, in no particular order.  In the FP32 form candidates
   near the cut-off are decided by the FP64 test, so both forms hold the
   pairs of sph_debug_pairs.  Writes up to max rows into out (host memory,
   [max][4] int64) and the total into *count.  Test aid; re-sorts the
   particles by cell.  Errors: SPH_ERR_ARG, SPH_ERR_STATE (kinematic
   context), SPH_ERR_ALLOC, SPH_ERR_CUDA, SPH_ERR_CAPACITY (a particle has
   more neighbours than its list holds; its surplus is missing). */
int sph_debug_list(sph_ctx *ctx, int64_t *out, int64_t max, int64_t *count);

/* Total mass and momentum of every instance, summed in FP64 on the GPU
   over the live particles (deleted rows excluded, copies of the last buffer
   update included) in an order that does not depend on timing, so two
   calls on the same state agree bit for bit.  mass: host [n_instances],
   momentum: host [n_instances][3] (z = 0 in 2D); either may be NULL.  The
   mass budget of the buffers (Sec. 2.4.2, 2.4.3: copies enter with their
   parent's mass, deleted particles leave with theirs) can be checked with
   it.  The first call allocates the reduction buffers (a few KB per
   instance).  Synchronises.  Errors: SPH_ERR_ARG, SPH_ERR_ALLOC,
   SPH_ERR_CUDA. */
int sph_reduce_mass_momentum(sph_ctx *ctx, double *mass, double *momentum);

/* The same FP64 totals without waiting: the reduction is enqueued on the
   context's stream and its results land in out[4 * n_instances] (per
   instance: mass, then momentum x, y, z).  out is memory the caller
   keeps, and leaves unread, until the stream has passed this point (an
   event recorded on the stream after the call, or sph_get_stats).  Device
   memory and page-locked host memory that the device can address are
   written by the reduction itself; other host memory gets a copy enqueued
   after it (pageable memory makes the call wait for that copy).  The first call
   allocates the reduction buffers.  Errors: SPH_ERR_ARG, SPH_ERR_ALLOC,
   SPH_ERR_CUDA. */
int sph_reduce_mass_momentum_async(sph_ctx *ctx, double *out);

/* Test aid (no counterpart in the paper): the binary64 -> binary32 and
   binary32 -> binary64 conversions that the FP32 form performs with integer
   operations instead of the conversion instructions (which issue on the
   FP64 pipe), applied to n values in host memory: out32[k] = in64[k]
   rounded to nearest, ties to even; out64[k] = in32[k] exactly.  Either
   direction may be skipped with a NULL input.  Uses temporary device
   buffers.  Errors: SPH_ERR_ARG (n outside 0..2^24, missing output),
   SPH_ERR_ALLOC, SPH_ERR_CUDA. */
int sph_debug_convert(const double *in64, float *out32, const float *in32, double *out64, int64_t n);

/* Test aid (no counterpart in the paper): the bounded wait of the grid
   barrier that the cooperative launches use.  Launches a two-block
   cooperative kernel on the context's barrier words in which every block
   waits for arrivals that never come, with a short poll limit (about 2^14
   polls), and synchronises.  *status_out receives the status word of that
   launch (a private word, not the context's): SPH_ERR_TIMEOUT when the
   waits ran out as they must; words_after (may be NULL, 4 uint32 in host
   memory) the barrier words after the launch, which the last block to
   leave resets to zero for the next cooperative launch.  Errors:
   SPH_ERR_ARG, SPH_ERR_ALLOC, SPH_ERR_CUDA. */
int sph_debug_barrier_timeout(sph_ctx *ctx, int32_t *status_out, uint32_t *words_after);

/* Measurement aid (no counterpart in the paper): the fused multiply-add
   throughput of the current GPU in FP32 or FP64 (SPH_PREC_*), in FLOP/s
   (one FMA = 2 FLOP), from eight independent FMA chains per thread on
   eight 256-thread blocks per SM, best of three timed launches after one
   warm-up.  The denominator of the ALU roofline of the pair sweeps.
   Allocates a small output buffer; synchronises.  Errors: SPH_ERR_ARG,
   SPH_ERR_ALLOC, SPH_ERR_CUDA. */
int sph_measure_fma_peak(int32_t precision, double *flops_per_s);

/* Cell sort of a caller's point set that allocates no device memory.  The
   paper has no counterpart: this exists for callers that cannot allocate,
   such as code running while a CUDA stream is being captured into a graph,
   or applications whose device memory is reserved up front and may not grow
   during a run.  It computes the cell index of every point on the grid of
   cfg (cells of 2 * cfg->h over [domain_lo, domain_hi), clamped at the edges,
   as sph_create builds it; no periodic wrap), sorts the point indices
   stably by cell, and writes
     order[n]                 point indices in cell order (device memory),
     cell_start[ncell + 1]    first position in order of each cell, and n at
                              the end (device memory, cell_start_len entries),
     *ncell_out               number of cells (host memory, may be NULL).
   pos is device memory, [n][3] doubles.  stream is a cudaStream_t (NULL =
   legacy stream); the call is asynchronous on it.
   Scratch is one static device array of about 9.4 MB that every GPU loading
   the library holds until exit; n above SPH_NOALLOC_MAX_POINTS, a bad grid
   or cell_start_len < ncell + 1 returns SPH_ERR_ARG, a CUDA failure
   SPH_ERR_CUDA.  All calls on a device share the array and leave their
   contents in it; calls that overlap on the GPU race.  The first call on a
   device looks up the array's address (cudaGetSymbolAddress) with that
   device current: make it before any stream capture.  That address is kept
   for the process, so the call is not valid after cudaDeviceReset.  Errors
   set the sph_last_error() message; a CUDA error already pending on the
   thread at entry is returned as SPH_ERR_CUDA before anything is launched. */
#define SPH_NOALLOC_MAX_POINTS (1 << 19)
int sph_cell_sort_noalloc(const sph_config *cfg, const double *pos, int32_t n, uint32_t *order,
                          uint32_t *cell_start, int64_t cell_start_len, int64_t *ncell_out, void *stream);

void sph_destroy(sph_ctx *ctx);
const char *sph_error_string(int code);
/* Message of the last SPH_ERR_ARG / SPH_ERR_CUDA on this thread. */
const char *sph_last_error(void);
/* SPH_ABI_VERSION (3: sph_config carries tvf_pbuf in the slot that was
   reserved, so a zeroed version-2 config keeps its meaning). */
int sph_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
