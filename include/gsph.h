/* gsph.h - C-ABI of the GB300-native (sm_103a) particle-decomposition Gamma-SPH-ALE hot path.
 *
 * One context owns all device state of one particle set on one GPU. The calls follow the paper's
 * statement of the problem: initialise particles and materials, step, query the state, the MGPU
 * boundary set and the exchange volume (Unfer, Colle, Limido, "A novel multi-GPU parallelization
 * paradigm for SPH applied to solid mechanics", Sec. II, Sec. III).
 *
 * Conventions (all calls):
 *  - Every call returns a gsph_status; nothing aborts the process. Kernel launches are asynchronous:
 *    an error raised inside a kernel (a bounded wait that ran out, an invalid label) is recorded in
 *    the context and returned by the next synchronising call (gsph_sync, gsph_get_*), once: reporting
 *    it clears it.
 *  - Caller pointers are borrowed for the duration of the call only. `on_device` = 1 means the
 *    pointer is a device pointer of the context's GPU, 0 a host pointer. Host transfers are
 *    synchronous with respect to the host; device transfers are ordered on `stream`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Particle arrays are in "slot" order. The library re-sorts particles by bucket hash every step,
 *    so slot order changes; GSPH_F_ID gives each slot's persistent particle id (0..n-1 in the order
 *    of gsph_set_particles).
 */
#ifndef GSPH_H
#define GSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSPH_MAX_MATERIALS 4
#define GSPH_MAX_WALLS 6
#define GSPH_MAX_LABELS 16
#define GSPH_NRATE 15
#define GSPH_BALANCE_HASH_MAX 1000

typedef enum {
    GSPH_OK = 0,
    GSPH_INVALID_ARG = 1,          /* a null pointer, size or config value out of range */
    GSPH_OOM = 2,                  /* device allocation failed; the context is unchanged */
    GSPH_CUDA_ERROR = 3,           /* a CUDA runtime call or kernel launch failed */
    GSPH_PARTICLE_LEFT_DOMAIN = 4, /* warning: particles outside the bucket grid (garbage hash) */
    GSPH_DEVICE_TIMEOUT = 5,       /* a bounded device-side wait gave up; results are invalid */
    GSPH_NOT_READY = 6,            /* the call needs particles (gsph_set_particles) first */
    GSPH_DEVICE_ERROR = 7          /* a kernel flagged invalid data (e.g. a label >= K) */
} gsph_status;

typedef enum {
    GSPH_FP64 = 0,        /* every step in FP64 */
    GSPH_FP32_SPLIT = 1   /* pair fluxes in FP32 with Kahan-compensated per-particle sums;
                             positions, integration and conservation sums in FP64 */
} gsph_precision;

typedef struct {
    double rho0;   /* reference density, kg/m^3 */
    double K;      /* bulk modulus, Pa (linear EOS p = K (rho/rho0 - 1)) */
    double G;      /* shear modulus, Pa */
    double Y;      /* yield stress, Pa (von Mises perfect plasticity) */
    int32_t eos;   /* GSPH_EOS_LINEAR (K) or GSPH_EOS_MIE_GRUNEISEN (c0, s, gamma0) */
    int32_t pad;
    double c0;     /* Mie-Gruneisen (Sec. IV names it; reading): bulk sound speed, m/s, c0 > 0 */
    double s;      /* slope of the shock relation Us = c0 + s up, 0 <= s */
    double gamma0; /* Gruneisen gamma at rho0 (Gamma rho = gamma0 rho0), >= 0. With mu = rho/rho0 - 1:
                      p_H = rho0 c0^2 mu (1 + mu) / (1 - (s - 1) mu)^2 (mu > 0), rho0 c0^2 mu (mu <= 0);
                      e_H = p_H mu / (2 rho0 (1 + mu)); p = p_H + gamma0 rho0 (e - e_H), e the specific
                      internal energy E - |v|^2/2; sound speed from the isentropic derivative */
    double p_min;  /* pressure cut-off for spalling (Sec. IV): p = max(p, p_min), Pa, <= 0; -INFINITY:
                      none. Either EOS */
} gsph_material;

#define GSPH_EOS_LINEAR 0
#define GSPH_EOS_MIE_GRUNEISEN 1

typedef struct {
    int32_t axis;  /* 0, 1, 2: rigid mirror plane x_axis = pos */
    int32_t pad;
    double pos;
} gsph_wall;

typedef struct {
    double grid_lo[3];          /* lower corner of the fixed bucket grid (Sec. I) */
    int32_t grid_dims[3];       /* buckets per axis; bucket side is 2h; product < 2^27 */
    int32_t n_materials;        /* 1..GSPH_MAX_MATERIALS; > 1 turns on per-type swaps (Sec. III.B) */
    double h;                   /* smoothing length (uniform, Sec. II); kernel support 2h */
    double cfl;                 /* dt = cfl * h / max(c + |v|), the signal speed in correctly
                                   rounded FP32 from the FP32 roundings of m, w, v */
    gsph_material materials[GSPH_MAX_MATERIALS];
    int32_t n_walls;
    int32_t K;                  /* ownership labels, 1..GSPH_MAX_LABELS (Sec. II) */
    gsph_wall walls[GSPH_MAX_WALLS];
    double gravity[3];
    double alpha;               /* Cg bias towards the all-types Cg, Sec. III.B (paper: 0.1) */
    int32_t swap_period;        /* run the swap heuristic every P steps (Sec. III: 20); 0 = never */
    int32_t precision;          /* gsph_precision */
    int32_t device;             /* CUDA device ordinal */
    int32_t diagnostics;        /* 1: keep neighbour counts and rates of the last step */
    int32_t overlap;            /* 1: run the interaction in the order of Sec. II steps d-f: the pairs of
                                   particles with neighbours of their own label, while the MGPU boundary
                                   set's records are gathered into a halo buffer on a second stream (the
                                   broadcast of step d on one device), then each boundary particle's pairs
                                   with other labels, their records read from the halo. Same results up to
                                   the order of the sums; 0: one pass over all pairs (faster on one GPU) */
    int32_t integrator;         /* 0: forward Euler (Sec. II step g); 1: two-stage Heun in its strong-
                                   stability-preserving form, y* = E(y_n), y_{n+1} = (y_n + E(y*)) / 2 on the
                                   conserved variables, E the Euler stage with radial return, both stages
                                   over the neighbour set of the step's start (not with overlap = 1) */
    int32_t reconstruction;     /* 0: first-order Riemann states (the particle values); 1: MUSCL (reading of
                                   the second-order SPH-ALE variant): a gradient pass sums the SPH gradients
                                   G_i(phi) = sum_j w_j (phi_j - phi_i) grad_i W_ij of v and sigma = -p I + S
                                   over the same neighbours and images, and each pair's Riemann problem takes
                                   v and sigma of both ends reconstructed at the midpoint, phi_L* = phi_L +
                                   minmod(G_L . d, phi_R - phi_L) / 2 (R alike, d = x_R - x_L); density,
                                   energy and impedance keep the particle values, the particle velocities
                                   stay the transport velocities. Euler only: not with integrator = 1 or
                                   overlap = 1, and gsph_adjoint_step refuses it */
    int32_t variable_h;         /* 0: one smoothing length h; 1: per-particle smoothing lengths h_i (Sec. V's
                                   varying particle sizes, reading), constant in time, set with
                                   gsph_put_field(GSPH_F_H) after gsph_set_particles (default h_i = h) in
                                   [h/4, h]: h is the largest. Pair smoothing length h_ij = (h_i + h_j)/2,
                                   support r_ij < 2 h_ij (r^2 < (h_i + h_j)^2, each operation rounded), the
                                   kernel W(r, h_ij) in every pair term; buckets keep the side 2h; time step
                                   dt = cfl / max_i fl32(s_i / fl32(h_i)). Not with overlap = 1 */
} gsph_config;

typedef enum {
    /* state, FP64, n values each */
    GSPH_F_X = 0, GSPH_F_Y, GSPH_F_Z, GSPH_F_VX, GSPH_F_VY, GSPH_F_VZ,
    GSPH_F_W,            /* particle volume */
    GSPH_F_M,            /* particle mass */
    GSPH_F_E,            /* specific total energy e + |v|^2/2 */
    GSPH_F_SXX, GSPH_F_SYY, GSPH_F_SZZ, GSPH_F_SXY, GSPH_F_SXZ, GSPH_F_SYZ, /* deviatoric stress */
    GSPH_F_MATERIAL,     /* uint8 */
    GSPH_F_LABEL,        /* uint8 ownership label */
    GSPH_F_ID,           /* uint32 persistent id */
    /* outputs of the last step, in the same slot order as the state after that step */
    GSPH_F_HASH,         /* uint32 bucket hash at the start of the step (sorted) */
    GSPH_F_COMM_HASH,    /* uint32 communication hash (Sec. II step c) */
    GSPH_F_FLAG,         /* uint8 MGPU boundary flag */
    GSPH_F_NREAL,        /* int32 real neighbours (diagnostics only) */
    GSPH_F_NIMAGE,       /* int32 wall-image neighbours (diagnostics only) */
    GSPH_F_RATES,        /* FP64 n x 15 rates: dw, dm, d(mv)[3], d(mE), L[9] (diagnostics only) */
    GSPH_F_BOUNDARY,     /* uint32 slots of the MGPU boundary set, label-major, each label in
                            communication-hash order (Sec. II step d); length = boundary_total */
    GSPH_F_H,            /* FP64 per-particle smoothing length (variable_h = 1 only; settable) */
    GSPH_F_COUNT_
} gsph_field;

typedef struct {
    int64_t step;                       /* steps taken by this context */
    int64_t n;
    int32_t K;
    int32_t pad;
    int64_t garbage;                    /* particles outside the grid at the last hash */
    int64_t boundary[GSPH_MAX_LABELS];  /* MGPU boundary particles per label, last step */
    int64_t boundary_total;
    double exchange_fraction;           /* boundary_total / n (Sec. II, the exchange volume) */
    int64_t record_bytes;               /* bytes of one particle's interaction record */
    int64_t bytes_hash_broadcast;       /* step b: n * 4 * (K - 1) */
    int64_t bytes_boundary_broadcast;   /* step d: boundary_total * record_bytes * (K - 1) */
    int64_t bytes_swap;                 /* state bytes of the particles moved by the last swap pass */
    int64_t swapped_last_pass;          /* particles that changed label in the last swap pass */
    int64_t swap_passes;
    int64_t pairs_total;                /* ordered pair interactions evaluated (sum over particles of
                                           real + image neighbours) since gsph_set_particles */
    int64_t kernel_launches;            /* kernels this context launched since gsph_set_particles */
    /* workload cost per label (the cost function of Sec. V, from each particle's actual neighbour
       number): pair interactions (real + image neighbours) of the particles of each label in the last
       step, and max over labels / mean over labels */
    int64_t cost[GSPH_MAX_LABELS];
    double cost_imbalance;
    /* exactness work of the last step (the time step and the balancing hash are defined in FP64 and
       decided in FP32 outside a proven rounding bound): particles the warp filter listed as time-step
       candidates, candidates whose FP32 interval reached the largest lower bound and were evaluated in
       FP64, and balancing hashes of the last swap pass that the FP64 sequence decided */
    int64_t dt_candidates;
    int64_t dt_fp64_evaluations;
    int64_t swap_fp64_hashes;
} gsph_exchange_stats;

typedef struct {
    /* summed device time per phase (ms) over the steps recorded since gsph_set_timing, from CUDA
       events recorded around each phase. After the swap pass a step runs two branches at once: the
       communication hash on the library's second stream and the neighbour-list build on the launch
       stream; the pair kernel starts when both have ended. comm_ms and nbr_list_ms are the two branches'
       own spans (they overlap), pair_ms runs from the end of the later one. */
    double hash_sort_ms;   /* bucket hash + radix sort */
    double reorder_ms;     /* permutation into sorted order, bucket ranges, interaction records */
    double swap_ms;        /* swap heuristic passes */
    double comm_ms;        /* communication hash, flags, boundary lists (second stream) */
    double interact_ms;    /* interaction loop + integration: nbr_list_ms + pair_ms */
    int64_t steps;         /* steps recorded */
    int64_t interact_launches;
    double nbr_list_ms;    /* of which the neighbour-list kernel (beside the communication hash) */
    double pair_ms;        /* of which the pair kernel(s) (fluxes, integration; with reconstruction = 1 also
                              the gradient pass); the time-step reduction that follows runs on the
                              second stream and is in no phase */
    /* overlap = 1 only: the two interaction passes on the launch stream, and the halo gather on the
       second stream (events there), which runs concurrently with the first pass */
    double local_ms;       /* pairs within a label, integration of particles without other labels near */
    double boundary_ms;    /* pairs across labels from the halo, integration of the boundary particles */
    double halo_ms;        /* gather of the boundary set's records into the halo buffer */
} gsph_timings;

typedef struct gsph_ctx gsph_ctx;

/* Status code as text (static storage). */
const char *gsph_status_str(gsph_status s);

/* Create a context on cfg->device with the configuration copied. Errors: INVALID_ARG for a null
 * pointer or an out-of-range field (h <= 0, cfl <= 0, dims < 1 or product >= 2^27, K not in
 * 1..16, materials not in 1..4, walls > 6, axis not in 0..2, precision unknown), CUDA_ERROR if
 * the device cannot be selected. */
gsph_status gsph_create(const gsph_config *cfg, gsph_ctx **out);

/* Free every device buffer and the context (null is accepted). */
void gsph_destroy(gsph_ctx *ctx);

/* Sec. II premise: load n particles (1 <= n < 2^26). pos and vel are n x 3 row-major FP64; vol is
 * the particle volume; material and label are uint8 (material < n_materials, label < K). Mass is
 * rho0 * vol, the specific total energy |v|^2 / 2, deviatoric stress 0; ids are 0..n-1 in input
 * order. Reallocates device buffers if n changes: the new set is allocated before the old one is
 * released, so OOM leaves the context with its previous particles. Errors: INVALID_ARG, OOM, CUDA_ERROR,
 * DEVICE_ERROR (a material or label out of range, found on the device). */
gsph_status gsph_set_particles(gsph_ctx *ctx, int64_t n, const double *pos, const double *vel,
                               const double *vol, const uint8_t *material, const uint8_t *label,
                               int32_t on_device, void *stream);

/* Overwrite one state field (GSPH_F_X .. GSPH_F_ID, or GSPH_F_H with variable_h = 1) of the current
 * slot order from src (n values of the field's type). The time step is recomputed before the next
 * step. Errors: INVALID_ARG (null pointers, another field, GSPH_F_H without variable_h or a length
 * outside [h/4, h]), NOT_READY, CUDA_ERROR. */
gsph_status gsph_put_field(gsph_ctx *ctx, gsph_field f, const void *src, int32_t on_device,
                           void *stream);

/* Copy one field to dst (n values of the field's type; GSPH_F_RATES: 15 n doubles;
 * GSPH_F_BOUNDARY: boundary_total uint32). Synchronises the stream for host copies.
 * Errors: NOT_READY before particles exist or for diagnostics fields when diagnostics are off. */
gsph_status gsph_get_field(gsph_ctx *ctx, gsph_field f, void *dst, int32_t on_device, void *stream);

/* Sec. II steps a-g, repeated nsteps times, enqueued on stream: dt from the current state, bucket
 * hash, radix sort, reorder, swap heuristic when the step index is a multiple of swap_period
 * (Sec. III), communication hash and MGPU boundary set (K > 1), interaction loop with integration.
 * Asynchronous: returns after enqueueing. Within a step the communication hash runs on a second,
 * high-priority stream of the context, forked from `stream` after the swap pass and joined back before
 * the pair kernel; each step's time-step reduction runs on that stream too, beside the next step's
 * hash, sort and reorder, and the last step of the call joins it back. Work enqueued on `stream`
 * afterwards is ordered after all of it. The kernels on `stream` (all but the swap pass's cooperative
 * kernel) are programmatic dependent launches: each may be scheduled while the work before it on the
 * stream drains, and waits for that work to complete before touching memory, so stream order is kept
 * for the caller's own work before and after the call. */
gsph_status gsph_step(gsph_ctx *ctx, int32_t nsteps, void *stream);

/* Sec. III.A/B: one swap-heuristic pass over all label pairs on the current state, enqueued on
 * stream (labels change in place; per-label particle counts do not). */
gsph_status gsph_swap_now(gsph_ctx *ctx, void *stream);

/* Waits for the context's work on stream and returns any error recorded by its kernels. */
gsph_status gsph_sync(gsph_ctx *ctx, void *stream);

/* Exchange statistics of the last step (synchronises). */
gsph_status gsph_get_exchange_stats(gsph_ctx *ctx, void *stream, gsph_exchange_stats *out);

/* FP64 device reductions of the current state (synchronises): out = {sum m, sum m vx, sum m vy,
 * sum m vz, sum m E, sum w}. */
gsph_status gsph_get_conserved(gsph_ctx *ctx, void *stream, double out[6]);

/* Time step the next step will use (synchronises). */
gsph_status gsph_get_dt(gsph_ctx *ctx, void *stream, double *dt);

/* Number of particles and of buckets (grid product; the garbage hash equals it). */
gsph_status gsph_get_sizes(gsph_ctx *ctx, int64_t *n, int64_t *ncell);

/* Per-phase CUDA-event timing: max_steps > 0 arms it for up to max_steps steps (resets the
 * totals), 0 disarms. gsph_get_timings synchronises and returns the totals so far. */
gsph_status gsph_set_timing(gsph_ctx *ctx, int32_t max_steps);
/* The same with a scope: pair_only = 0 times every phase (gsph_set_timing), pair_only = 1 records only
 * the three events per step that bound the pair kernel (the ends of the two branches and of the step)
 * instead of seven, so that the dominant kernel is timed with the least added work in the stream;
 * gsph_get_timings then fills pair_ms and steps and leaves the other phases 0. Other values of
 * pair_only: GSPH_INVALID_ARG. */
gsph_status gsph_set_timing_ex(gsph_ctx *ctx, int32_t max_steps, int32_t pair_only);
gsph_status gsph_get_timings(gsph_ctx *ctx, gsph_timings *out);

/* Overrides the time step of the next gsph_step (the one after is again the CFL step). Used to replay
 * a recorded dt schedule, e.g. for finite differences with the schedule frozen. dt > 0. */
gsph_status gsph_set_dt(gsph_ctx *ctx, double dt, void *stream);

/* One reverse-mode step of the interaction loop and integration (Sec. II steps f-g), FP64, with the
 * neighbour set of the current state and the time step dt held fixed: the transpose of the Jacobian
 * of the step y_{n+1} = Step(y_n) at the current state y_n. Needs a context created with
 * precision GSPH_FP64 and diagnostics = 1 (the step's FP64 rates are recomputed internally).
 * lam_next: device, 15 x n doubles, field-major (field f of slot s at f*n + s, fields in gsph_field
 * order X..SYZ), dJ/dy_{n+1} in the slot order y_{n+1} has (the hash order of this step, as after
 * gsph_step). lam_prev: device, same layout, receives dJ/dy_n in the current slot order.
 * grad: host, receives this step's direct contributions to dJ/dY and dJ/dG of material 0.
 * Covers the linear EOS without a pressure cut-off (every material GSPH_EOS_LINEAR, p_min = -INFINITY)
 * with first-order Riemann states and one smoothing length (reconstruction = 0, variable_h = 0). Does not
 * advance the state. Errors: INVALID_ARG (null pointers, dt <= 0, wrong context kind or EOS),
 * NOT_READY, OOM, CUDA_ERROR. */
gsph_status gsph_adjoint_step(gsph_ctx *ctx, const double *lam_next, double *lam_prev, double dt,
                              double grad[2], void *stream);

/* Checkpoint and resume of a context's particle state: the 15 FP64 fields, material, label and
 * persistent id of every particle in the current slot order (and the smoothing lengths with
 * variable_h = 1), with the step counter (the swap heuristic's phase, Sec. III) and the next time step.
 * The blob is self-describing (a 64-byte header: magic "GSPHSTA1", particle count, flags, step, dt)
 * and restoring it reproduces the following steps bit for bit. gsph_state_bytes gives the blob size
 * for the context's current particle count. dst / src: host (on_device = 0) or device memory of the
 * context's GPU, at least gsph_state_bytes bytes; device copies are ordered on stream, host copies are
 * synchronous. gsph_load_state accepts a blob of another particle count (the context reallocates, as
 * gsph_set_particles does) but not one saved with another variable_h setting. Errors: INVALID_ARG
 * (null pointers, a buffer too small, a blob that is not a state blob or does not match the context),
 * NOT_READY (save without particles), OOM, CUDA_ERROR. */
size_t gsph_state_bytes(const gsph_ctx *ctx);
gsph_status gsph_save_state(gsph_ctx *ctx, void *dst, size_t bytes, int32_t on_device, void *stream);
gsph_status gsph_load_state(gsph_ctx *ctx, const void *src, size_t bytes, int32_t on_device, void *stream);

/* Gradient of an impact observable (the differentiation pattern over Sec. II steps f-g): from the
 * context's current state y_0, `steps` forward steps in the context's precision with a device
 * checkpoint of the state every `every` steps, the observable J = mean z velocity of the particles whose
 * persistent ids are listed, then the reverse sweep: each segment is recomputed from its checkpoint
 * (bit for bit) and the FP64 reverse step (gsph_adjoint_step's operations, on an internal FP64 context)
 * runs back through it. grad receives (dJ/dY, dJ/dG) of material 0 and dJ/dv0, v0 the initial z
 * velocity common to every particle (v_z = v0 and E = |v|^2 / 2 + e with e independent of v0 in y_0).
 * The time-step schedule is part of J's definition: with dts given (host, `steps` values) the forward
 * takes those steps; with dts null it takes its own CFL steps, records them in dts_out (when given), and
 * J and its gradient are those of the run with that schedule held fixed (the CFL step's own dependence
 * on G and v0 is not differentiated). Memory: ceil(steps / every) + every + 1 state blobs and two adjoint
 * vectors on the device, allocated for the call. Afterwards the context holds y_steps. Covers the
 * configurations gsph_adjoint_step covers, with the Euler integrator. Errors: INVALID_ARG (null pointers,
 * steps or every < 1, no observed particle, an id out of range, a non-positive dt, an unsupported
 * configuration), NOT_READY, OOM, CUDA_ERROR, DEVICE_ERROR / DEVICE_TIMEOUT from the steps. */
typedef struct {
    int32_t steps;              /* forward steps, >= 1 */
    int32_t every;              /* checkpoint interval in steps, >= 1 */
    int64_t n_obs;              /* number of observed particles, >= 1 */
    const uint32_t *obs_ids;    /* host: their persistent ids (e.g. the rear face of an impacting body) */
    const double *dts;          /* host, `steps` values, or null (record the CFL steps) */
    double *dts_out;            /* host, `steps` values, or null: the schedule the call used */
    double *J;                  /* host, out (may be null): the observable after `steps` steps */
    int32_t want_gradient;      /* 0: forward only (J and the schedule); grad is left untouched */
    int32_t pad;
} gsph_adj_cfg;
gsph_status gsph_adjoint(gsph_ctx *ctx, const gsph_adj_cfg *cfg, double grad[3], void *stream);

/* Failure-detection hooks (the paper has no counterpart; used by the tests of the error paths).
 * gsph_set_wait_limit: the bounded wait of the swap pass's grid barrier gives up after spin_limit polls of
 * about 64 ns each (0 restores the default, about a second) and records a timeout, which the next
 * synchronising call returns as GSPH_DEVICE_TIMEOUT; extra_blocks = 1 makes the barrier expect one block
 * more than the pass launches, so that the wait runs out in every block (the pass then returns without
 * changing any label). Errors: INVALID_ARG (null context, extra_blocks > 1).
 * gsph_debug_fail_alloc: the k-th device allocation the library makes from now on (any context) fails as
 * on an exhausted device, without calling cudaMalloc; 0 turns it off. */
gsph_status gsph_set_wait_limit(gsph_ctx *ctx, uint32_t spin_limit, uint32_t extra_blocks);
void gsph_debug_fail_alloc(int32_t k);

/* Stateless radix sort (Sec. I "radix sort" of the bucket hashes): stable ascending sort of n
 * (key, value) uint32 pairs in device memory by the low key_bits bits of the key (1..32), in
 * place. workspace: device scratch of at least gsph_radix_sort_workspace(n, key_bits) bytes,
 * owned by the caller. Asynchronous on stream. Errors: INVALID_ARG (null pointers, n < 0 or
 * n >= 2^31, key_bits out of range, workspace too small), CUDA_ERROR. */
size_t gsph_radix_sort_workspace(int64_t n, int32_t key_bits);
gsph_status gsph_radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int32_t key_bits,
                                  void *workspace, size_t workspace_bytes, void *stream);

/* The same stable sort, for callers that cannot allocate device memory: for instance code that runs
 * while another component owns every free byte of the GPU in its own pool, or code on a
 * latency-critical stream that must not pay the device-wide synchronisation cudaMalloc/cudaFree can
 * bring. The paper has no counterpart; this is a deployment convenience.
 * The scratch is a fixed array inside the library: GSPH_SORT_NOALLOC_BYTES of device memory, held on
 * every GPU that loads the library until the process exits. n must not exceed
 * GSPH_SORT_NOALLOC_MAX_N; larger n returns GSPH_INVALID_ARG before any work. keys and vals are
 * device pointers on the current device; the call allocates nothing and needs no workspace.
 * The first call on a device looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture. All calls share the one array and it
 * keeps the last call's contents: calls that overlap on the GPU (two streams, two host threads)
 * race, so serialise them. The looked-up address stays cached for the life of the process: a
 * cudaDeviceReset of that device invalidates it, so do not reset a device this entry point has run on.
 * Errors: INVALID_ARG (null pointers, n out of range, key_bits not in 1..32), CUDA_ERROR. */
#define GSPH_SORT_NOALLOC_MAX_N 1048576
#define GSPH_SORT_NOALLOC_BYTES 9439232
gsph_status gsph_radix_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t key_bits,
                                          void *stream);

#ifdef __cplusplus
}
#endif
#endif
