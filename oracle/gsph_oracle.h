/* gsph_oracle.h - plain, slow FP64 CPU oracle for the particle-decomposition Gamma-SPH-ALE hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load or call this library. It shares no code, header, table or constant with the CUDA path.
 *
 * Every function restates one step of the method in the order the paper gives it (Sec. II steps a-g,
 * Sec. III.A, Sec. III.B), in FP64, without blocking, fusion or reordering. Where the paper is silent
 * (it cites the Gamma-SPH-ALE equations from another work and gives no formula) the functions follow
 * a stated reading: standard SPH-ALE in conservative form with an acoustic Riemann solver, forward
 * Euler, Wendland C2 kernel with support 2h, linear EOS, von Mises perfect plasticity, mirror walls.
 *
 * Conventions: SoA arrays of length n, particles in "slot" order. Rates per particle are 15 doubles:
 *   [0] dw/dt  [1] dm/dt  [2..4] d(m v)/dt  [5] d(m E)/dt  [6..14] L = grad v (row-major, L_ab = dv_a/dx_b).
 * Deviatoric stress is stored as 6 components: xx yy zz xy xz yz.
 */
#ifndef GSPH_ORACLE_H
#define GSPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_MAT 4
#define ORC_MAX_WALL 6
#define ORC_MAX_LABEL 16
#define ORC_NRATE 15
#define ORC_HASH_MAX 1000

typedef struct {
    double rho0, K, G, Y;            /* reference density, bulk and shear modulus, yield stress */
    int32_t eos;                     /* 0: linear p = K (rho/rho0 - 1); 1: Mie-Gruneisen (c0, s, gamma0) */
    int32_t pad;
    double c0, s, gamma0;            /* Mie-Gruneisen: bulk sound speed, Us-up slope, Gruneisen gamma */
    double p_min;                    /* pressure cut-off (spall): p = max(p, p_min); -inf: none */
} orc_material;

typedef struct {
    int32_t axis;                    /* 0, 1 or 2 */
    int32_t pad;
    double pos;                      /* the wall plane is x_axis = pos */
} orc_wall;

typedef struct {
    double lo[3];                    /* fixed lower corner of the bucket grid */
    int32_t dims[3];                 /* buckets per axis */
    int32_t nmat;
    double h;                        /* smoothing length; bucket side and kernel support are 2h */
    double cfl;
    orc_material mat[ORC_MAX_MAT];
    int32_t nwalls;
    int32_t K;                       /* number of ownership labels */
    orc_wall wall[ORC_MAX_WALL];
    double g[3];                     /* body acceleration */
    double alpha;                    /* Cg bias towards the all-types Cg (Sec. III.B) */
    int32_t integrator;              /* 0: forward Euler; 1: two-stage Heun (SSP-RK2), both stages with
                                        the neighbour set of the step's start */
    int32_t pad2;
    int32_t reconstruction;          /* 0: first-order Riemann states (the particle values); 1: MUSCL,
                                        minmod-limited linear reconstruction of v and sigma at the pair
                                        midpoint from SPH gradients */
    int32_t variable_h;              /* 0: uniform h; 1: per-particle smoothing lengths h_i (orc_state.h,
                                        0 < h_i <= h, constant in time; Sec. V's varying particle sizes,
                                        reading): pair smoothing length h_ij = (h_i + h_j) / 2, support
                                        r_ij < 2 h_ij, i.e. r^2 < (h_i + h_j)^2 each operation rounded;
                                        buckets keep the side 2h (h = the largest h_i); time step
                                        dt = cfl / max_i (s_i / h_i) with s_i the FP64 signal speed */
} orc_params;

typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz;
    double *w, *m, *E;               /* volume, mass, specific total energy */
    double *sxx, *syy, *szz, *sxy, *sxz, *syz;
    uint8_t *mat, *label;
    uint32_t *id;                    /* persistent particle id */
    double *h;                       /* per-particle smoothing length (variable_h = 1), else unused */
} orc_state;

/* Sec. I: bucket hash of each particle; GARBAGE = dims product for particles outside the grid. */
void orc_hash(const orc_params *P, int64_t n, const double *x, const double *y, const double *z,
              uint32_t *key);
/* Sec. I: stable order of slots by key (ties keep slot order). perm[s] = old slot of new slot s. */
void orc_sort_order(int64_t n, const uint32_t *key, int64_t *perm);
/* Bucket ranges of the sorted keys: start[c], end[c] (end exclusive; empty bucket: 0, 0). */
void orc_cell_ranges(int64_t n, const uint32_t *sorted_key, int64_t ncell, int64_t *start, int64_t *end);

/* Sec. I: neighbours of each particle within 2h, by brute force over all pairs or by the 27-bucket
 * search. Lists hold slot indices; image (wall) neighbours are encoded as j + n*(1 + wall index).
 * count[i] real + image neighbours; lists are truncated at cap entries per particle.
 * Returns the largest count seen. */
/* h: per-particle smoothing lengths (support (h_i + h_j)^2), or null for the uniform 2h. */
int64_t orc_neighbours_brute(const orc_params *P, int64_t n, const double *x, const double *y,
                             const double *z, int64_t cap, int32_t *count, int64_t *list, const double *h);
int64_t orc_neighbours_cells(const orc_params *P, int64_t n, const double *x, const double *y,
                             const double *z, int64_t cap, int32_t *count, int64_t *list, const double *h);

/* Sec. II step f (interaction loop): per-particle rates (15 per particle, see above) and counts of
 * real and image neighbours. Particles are found with the 27-bucket search. If subset is non-null,
 * only the nsub listed slots are evaluated (rates of the others are left untouched). */
void orc_rates(const orc_params *P, const orc_state *S, int64_t nsub, const int64_t *subset,
               double *rates, int32_t *nreal, int32_t *nimage);
/* Gradients of the MUSCL reconstruction by the SPH gradient operator over real and image neighbours,
 * G_i(phi) = sum_j w_j (phi_j - phi_i) grad_i W_ij, 27 per particle: [0..8] grad v (row-major,
 * dv_a/dx_b), [9 + 3c + b] d sigma_c / dx_b for the components c = xx yy zz xy xz yz of the full
 * stress sigma = -p I + S. */
#define ORC_NGRAD 27
void orc_gradients(const orc_params *P, const orc_state *S, double *grads);
/* Equation of state of material mat (Sec. IV, reading): pressure at density rho and specific internal
 * energy e (with the cut-off) and the square of the bulk sound speed (isentropic derivative of the
 * uncut pressure, floored at 0). */
void orc_eos(const orc_params *P, int32_t mat, double rho, double e, double *p, double *cb2);

/* Floating-point operations (+, -, *, /, sqrt) of one ordered pair interaction as the oracle writes it:
 * the pair flux and its accumulation into one end's 15 rates, counted by running them on a counting
 * scalar type. */
int64_t orc_flops_per_pair(void);

/* Host threads of the per-particle loops (rates, gradients): results are the same for any count.
 * Returns the count in effect (1 when built without OpenMP). */
int32_t orc_set_threads(int32_t nthreads);
/* Time step from the current state: CFL * h / max_i (c_i + |v_i|). */
/* CFL signal speed c + |v| of particle i in FP64 (the quantity whose maximum sets the time step). */
double orc_signal_speed(const orc_params *P, const orc_state *S, int64_t i);
double orc_dt(const orc_params *P, const orc_state *S);
/* Sec. II step g: forward Euler update of the state (in place) from the rates. */
void orc_integrate(const orc_params *P, orc_state *S, const double *rates, double dt);

/* Sec. II step c: communication hash. flag[i] = 1 if a particle with another label lies in the
 * particle's bucket or one of the 26 around it; comm[i] = key[i] if flagged, else GARBAGE.
 * count[label] = flagged particles per label. */
void orc_comm_hash(const orc_params *P, int64_t n, const uint32_t *key, const uint8_t *label,
                   uint8_t *flag, uint32_t *comm, int64_t *count);
/* Sec. II step d: the MGPU boundary set of each label, in the order a sort by communication hash
 * gives it. Label-major: offsets[k]..offsets[k+1] in out hold label k's flagged slots. */
void orc_boundary_lists(int64_t n, const uint8_t *label, const uint32_t *comm, uint32_t garbage,
                        int32_t K, int64_t *offsets, int64_t *out);

/* Sec. III.A: centre of gravity of the particles selected by (label, material) (material < 0: all
 * materials) from exact fixed-point sums. Returns the particle count. */
int64_t orc_cg(const orc_params *P, int64_t n, const double *x, const double *y, const double *z,
               const uint8_t *label, const uint8_t *mat, int32_t lab, int32_t material, double cg[3]);
/* Sec. III.A: balancing hash of one position for the owner Cg `own` w.r.t. the other Cg `oth`. */
int32_t orc_balancing_hash(const double own[3], const double oth[3], const double p[3]);
/* Sec. III.A / III.B: one full pass of the swap heuristic over all label pairs (per material when
 * the scene has several). Labels are changed in place. swapped[a*K+b] receives the particles moved
 * each way for pair (a, b). Returns the total number of particles that changed label. */
int64_t orc_swap_pass(const orc_params *P, int64_t n, const double *x, const double *y,
                      const double *z, const uint8_t *mat, const uint32_t *id, uint8_t *label,
                      int64_t *swapped);

/* One whole step in the paper's order: dt from the current state; hash; stable sort; reorder;
 * swap pass if do_swap; communication hash; interaction loop; integration. The state is
 * replaced by the new state in the sorted order. Outputs (each may be null): sorted keys,
 * communication hash, flags, per-label flag counts, neighbour counts, the rates used, dt. */
/* dt_out: in, a fixed time step when > 0 (else the CFL step); out, the step's dt. */
void orc_step(const orc_params *P, orc_state *S, int32_t do_swap, uint32_t *key_out,
              uint32_t *comm_out, uint8_t *flag_out, int64_t *count_out, int32_t *nreal_out,
              int32_t *nimage_out, double *rates_out, double *dt_out);

/* Kernel function (Wendland C2, 3D, support 2h) and |dW/dr|, exposed for the tests. */
double orc_kernel_w(double r, double h);
double orc_kernel_dw(double r, double h);

/* Acoustic Riemann solver on the normal: given left/right normal velocities, normal tractions and
 * impedances, returns u* and t* (exposed for the tests). */
void orc_riemann(double uL, double uR, double tL, double tR, double ZL, double ZR, double out[2]);

/* Forward-mode derivative of J = mean v_z over `nobs` observed persistent ids after `nsteps` steps,
 * w.r.t. (Y, G, v0) of material 0 and the initial z speed, with the dt schedule frozen to dts.
 * The state is advanced in place (values only); grad receives dJ/dY, dJ/dG, dJ/dv0. Returns J. */
double orc_forward_gradient(const orc_params *P, orc_state *S, int32_t nsteps, const double *dts,
                            int64_t nobs, const uint32_t *obs_id, double grad[3]);

#ifdef __cplusplus
}
#endif
#endif
