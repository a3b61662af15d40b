// gsph_api.cu - the C-ABI of libgsph: context, device buffers, the step in the paper's order
// (Sec. II steps a-g with the swap heuristic of Sec. III), field access, statistics and timing.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gsph_internal.cuh"

namespace gsph {
// k_sort.cu
cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t *hist, uint32_t *tot,
                             int64_t n, int bits, cudaStream_t s, bool *in_alt, bool first_hist);
size_t radix_hist_words(int64_t n);
int radix_passes(int bits);
cudaError_t launch_hash(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                        uint32_t *key, uint32_t *val, unsigned long long *garbage, cudaStream_t s);
cudaError_t launch_hash_hist(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                             uint32_t *key, uint32_t *val, unsigned long long *garbage, uint32_t *hist, int bits,
                             uint2 *zero8, int64_t nzero8, uint32_t *zero4, int64_t nzero4, cudaStream_t s);
// k_reorder_comm.cu
cudaError_t launch_reorder(bool split, const DevParams &P, int64_t n, const uint32_t *skey, const uint32_t *perm,
                           const State &A, double *xs, double *ys, double *zs, uint8_t *lab_s, uint8_t *mat_s,
                           uint32_t *id_s, uint2 *cellr, float *cxs, void *pos, void *rec, float *xf, float *yf,
                           float *zf, uint32_t *qx, uint32_t *qy, uint32_t *qz, double *hs, float *hsf,
                           const void *rec_in, float4 *posf, int *err, unsigned long long *garbage,
                           cudaStream_t s);
cudaError_t launch_comm(const DevParams &P, int64_t n, const uint32_t *skey, const uint8_t *lab_s, uint32_t *mask,
                        uint8_t *flag, uint32_t *comm, uint32_t *block_counts, unsigned long long *label_total,
                        uint32_t *blist, uint32_t *hidx, uint32_t *scan_part, int *launches, cudaStream_t s);
int comm_blocks(int64_t n);
int comm_scan_chunks(int64_t n);
cudaError_t launch_init(const DevParams &P, int64_t n, const double *pos, const double *vel, const double *vol,
                        const uint8_t *mat, const uint8_t *lab, const State &A, int *err, cudaStream_t s);
cudaError_t launch_dt_from_state(const DevParams &P, int64_t n, const State &A, const DtArgs &d, double *dt,
                                 cudaStream_t s);
cudaError_t launch_finalize_dt(const DevParams &P, int64_t n, const DtArgs &d, const State &S, double *dt,
                               cudaStream_t s);
cudaError_t launch_conserved(int64_t n, const State &A, double *part, double *out, cudaStream_t s);
// k_interact.cu
cudaError_t launch_interact(bool split, bool diag, const DevParams &P, int64_t n, const uint32_t *skey,
                            const uint2 *cellr, const void *pos, const void *rec, const float *cxs,
                            const double *xs, const double *ys, const double *zs, int kmax, uint2 *list,
                            uint32_t *cnt, const uint32_t *perm, const State &A, const State &B, cudaEvent_t mid,
                            const uint8_t *lab_s, const uint8_t *mat_s, const uint32_t *id_s, const double *dt,
                            const DtArgs &dtc, unsigned long long *pairs, unsigned long long *cost,
                            int32_t *nreal, int32_t *nimage, double *rates, const OverlapBufs *ov,
                            int stage, void *grad, const double *hs, const float *hsf, void *rec_next,
                            cudaStream_t s);
cudaError_t launch_nbr_list(const DevParams &P, int64_t n, const uint32_t *skey, const uint2 *cellr,
                            const float4 *pos_rel, const float *cxs, const double *xs, const double *ys,
                            const double *zs, int kmax, uint2 *list, uint32_t *cnt, const double *hs,
                            const float *hsf, unsigned long long *cost_clear, cudaStream_t s);
cudaError_t launch_refresh(bool split, const DevParams &P, int64_t n, const uint32_t *skey, const State &B,
                           void *pos, void *rec, cudaStream_t s);
// k_swap.cu
size_t swap_scratch_bytes(int K, int nmat);
cudaError_t launch_round_positions(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                                   float *xf, float *yf, float *zf, uint32_t *qx, uint32_t *qy, uint32_t *qz,
                                   cudaStream_t s);
cudaError_t launch_swap_pass(const DevParams &P, int64_t n, const SwapPos &pos, uint8_t *lab, const uint8_t *mat,
                             const uint32_t *id, void *scratch, uint16_t *bh, uint32_t *sidx, int *err, int grid,
                             unsigned spin_limit, unsigned extra_blocks, bool scratch_clear, cudaStream_t s);
int swap_grid_blocks();
unsigned long long *swap_moved_ptr(void *scratch);
// k_adjoint.cu
size_t adjoint_scratch_doubles(int64_t n);
cudaError_t launch_adjoint(const DevParams &P, int64_t n, const uint32_t *skey, const uint2 *cellr, const void *pos,
                           const void *rec, const double *xs, const double *ys, const double *zs, int kmax,
                           const uint2 *list, const uint32_t *cnt, const uint32_t *perm, const State &A,
                           const uint8_t *mat_s, const double *rates, double dt, const double *lam_next,
                           double *lam_prev, double *scratch, double *grad_out, cudaStream_t s);
}  // namespace gsph

using namespace gsph;

enum { PH_START = 0, PH_SORT, PH_REORDER, PH_SWAP, PH_COMM, PH_LIST, PH_INTERACT,
       PH_LOCAL, PH_HALO0, PH_HALO1,   // two-pass order only: end of the first pass; halo gather on the aux stream
       PH_COUNT };

// Neighbour-list capacity per particle, in entries of one 32-candidate batch each (an interior
// particle of the lattice has 80 real neighbours in about 20 batches; particles with more entries
// finish the rest by re-scanning, so results do not depend on it).
constexpr int kNbrMax = 40;

struct gsph_ctx {
    gsph_config cfg;
    DevParams P;
    bool split = false;
    int64_t n = 0;
    int64_t step = 0;
    bool dt_dirty = true;
    bool have_step = false;
    State A{}, B{};
    std::vector<void *> allocs;
    // per-step buffers
    uint32_t *key0 = nullptr, *val0 = nullptr, *key1 = nullptr, *val1 = nullptr, *hist = nullptr, *tot = nullptr;
    uint32_t *skey = nullptr, *perm = nullptr;
    uint2 *cellr = nullptr;
    uint32_t *mask = nullptr;
    double *xs = nullptr, *ys = nullptr, *zs = nullptr;
    float *cxs = nullptr;
    float *xf = nullptr, *yf = nullptr, *zf = nullptr;   // FP32 roundings of the positions (swap pass)
    uint32_t *qx = nullptr, *qy = nullptr, *qz = nullptr;   // fixed-point coordinates (swap pass Cg sums)
    uint2 *nbr = nullptr;                         // neighbour lists (kNbrMax x n entries, column-major)
    uint32_t *nbr_cnt = nullptr;                  // entries per particle
    uint8_t *lab_s = nullptr, *mat_s = nullptr;
    uint32_t *id_s = nullptr;
    void *pos = nullptr, *rec = nullptr;
    float4 *posf = nullptr;   // FP64 path: FP32 bucket-relative positions for the neighbour-list build
    // split path with the linear EOS: the interaction records of the state the last step integrated, in
    // that step's slot order, written by its integration; the next reorder gathers them instead of
    // converting the FP64 state (valid only while no call other than a step has changed the state)
    RecF *rec_next = nullptr;
    bool rec_next_ok = false;
    uint8_t *flag = nullptr;
    uint32_t *comm = nullptr, *blist = nullptr, *bcounts = nullptr;
    uint32_t *scan_part = nullptr;               // chunk sums of the boundary-count scan
    // two-pass interaction order (cfg.overlap)
    uint32_t *hidx = nullptr;
    void *hpos = nullptr, *hrec = nullptr, *part = nullptr;
    float *hcx = nullptr;
    int32_t *part_cnt = nullptr;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the time-step reduction of a step runs on the second stream beside the next step's first phases;
    // ev_dt marks its end, which the next pair kernel (or the end of the gsph_step call) waits for
    cudaEvent_t ev_pair = nullptr, ev_dt = nullptr;
    bool dt_pending = false;
    unsigned gather_grid = 0, boundary_grid = 0;
    unsigned long long *label_off = nullptr;   // K + 1
    unsigned long long *cost = nullptr;        // pair interactions per label, last step
    unsigned long long *garbage = nullptr;
    DtWords *dtw = nullptr;                   // time-step reduction words
    DtCand *dt_cand = nullptr;                // time-step candidates (dt_cap)
    uint32_t dt_cap = 0;
    unsigned long long *pairs = nullptr;
    double *dt = nullptr;
    int *err = nullptr;
    int32_t *nreal = nullptr, *nimage = nullptr;
    double *rates = nullptr;
    void *grad = nullptr;                      // MUSCL gradient records (reconstruction = 1)
    double *hs = nullptr;                      // variable h: sorted smoothing lengths
    float *hsf = nullptr;
    void *swap_scratch = nullptr;
    uint32_t *sidx = nullptr;                  // swap pass label segments (2n)
    uint16_t *bh = nullptr;
    double *cons_part = nullptr, *cons_out = nullptr;
    double *adj_scratch = nullptr;   // allocated on the first adjoint step
    size_t adj_scratch_n = 0;
    int swap_grid = 0;
    unsigned wait_spin = 0, wait_extra = 0;   // the swap barrier's bounded wait (0: default limit)
    // statistics
    int64_t swap_passes = 0;
    int64_t launches = 0;
    // timing
    int timing_max = 0, timing_used = 0;
    bool timing_pair_only = false;   // only the events that bound the pair kernel are recorded
    std::vector<cudaEvent_t> ev;
};

static DtArgs dt_args(const gsph_ctx *c) { return DtArgs{c->dtw, c->dt_cand, c->dt_cap}; }

#define GSPH_CK(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return GSPH_CUDA_ERROR;     \
    } while (0)

static void free_buffers(gsph_ctx *c) {
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->adj_scratch = nullptr;
    c->adj_scratch_n = 0;
    c->A = State{};
    c->B = State{};
    c->n = 0;
}

// Failure-detection test hook: the k-th device allocation from now on (0: none) fails as on an
// exhausted device, before cudaMalloc is called.
static int g_alloc_fail_at = 0;

template <class T> static cudaError_t dalloc(gsph_ctx *c, T **p, size_t count) {
    if (g_alloc_fail_at > 0 && --g_alloc_fail_at == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) { *p = nullptr; return e; }
    c->allocs.push_back(q);
    *p = (T *)q;
    return cudaSuccess;
}

static cudaError_t alloc_state(gsph_ctx *c, State &S, int64_t n) {
    for (int k = 0; k < 15; ++k) {
        cudaError_t e = dalloc(c, &S.f[k], (size_t)n);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = dalloc(c, &S.mat, (size_t)n);
    if (e == cudaSuccess) e = dalloc(c, &S.label, (size_t)n);
    if (e == cudaSuccess) e = dalloc(c, &S.id, (size_t)n);
    S.h = nullptr;
    if (e == cudaSuccess && c->cfg.variable_h) e = dalloc(c, &S.h, (size_t)n);
    return e;
}

// The integration writes the next step's records (split path, every material on the linear EOS).
static bool record_cache_applies(const gsph_ctx *c) {
    if (!c->split) return false;
    for (int k = 0; k < c->P.nmat; ++k)
        if (c->P.eos[k] != 0) return false;
    return true;
}

static cudaError_t alloc_all(gsph_ctx *c, int64_t n) {
    const size_t N = (size_t)n, C = (size_t)c->P.ncell;
    cudaError_t e;
#define A_(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    A_(alloc_state(c, c->A, n));
    A_(alloc_state(c, c->B, n));
    A_(dalloc(c, &c->key0, N)); A_(dalloc(c, &c->val0, N));
    A_(dalloc(c, &c->key1, N)); A_(dalloc(c, &c->val1, N));
    A_(dalloc(c, &c->hist, radix_hist_words(n)));
    A_(dalloc(c, &c->tot, 512));   // one total per digit value (digits of at most 9 bits)
    A_(dalloc(c, &c->cellr, C));
    for (int a = 0; a < 3; ++a) {   // bucket corners fma(i, 2h, lo), the same bits as the device's __fma_rn
        double *t = nullptr;
        const int d = c->P.dims[a] > 0 ? c->P.dims[a] : 1;
        A_(dalloc(c, &t, (size_t)d));
        std::vector<double> h((size_t)d);
        for (int i = 0; i < d; ++i) h[(size_t)i] = std::fma((double)i, c->P.cell, c->P.lo[a]);
        A_(cudaMemcpy(t, h.data(), (size_t)d * sizeof(double), cudaMemcpyHostToDevice));
        c->P.corner[a] = t;
    }
    A_(dalloc(c, &c->mask, C));
    A_(dalloc(c, &c->xs, N)); A_(dalloc(c, &c->ys, N)); A_(dalloc(c, &c->zs, N));
    A_(dalloc(c, &c->cxs, N));
    A_(dalloc(c, &c->xf, N)); A_(dalloc(c, &c->yf, N)); A_(dalloc(c, &c->zf, N));
    A_(dalloc(c, &c->qx, N)); A_(dalloc(c, &c->qy, N)); A_(dalloc(c, &c->qz, N));
    A_(dalloc(c, &c->nbr, N * (size_t)kNbrMax));
    A_(dalloc(c, &c->nbr_cnt, N));
    A_(dalloc(c, &c->lab_s, N)); A_(dalloc(c, &c->mat_s, N)); A_(dalloc(c, &c->id_s, N));
    if (c->split) {
        A_(dalloc(c, (float4 **)&c->pos, N));
        A_(dalloc(c, (RecF **)&c->rec, N));
        if (record_cache_applies(c)) A_(dalloc(c, &c->rec_next, N));
    } else {
        A_(dalloc(c, (D4 **)&c->pos, N));
        A_(dalloc(c, (RecD **)&c->rec, N));
        A_(dalloc(c, &c->posf, N));
    }
    A_(dalloc(c, &c->flag, N));
    A_(dalloc(c, &c->comm, N));
    A_(dalloc(c, &c->blist, N));
    A_(dalloc(c, &c->bcounts, (size_t)kMaxLabel * (size_t)comm_blocks(n)));
    A_(dalloc(c, &c->scan_part, (size_t)comm_scan_chunks(n)));
    A_(dalloc(c, &c->label_off, (size_t)kMaxLabel + 1));
    A_(dalloc(c, &c->cost, (size_t)kMaxLabel));
    A_(dalloc(c, &c->garbage, 1));
    A_(dalloc(c, &c->dtw, 1));
    c->dt_cap = (uint32_t)(N / 4 + 1024);
    A_(dalloc(c, &c->dt_cand, (size_t)c->dt_cap));
    A_(dalloc(c, &c->pairs, 1));
    A_(dalloc(c, &c->dt, 1));
    A_(dalloc(c, &c->err, 1));
    if (c->cfg.diagnostics) {
        A_(dalloc(c, &c->nreal, N));
        A_(dalloc(c, &c->nimage, N));
        A_(dalloc(c, &c->rates, N * kNRate));
    }
    A_(dalloc(c, (char **)&c->swap_scratch, swap_scratch_bytes(c->P.K_labels, c->P.nmat)));
    A_(dalloc(c, &c->bh, N));
    A_(dalloc(c, &c->sidx, 2 * N + 2));   // swap pass: label segments and moved lists
    A_(dalloc(c, &c->cons_part, ((N + 255) / 256 + 1) * 6));
    A_(dalloc(c, &c->cons_out, 6));
    if (c->cfg.variable_h) {   // sorted smoothing lengths, FP64 and FP32
        A_(dalloc(c, &c->hs, N));
        A_(dalloc(c, &c->hsf, N));
    }
    if (c->cfg.reconstruction) {   // MUSCL gradient records: 7 float4 (split) or 7 D4 per slot
        if (c->split) A_(dalloc(c, (float4 **)&c->grad, N * 7));
        else A_(dalloc(c, (D4 **)&c->grad, N * 7));
    }
    if (c->cfg.overlap) {
        A_(dalloc(c, &c->hidx, N));
        if (c->split) {
            A_(dalloc(c, (float4 **)&c->hpos, N));
            A_(dalloc(c, (RecF **)&c->hrec, N));
        } else {
            A_(dalloc(c, (D4 **)&c->hpos, N));
            A_(dalloc(c, (RecD **)&c->hrec, N));
        }
        A_(dalloc(c, &c->hcx, N));
        A_(dalloc(c, (char **)&c->part, N * 120));   // 21 floats or 15 doubles per boundary particle
        A_(dalloc(c, &c->part_cnt, 2 * N));
    }
#undef A_
    e = cudaMemset(c->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->dtw, 0, sizeof(DtWords));
    if (e == cudaSuccess) e = cudaMemset(c->garbage, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->pairs, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->label_off, 0, (kMaxLabel + 1) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->swap_scratch, 0, swap_scratch_bytes(c->P.K_labels, c->P.nmat));
    return e;
}

// Buffers for n particles. A trial set is allocated beside the current one first, so that a failed
// allocation leaves the context (its particles and buffers) as it was; then the current set is
// replaced. (Only if the second allocation fails after the trial succeeded - another user took the
// memory in between - is the context left without particles.)
static gsph_status realloc_for(gsph_ctx *c, int64_t n) {
    gsph_ctx *t = new (std::nothrow) gsph_ctx();
    if (!t) return GSPH_OOM;
    t->cfg = c->cfg;
    t->P = c->P;
    t->split = c->split;
    cudaError_t e = alloc_all(t, n);
    free_buffers(t);
    delete t;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSPH_OOM : GSPH_CUDA_ERROR;
    }
    free_buffers(c);
    e = alloc_all(c, n);
    if (e != cudaSuccess) {
        free_buffers(c);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSPH_OOM : GSPH_CUDA_ERROR;
    }
    c->n = n;
    return GSPH_OK;
}

static bool config_ok(const gsph_config *c) {
    if (!(c->h > 0.0) || !(c->cfl > 0.0)) return false;
    int64_t prod = 1;
    for (int a = 0; a < 3; ++a) {
        if (c->grid_dims[a] < 1 || !std::isfinite(c->grid_lo[a])) return false;
        prod *= c->grid_dims[a];
        if (prod >= ((int64_t)1 << 27)) return false;
    }
    if (c->K < 1 || c->K > GSPH_MAX_LABELS) return false;
    if (c->n_materials < 1 || c->n_materials > GSPH_MAX_MATERIALS) return false;
    for (int k = 0; k < c->n_materials; ++k) {
        const gsph_material &m = c->materials[k];
        if (!(m.rho0 > 0) || !(m.K > 0) || !(m.G >= 0) || !(m.Y > 0)) return false;
        if (m.eos != GSPH_EOS_LINEAR && m.eos != GSPH_EOS_MIE_GRUNEISEN) return false;
        if (m.eos == GSPH_EOS_MIE_GRUNEISEN && (!(m.c0 > 0) || !(m.s >= 0) || !(m.gamma0 >= 0))) return false;
        if (!(m.p_min <= 0.0)) return false;   // NaN and positive cut-offs rejected
    }
    if (c->n_walls < 0 || c->n_walls > GSPH_MAX_WALLS) return false;
    for (int k = 0; k < c->n_walls; ++k)
        if (c->walls[k].axis < 0 || c->walls[k].axis > 2 || !std::isfinite(c->walls[k].pos)) return false;
    if (c->precision != GSPH_FP64 && c->precision != GSPH_FP32_SPLIT) return false;
    if (c->swap_period < 0) return false;
    if (c->overlap != 0 && c->overlap != 1) return false;
    if (c->integrator != 0 && c->integrator != 1) return false;
    if (c->integrator == 1 && c->overlap) return false;   // the two-pass order runs the Euler step only
    if (c->reconstruction != 0 && c->reconstruction != 1) return false;
    if (c->reconstruction == 1 && (c->integrator != 0 || c->overlap != 0)) return false;   // MUSCL: Euler, one pass
    if (c->variable_h != 0 && c->variable_h != 1) return false;
    if (c->variable_h == 1 && c->overlap != 0) return false;   // the halo records carry no smoothing length
    if (!(c->alpha >= 0.0 && c->alpha <= 1.0)) return false;
    return true;
}

static void fill_params(const gsph_config &c, DevParams &P) {
    std::memset(&P, 0, sizeof(P));
    const double PI = 3.14159265358979323846;
    for (int a = 0; a < 3; ++a) {
        P.lo[a] = c.grid_lo[a];
        P.dims[a] = c.grid_dims[a];
        P.g[a] = c.gravity[a];
        if (c.gravity[a] != 0.0) P.has_gravity = 1;
    }
    P.h = c.h;
    P.cell = 2.0 * c.h;
    P.R2 = P.cell * P.cell;
    P.cfl = c.cfl;
    P.ncell = (uint32_t)((int64_t)c.grid_dims[0] * c.grid_dims[1] * c.grid_dims[2]);
    P.nwalls = c.n_walls;
    for (int k = 0; k < c.n_walls; ++k) {
        P.wall_axis[k] = c.walls[k].axis;
        P.wall_pos[k] = c.walls[k].pos;
    }
    P.nmat = c.n_materials;
    for (int k = 0; k < c.n_materials; ++k) {
        const gsph_material &m = c.materials[k];
        P.rho0[k] = m.rho0; P.K[k] = m.K; P.G[k] = m.G; P.Y[k] = m.Y;
        P.Mmod[k] = m.K + 4.0 * m.G / 3.0;
        P.f_rho0[k] = (float)m.rho0; P.f_K[k] = (float)m.K; P.f_G[k] = (float)m.G;
        P.f_Mmod[k] = (float)P.Mmod[k];
        P.eos[k] = m.eos;
        P.c0[k] = m.c0; P.s_hug[k] = m.s; P.gamma0[k] = m.gamma0;
        P.p_min[k] = m.p_min;
        P.inv_rho0[k] = 1.0 / m.rho0; P.k0[k] = m.rho0 * m.c0 * m.c0; P.inv_2rho0[k] = 1.0 / (2.0 * m.rho0);
        P.f_c0[k] = (float)m.c0; P.f_sm1[k] = (float)(m.s - 1.0); P.f_g0[k] = (float)m.gamma0;
        P.f_G43[k] = (float)(4.0 * m.G / 3.0);
    }
    double aw = 21.0 / (16.0 * PI * c.h * c.h * c.h);
    P.kdw = 5.0 * aw / c.h;
    P.alpha = c.alpha;
    P.K_labels = c.K;
    P.f_cell = (float)P.cell;
    P.f_inv_cell = (float)(1.0 / P.cell);
    for (int a = 0; a < 3; ++a) P.f_lo[a] = (float)P.lo[a];
    P.variable_h = c.variable_h;
    P.f_vlo = (float)(1.0 - kVarBand);
    P.f_vhi = (float)(1.0 + kVarBand);
    P.k5 = 210.0 / PI;
    P.f_k5 = (float)P.k5;
    if (!std::isnormal(P.f_inv_cell)) P.f_inv_cell = std::nanf("");   // the hash then always divides in FP64
    P.f_inv_h = (float)(1.0 / c.h);
    P.wall_reach = P.cell * (1.0 + 1e-6);
    for (int a = 0; a < 3; ++a) {
        const double ext = (double)c.grid_dims[a] * P.cell;
        P.q_s[a] = 4294967296.0 / ext;
        P.q_step[a] = ext * 0x1p-32;
    }
    P.f_kdw = (float)P.kdw;
    // The FP32 evaluation of r^2 - R2lo for a candidate (the list kernel's |c|^2 + (|o|^2 - R2lo) - 2 c.o
    // in frames with |coordinates| < 5h, the re-scan's direct differences) is within 7e-6 R2 of the
    // FP64 value (coordinate roundings plus the roundings of the evaluation); outside +-3e-5 R2 the FP32
    // comparison is therefore exact, inside it the FP64 positions decide.
    P.f_R2lo = (float)(P.R2 * (1.0 - 3e-5));
    P.f_R2hi = (float)(P.R2 * (1.0 + 3e-5));
}

static int64_t swap_pass_launches(const DevParams &P) {
    (void)P;
    return 3;   // sums, speculative counts (with the pair geometries), the cooperative pair loop
}

static int key_bits(uint32_t ncell) {
    int b = 1;
    while (b < 32 && (((uint64_t)1 << b) <= (uint64_t)ncell)) ++b;
    return b;
}

// Whether the step being enqueued records the event of `phase` (timing armed, and the phase in scope:
// all phases, or with pair-only timing the ends of the two branches and of the step).
static bool timed_phase(const gsph_ctx *c, int phase) {
    if (c->timing_used >= c->timing_max) return false;
    return !c->timing_pair_only || phase == PH_LIST || phase == PH_COMM || phase == PH_INTERACT;
}

static void rec_event(gsph_ctx *c, int phase, cudaStream_t s) {
    if (timed_phase(c, phase)) cudaEventRecord(c->ev[(size_t)c->timing_used * PH_COUNT + phase], s);
}

// The event of `phase` in the step being enqueued when it is timed (recorded by the callee), else null.
static cudaEvent_t phase_event(gsph_ctx *c, int phase) {
    return timed_phase(c, phase) ? c->ev[(size_t)c->timing_used * PH_COUNT + phase] : nullptr;
}

// One step. settle = false (a further step of the same gsph_step call follows) leaves the step's
// time-step reduction running on the second stream; the next step's pair kernel waits for it.
static gsph_status enqueue_step(gsph_ctx *c, cudaStream_t s, bool settle = true) {
    const DevParams &P = c->P;
    const int64_t n = c->n;
    if (c->dt_dirty) {
        GSPH_CK(launch_dt_from_state(P, n, c->A, dt_args(c), c->dt, s));
        c->dt_dirty = false;
        c->launches += 2;
    }
    const bool do_swap = P.K_labels > 1 && c->cfg.swap_period > 0 && (c->step % c->cfg.swap_period) == 0;
    rec_event(c, PH_START, s);
    // a. bucket hash and the radix sort by hash (Sec. I)
    // (the hash writes the first sort pass's tile histogram as well, and clears the bucket ranges and, on a
    // swap step, the swap pass's sums, so that the kernels from the hash to the swap pass follow one another
    // as programmatic dependent launches with no clearing between them)
    const int64_t swap_words = do_swap ? (int64_t)(swap_scratch_bytes(P.K_labels, P.nmat) / 4) : 0;
    GSPH_CK(launch_hash_hist(P, n, c->A.f[FX], c->A.f[FY], c->A.f[FZ], c->key0, c->val0, nullptr, c->hist,
                             key_bits(P.ncell), c->cellr, (int64_t)P.ncell, (uint32_t *)c->swap_scratch, swap_words,
                             s));
    bool alt = false;
    GSPH_CK(radix_sort_pairs(c->key0, c->val0, c->key1, c->val1, c->hist, c->tot, n, key_bits(P.ncell), s, &alt,
                             true));
    c->skey = alt ? c->key1 : c->key0;
    c->perm = alt ? c->val1 : c->val0;
    c->launches += 3 * radix_passes(key_bits(P.ncell));
    rec_event(c, PH_SORT, s);
    // sorted view, bucket ranges, interaction records
    GSPH_CK(launch_reorder(c->split, P, n, c->skey, c->perm, c->A, c->xs, c->ys, c->zs, c->lab_s, c->mat_s, c->id_s,
                           c->cellr, c->cxs, c->pos, c->rec, do_swap ? c->xf : nullptr, c->yf, c->zf, c->qx, c->qy,
                           c->qz, c->hs, c->hsf, c->rec_next_ok ? c->rec_next : nullptr, c->posf, c->err,
                           c->garbage, s));
    c->rec_next_ok = false;   // until this step's integration has rewritten them
    c->launches += 1;
    rec_event(c, PH_REORDER, s);
    // Sec. III: periodic swap heuristic on the sorted view
    if (do_swap) {
        const SwapPos sp{c->xf, c->yf, c->zf, c->xs, c->ys, c->zs, c->qx, c->qy, c->qz};
        GSPH_CK(launch_swap_pass(P, n, sp, c->lab_s, c->mat_s, c->id_s, c->swap_scratch, c->bh, c->sidx, c->err,
                                 c->swap_grid, c->wait_spin, c->wait_extra, true, s));
        ++c->swap_passes;
        c->launches += swap_pass_launches(P);
    }
    rec_event(c, PH_SWAP, s);
    // Two branches from here until the pair kernel: the communication hash (flags, boundary set) on the
    // second stream, at high priority, while the neighbour lists are built on the launch stream. The lists
    // read the sorted positions and bucket ranges only, and the communication hash reads no list.
    GSPH_CK(cudaEventRecord(c->ev_fork, s));
    GSPH_CK(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    const cudaStream_t sl = c->aux;
    // b-d. communication hash, MGPU boundary flags and set
    int nl = 0;
    GSPH_CK(launch_comm(P, n, c->skey, c->lab_s, c->mask, c->flag, c->comm, c->bcounts, c->label_off, c->blist,
                        c->hidx, c->scan_part, &nl, sl));
    c->launches += nl;
    rec_event(c, PH_COMM, sl);
    GSPH_CK(cudaEventRecord(c->ev_join, sl));
    // f. neighbour lists of the step (real neighbours), then the join of the two branches
    GSPH_CK(launch_nbr_list(P, n, c->skey, c->cellr, c->split ? (const float4 *)c->pos : c->posf, c->cxs, c->xs,
                            c->ys, c->zs, kNbrMax, c->nbr, c->nbr_cnt, c->hs, c->hsf, c->cost, s));
    c->launches += 1;
    rec_event(c, PH_LIST, s);
    GSPH_CK(cudaStreamWaitEvent(s, c->ev_join, 0));
    // f-g. interaction loop fused with the integration; next dt
    if (c->dt_pending) {   // the previous step's time step, which the integration uses
        GSPH_CK(cudaStreamWaitEvent(s, c->ev_dt, 0));
        c->dt_pending = false;
    }
    OverlapBufs ov{};
    if (c->cfg.overlap) {
        ov = OverlapBufs{c->flag, c->blist, c->label_off + P.K_labels, c->hidx, c->hpos, c->hrec, c->hcx, c->part,
                         c->part_cnt, c->aux, c->ev_fork, c->ev_join, phase_event(c, PH_HALO0),
                         phase_event(c, PH_HALO1), phase_event(c, PH_LOCAL), c->gather_grid, c->boundary_grid};
    }
    GSPH_CK(launch_interact(c->split, c->cfg.diagnostics != 0, P, n, c->skey, c->cellr, c->pos, c->rec, c->cxs, c->xs,
                            c->ys, c->zs, kNbrMax, c->nbr, c->nbr_cnt, c->perm, c->A, c->B, nullptr, c->lab_s,
                            c->mat_s, c->id_s, c->dt, dt_args(c), c->pairs, c->cost, c->nreal, c->nimage, c->rates,
                            c->cfg.overlap ? &ov : nullptr, c->cfg.integrator == 1 ? 1 : 0, c->grad, c->hs,
                            c->hsf, c->rec_next, s));
    if (c->cfg.overlap) c->launches += 2;   // halo gather, second pair pass
    if (c->cfg.integrator == 1) {
        // second Heun stage: records of the prediction, then its pairs over the same lists and the average
        GSPH_CK(launch_refresh(c->split, P, n, c->skey, c->B, c->pos, c->rec, s));
        GSPH_CK(launch_interact(c->split, c->cfg.diagnostics != 0, P, n, c->skey, c->cellr, c->pos, c->rec, c->cxs,
                                c->xs, c->ys, c->zs, kNbrMax, c->nbr, c->nbr_cnt, c->perm, c->A, c->B, nullptr,
                                c->lab_s, c->mat_s, c->id_s, c->dt, dt_args(c), c->pairs, c->cost, c->nreal,
                                c->nimage, c->rates, nullptr, 2, nullptr, c->hs, c->hsf, c->rec_next, s));
        c->launches += 2;
    }
    // the next time step from the integration's candidates, on the second stream: it needs only the
    // pair kernel's output, and only the next pair kernel needs it
    rec_event(c, PH_INTERACT, s);
    GSPH_CK(cudaEventRecord(c->ev_pair, s));
    GSPH_CK(cudaStreamWaitEvent(c->aux, c->ev_pair, 0));
    GSPH_CK(launch_finalize_dt(P, n, dt_args(c), c->B, c->dt, c->aux));
    GSPH_CK(cudaEventRecord(c->ev_dt, c->aux));
    c->dt_pending = true;
    c->launches += 2;   // pair kernel, time step
    if (c->timing_used < c->timing_max) ++c->timing_used;
    State t = c->A;
    c->A = c->B;
    c->B = t;
    ++c->step;
    c->have_step = true;
    c->rec_next_ok = c->rec_next != nullptr;
    if (settle) {   // work enqueued on s after this call sees the step's time step
        GSPH_CK(cudaStreamWaitEvent(s, c->ev_dt, 0));
        c->dt_pending = false;
    }
    return GSPH_OK;
}

// Hash, sort, reorder, neighbour lists and the step's FP64 rates of the current state, without
// advancing it (the integration result goes to the scratch state B).
static gsph_status enqueue_forward_pieces(gsph_ctx *c, cudaStream_t s) {
    const DevParams &P = c->P;
    const int64_t n = c->n;
    GSPH_CK(cudaMemsetAsync(c->garbage, 0, sizeof(unsigned long long), s));
    GSPH_CK(launch_hash(P, n, c->A.f[FX], c->A.f[FY], c->A.f[FZ], c->key0, c->val0, c->garbage, s));
    bool alt = false;
    GSPH_CK(radix_sort_pairs(c->key0, c->val0, c->key1, c->val1, c->hist, c->tot, n, key_bits(P.ncell), s, &alt,
                             false));
    c->skey = alt ? c->key1 : c->key0;
    c->perm = alt ? c->val1 : c->val0;
    GSPH_CK(cudaMemsetAsync(c->cellr, 0, (size_t)P.ncell * sizeof(uint2), s));
    GSPH_CK(launch_reorder(c->split, P, n, c->skey, c->perm, c->A, c->xs, c->ys, c->zs, c->lab_s, c->mat_s, c->id_s,
                           c->cellr, c->cxs, c->pos, c->rec, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, c->posf, c->err, nullptr, s));
    GSPH_CK(launch_nbr_list(P, n, c->skey, c->cellr, c->split ? (const float4 *)c->pos : c->posf, c->cxs, c->xs,
                            c->ys, c->zs, kNbrMax, c->nbr, c->nbr_cnt, c->hs, c->hsf, nullptr, s));
    GSPH_CK(launch_interact(c->split, true, P, n, c->skey, c->cellr, c->pos, c->rec, c->cxs, c->xs, c->ys, c->zs,
                            kNbrMax, c->nbr, c->nbr_cnt, c->perm, c->A, c->B, nullptr, c->lab_s, c->mat_s, c->id_s,
                            c->dt, dt_args(c), c->pairs, c->cost, c->nreal, c->nimage, c->rates, nullptr, 0, nullptr,
                            nullptr, nullptr, nullptr, s));
    c->launches += 4 + 3 * radix_passes(key_bits(P.ncell));
    c->dt_dirty = true;   // the time-step words now hold the scratch state's candidates
    c->rec_next_ok = false;
    return GSPH_OK;
}

static gsph_status read_err(gsph_ctx *c, cudaStream_t s) {
    int h = 0;
    GSPH_CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    if (h) {   // reported once: the word is cleared for the work that follows
        GSPH_CK(cudaMemsetAsync(c->err, 0, sizeof(int), s));
        GSPH_CK(cudaStreamSynchronize(s));
    }
    if (h & kErrTimeout) return GSPH_DEVICE_TIMEOUT;
    if (h) return GSPH_DEVICE_ERROR;
    return GSPH_OK;
}

static size_t field_elem_bytes(gsph_field f) {
    switch (f) {
        case GSPH_F_MATERIAL: case GSPH_F_LABEL: case GSPH_F_FLAG: return 1;
        case GSPH_F_ID: case GSPH_F_HASH: case GSPH_F_COMM_HASH: case GSPH_F_NREAL: case GSPH_F_NIMAGE:
        case GSPH_F_BOUNDARY: return 4;
        case GSPH_F_RATES: return 8 * kNRate;
        default: return 8;   // FP64 fields, GSPH_F_H
    }
}

extern "C" {

const char *gsph_status_str(gsph_status s) {
    switch (s) {
        case GSPH_OK: return "ok";
        case GSPH_INVALID_ARG: return "invalid argument";
        case GSPH_OOM: return "device out of memory";
        case GSPH_CUDA_ERROR: return "CUDA error";
        case GSPH_PARTICLE_LEFT_DOMAIN: return "particles left the bucket grid";
        case GSPH_DEVICE_TIMEOUT: return "bounded device wait timed out";
        case GSPH_NOT_READY: return "no particles loaded";
        case GSPH_DEVICE_ERROR: return "invalid data found on the device";
    }
    return "unknown status";
}

gsph_status gsph_create(const gsph_config *cfg, gsph_ctx **out) {
    if (!cfg || !out) return GSPH_INVALID_ARG;
    *out = nullptr;
    if (!config_ok(cfg)) return GSPH_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return GSPH_CUDA_ERROR;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return GSPH_CUDA_ERROR;
    gsph_ctx *c = new (std::nothrow) gsph_ctx();
    if (!c) return GSPH_OOM;
    c->cfg = *cfg;
    c->split = cfg->precision == GSPH_FP32_SPLIT;
    fill_params(*cfg, c->P);
    if (cfg->K > 1) {
        c->swap_grid = swap_grid_blocks();
        if (c->swap_grid < 1) {
            delete c;
            return GSPH_CUDA_ERROR;
        }
    }
    {
        // the second stream runs at the highest priority: the swap pass and the communication hash beside
        // the list build, so that their few blocks are scheduled ahead of the list kernel's, and with
        // overlap = 1 the halo gather, ahead of the first pair pass's blocks, so that the gather (the
        // broadcast) completes early in that pass
        int sms = 0, prio_lo = 0, prio_hi = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess ||
            cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_pair, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_dt, cudaEventDisableTiming) != cudaSuccess) {
            gsph_destroy(c);
            return GSPH_CUDA_ERROR;
        }
        c->gather_grid = (unsigned)(2 * sms);     // 256-thread blocks, grid-stride over the boundary set
        c->boundary_grid = (unsigned)(5 * sms);   // the pair kernel's resident blocks, grid-stride
    }
    *out = c;
    return GSPH_OK;
}

void gsph_destroy(gsph_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->cfg.device);
    cudaDeviceSynchronize();
    free_buffers(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_pair) cudaEventDestroy(c->ev_pair);
    if (c->ev_dt) cudaEventDestroy(c->ev_dt);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
}

gsph_status gsph_set_particles(gsph_ctx *c, int64_t n, const double *pos, const double *vel, const double *vol,
                               const uint8_t *material, const uint8_t *label, int32_t on_device, void *stream) {
    if (!c || n < 1 || n >= ((int64_t)1 << 26) || !pos || !vel || !vol || !material || !label) return GSPH_INVALID_ARG;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    GSPH_CK(cudaStreamSynchronize(s));
    if (n != c->n) {
        gsph_status st = realloc_for(c, n);
        if (st != GSPH_OK) return st;
    }
    void *stage = nullptr;
    const double *dpos = pos, *dvel = vel, *dvol = vol;
    const uint8_t *dmat = material, *dlab = label;
    if (!on_device) {
        const size_t nb = (size_t)n;
        cudaError_t e = cudaMalloc(&stage, nb * 8 * 7 + nb * 2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? GSPH_OOM : GSPH_CUDA_ERROR;
        }
        char *q = (char *)stage;
        e = cudaMemcpyAsync(q, pos, nb * 24, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q + nb * 24, vel, nb * 24, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q + nb * 48, vol, nb * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q + nb * 56, material, nb, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q + nb * 57, label, nb, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            cudaFree(stage);
            return GSPH_CUDA_ERROR;
        }
        dpos = (const double *)q;
        dvel = (const double *)(q + nb * 24);
        dvol = (const double *)(q + nb * 48);
        dmat = (const uint8_t *)(q + nb * 56);
        dlab = (const uint8_t *)(q + nb * 57);
    }
    cudaError_t e = cudaMemsetAsync(c->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->pairs, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_init(c->P, n, dpos, dvel, dvol, dmat, dlab, c->A, c->err, s);
    if (e == cudaSuccess) e = launch_dt_from_state(c->P, n, c->A, dt_args(c), c->dt, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (stage) cudaFree(stage);
    if (e != cudaSuccess || e2 != cudaSuccess) return GSPH_CUDA_ERROR;
    c->dt_dirty = false;
    c->step = 0;
    c->have_step = false;
    c->rec_next_ok = false;
    c->swap_passes = 0;
    c->launches = 3;
    return read_err(c, s);
}

gsph_status gsph_put_field(gsph_ctx *c, gsph_field f, const void *src, int32_t on_device, void *stream) {
    if (!c || !src || (int)f < 0 || (f > GSPH_F_ID && f != GSPH_F_H)) return GSPH_INVALID_ARG;
    if (f == GSPH_F_H && !c->cfg.variable_h) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> hcheck;
    if (f == GSPH_F_H) {   // smoothing lengths in [h/4, h] (the bucket side and the list test's band)
        const double *hv = (const double *)src;
        if (on_device) {
            hcheck.resize((size_t)c->n);
            GSPH_CK(cudaMemcpyAsync(hcheck.data(), src, (size_t)c->n * 8, cudaMemcpyDeviceToHost, s));
            GSPH_CK(cudaStreamSynchronize(s));
            hv = hcheck.data();
        }
        for (int64_t i = 0; i < c->n; ++i)
            if (!(hv[i] <= c->cfg.h && hv[i] >= 0.25 * c->cfg.h)) return GSPH_INVALID_ARG;
    }
    void *dst = f <= GSPH_F_SYZ ? (void *)c->A.f[f]
              : f == GSPH_F_MATERIAL ? (void *)c->A.mat : f == GSPH_F_LABEL ? (void *)c->A.label
              : f == GSPH_F_H ? (void *)c->A.h : (void *)c->A.id;
    GSPH_CK(cudaMemcpyAsync(dst, src, (size_t)c->n * field_elem_bytes(f),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (!on_device) GSPH_CK(cudaStreamSynchronize(s));
    c->dt_dirty = true;
    c->rec_next_ok = false;
    return GSPH_OK;
}

gsph_status gsph_get_field(gsph_ctx *c, gsph_field f, void *dst, int32_t on_device, void *stream) {
    if (!c || !dst || (int)f < 0 || f >= GSPH_F_COUNT_) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const void *src = nullptr;
    size_t count = (size_t)c->n;
    if (f <= GSPH_F_SYZ) src = c->A.f[f];
    else if (f == GSPH_F_H) {
        if (!c->cfg.variable_h) return GSPH_INVALID_ARG;
        src = c->A.h;
    } else if (f == GSPH_F_MATERIAL) src = c->A.mat;
    else if (f == GSPH_F_LABEL) src = c->A.label;
    else if (f == GSPH_F_ID) src = c->A.id;
    else {
        if (!c->have_step) return GSPH_NOT_READY;
        if (f == GSPH_F_HASH) src = c->skey;
        else if (f == GSPH_F_COMM_HASH) src = c->comm;
        else if (f == GSPH_F_FLAG) src = c->flag;
        else if (f == GSPH_F_BOUNDARY) {
            unsigned long long tot = 0;
            GSPH_CK(cudaMemcpyAsync(&tot, c->label_off + c->P.K_labels, sizeof(tot), cudaMemcpyDeviceToHost, s));
            GSPH_CK(cudaStreamSynchronize(s));
            count = (size_t)tot;
            src = c->blist;
        } else {
            if (!c->cfg.diagnostics) return GSPH_NOT_READY;
            src = f == GSPH_F_NREAL ? (const void *)c->nreal : f == GSPH_F_NIMAGE ? (const void *)c->nimage
                                                                                   : (const void *)c->rates;
        }
    }
    if (count > 0)
        GSPH_CK(cudaMemcpyAsync(dst, src, count * field_elem_bytes(f),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!on_device) GSPH_CK(cudaStreamSynchronize(s));
    return GSPH_OK;
}

gsph_status gsph_step(gsph_ctx *c, int32_t nsteps, void *stream) {
    if (!c || nsteps < 0) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < nsteps; ++k) {
        gsph_status st = enqueue_step(c, s, k == nsteps - 1);
        if (st != GSPH_OK) return st;
    }
    return GSPH_OK;
}

gsph_status gsph_swap_now(gsph_ctx *c, void *stream) {
    if (!c) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    GSPH_CK(launch_round_positions(c->P, c->n, c->A.f[FX], c->A.f[FY], c->A.f[FZ], c->xf, c->yf, c->zf, c->qx, c->qy,
                                   c->qz, s));
    const SwapPos sp{c->xf, c->yf, c->zf, c->A.f[FX], c->A.f[FY], c->A.f[FZ], c->qx, c->qy, c->qz};
    GSPH_CK(launch_swap_pass(c->P, c->n, sp, c->A.label, c->A.mat, c->A.id, c->swap_scratch, c->bh, c->sidx, c->err,
                             c->swap_grid, c->wait_spin, c->wait_extra, false, s));
    ++c->swap_passes;
    c->launches += 1 + swap_pass_launches(c->P);
    return GSPH_OK;
}

gsph_status gsph_sync(gsph_ctx *c, void *stream) {
    if (!c) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_OK;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    return read_err(c, (cudaStream_t)stream);
}

gsph_status gsph_get_exchange_stats(gsph_ctx *c, void *stream, gsph_exchange_stats *out) {
    if (!c || !out) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    unsigned long long off[kMaxLabel + 1] = {0}, garb = 0, moved[2] = {0, 0}, pairs = 0, cost[kMaxLabel] = {0};
    DtWords dw{};
    GSPH_CK(cudaMemcpyAsync(off, c->label_off, sizeof(off), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(cost, c->cost, sizeof(cost), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(&garb, c->garbage, sizeof(garb), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(moved, swap_moved_ptr(c->swap_scratch), sizeof(moved), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(&dw, c->dtw, sizeof(dw), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(&pairs, c->pairs, sizeof(pairs), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    const int K = c->P.K_labels;
    out->step = c->step;
    out->n = c->n;
    out->K = K;
    out->garbage = c->have_step ? (int64_t)garb : 0;
    if (c->have_step) {
        for (int k = 0; k < K; ++k) out->boundary[k] = (int64_t)((k + 1 < K ? off[k + 1] : off[K]) - off[k]);
        out->boundary_total = (int64_t)off[K];
    }
    out->exchange_fraction = (double)out->boundary_total / (double)c->n;
    out->record_bytes = c->split ? (int64_t)(sizeof(float4) + sizeof(RecF)) : (int64_t)(sizeof(D4) + sizeof(RecD));
    out->bytes_hash_broadcast = c->n * 4 * (K - 1);
    out->bytes_boundary_broadcast = out->boundary_total * out->record_bytes * (K - 1);
    out->swapped_last_pass = (int64_t)moved[0];
    out->bytes_swap = (int64_t)moved[0] * (15 * 8 + 6);
    out->swap_fp64_hashes = (int64_t)moved[1];
    out->dt_candidates = dw.last_ccount;
    out->dt_fp64_evaluations = dw.last_eval;
    out->swap_passes = c->swap_passes;
    out->pairs_total = (int64_t)pairs;
    out->kernel_launches = c->launches;
    if (c->have_step) {
        double mx = 0.0, sum = 0.0;
        for (int k = 0; k < K; ++k) {
            out->cost[k] = (int64_t)cost[k];
            sum += (double)cost[k];
            mx = mx > (double)cost[k] ? mx : (double)cost[k];
        }
        out->cost_imbalance = sum > 0.0 ? mx / (sum / K) : 0.0;
    }
    return out->garbage > 0 ? GSPH_PARTICLE_LEFT_DOMAIN : GSPH_OK;
}

gsph_status gsph_get_conserved(gsph_ctx *c, void *stream, double out[6]) {
    if (!c || !out) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    GSPH_CK(launch_conserved(c->n, c->A, c->cons_part, c->cons_out, s));
    GSPH_CK(cudaMemcpyAsync(out, c->cons_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    return GSPH_OK;
}

gsph_status gsph_get_dt(gsph_ctx *c, void *stream, double *dt) {
    if (!c || !dt) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dt_dirty) {
        GSPH_CK(launch_dt_from_state(c->P, c->n, c->A, dt_args(c), c->dt, s));
        c->dt_dirty = false;
    }
    GSPH_CK(cudaMemcpyAsync(dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    return GSPH_OK;
}

gsph_status gsph_set_dt(gsph_ctx *c, double dt, void *stream) {
    if (!c || !(dt > 0.0)) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    GSPH_CK(cudaMemcpyAsync(c->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, s));
    GSPH_CK(cudaMemsetAsync(c->dtw, 0, offsetof(DtWords, hint), s));   // the state (and its hint) stays
    GSPH_CK(cudaStreamSynchronize(s));
    c->dt_dirty = false;
    return GSPH_OK;
}

gsph_status gsph_adjoint_step(gsph_ctx *c, const double *lam_next, double *lam_prev, double dt, double grad[2],
                              void *stream) {
    if (!c || !lam_next || !lam_prev || !grad || !(dt > 0.0)) return GSPH_INVALID_ARG;
    if (c->split || !c->cfg.diagnostics || c->cfg.reconstruction || c->cfg.variable_h) return GSPH_INVALID_ARG;
    for (int k = 0; k < c->cfg.n_materials; ++k)   // the reverse mode covers the linear EOS without cut-off
        if (c->cfg.materials[k].eos != GSPH_EOS_LINEAR || !std::isinf(c->cfg.materials[k].p_min)) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = adjoint_scratch_doubles(c->n);
    if (c->adj_scratch_n < need) {
        double *p = nullptr;
        cudaError_t e = dalloc(c, &p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? GSPH_OOM : GSPH_CUDA_ERROR;
        }
        c->adj_scratch = p;
        c->adj_scratch_n = need;
    }
    GSPH_CK(cudaMemcpyAsync(c->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, s));
    gsph_status st = enqueue_forward_pieces(c, s);
    if (st != GSPH_OK) return st;
    double *gdev = c->adj_scratch + need - 2;
    GSPH_CK(launch_adjoint(c->P, c->n, c->skey, c->cellr, c->pos, c->rec, c->xs, c->ys, c->zs, kNbrMax, c->nbr,
                           c->nbr_cnt, c->perm, c->A, c->mat_s, c->rates, dt, lam_next, lam_prev, c->adj_scratch,
                           gdev, s));
    c->launches += 3;
    GSPH_CK(cudaMemcpyAsync(grad, gdev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    return read_err(c, s);
}

gsph_status gsph_get_sizes(gsph_ctx *c, int64_t *n, int64_t *ncell) {
    if (!c) return GSPH_INVALID_ARG;
    if (n) *n = c->n;
    if (ncell) *ncell = (int64_t)c->P.ncell;
    return GSPH_OK;
}

gsph_status gsph_set_timing(gsph_ctx *c, int32_t max_steps) { return gsph_set_timing_ex(c, max_steps, 0); }

gsph_status gsph_set_timing_ex(gsph_ctx *c, int32_t max_steps, int32_t pair_only) {
    if (!c || max_steps < 0 || (pair_only != 0 && pair_only != 1)) return GSPH_INVALID_ARG;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    GSPH_CK(cudaDeviceSynchronize());
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->timing_max = 0;
    c->timing_used = 0;
    c->timing_pair_only = pair_only != 0;
    if (max_steps == 0) return GSPH_OK;
    c->ev.resize((size_t)max_steps * PH_COUNT);
    for (auto &e : c->ev) GSPH_CK(cudaEventCreate(&e));
    c->timing_max = max_steps;
    return GSPH_OK;
}

gsph_status gsph_get_timings(gsph_ctx *c, gsph_timings *out) {
    if (!c || !out) return GSPH_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    GSPH_CK(cudaSetDevice(c->cfg.device));
    for (int k = 0; k < c->timing_used; ++k) {
        cudaEvent_t *e = &c->ev[(size_t)k * PH_COUNT];
        GSPH_CK(cudaEventSynchronize(e[PH_INTERACT]));
        if (c->timing_pair_only) {   // from the end of the later branch to the end of the step
            float a = 0.f, b = 0.f;
            GSPH_CK(cudaEventElapsedTime(&a, e[PH_LIST], e[PH_INTERACT]));
            GSPH_CK(cudaEventElapsedTime(&b, e[PH_COMM], e[PH_INTERACT]));
            out->pair_ms += a < b ? a : b;
            continue;
        }
        float t[PH_COUNT] = {0};
        for (int p = 1; p <= PH_COMM; ++p) GSPH_CK(cudaEventElapsedTime(&t[p], e[p - 1], e[p]));
        // the two branches after the swap pass: communication hash on the second stream, the list build on
        // the launch stream; the pair kernel starts once both have ended
        GSPH_CK(cudaEventElapsedTime(&t[PH_LIST], e[PH_SWAP], e[PH_LIST]));
        float t_join = 0.f;   // from the end of the later branch to the end of the step
        {
            float a = 0.f, b = 0.f;
            GSPH_CK(cudaEventElapsedTime(&a, e[PH_LIST], e[PH_INTERACT]));
            GSPH_CK(cudaEventElapsedTime(&b, e[PH_COMM], e[PH_INTERACT]));
            t_join = a < b ? a : b;
        }
        t[PH_INTERACT] = t_join;
        if (c->cfg.overlap) {
            float tl = 0.f, tb = 0.f, th = 0.f;
            GSPH_CK(cudaEventElapsedTime(&tl, e[PH_LIST], e[PH_LOCAL]));
            {
                float b = 0.f;
                GSPH_CK(cudaEventElapsedTime(&b, e[PH_COMM], e[PH_LOCAL]));
                tl = tl < b ? tl : b;
            }
            GSPH_CK(cudaEventElapsedTime(&tb, e[PH_LOCAL], e[PH_INTERACT]));
            GSPH_CK(cudaEventElapsedTime(&th, e[PH_HALO0], e[PH_HALO1]));
            out->local_ms += tl;
            out->boundary_ms += tb;
            out->halo_ms += th;
        }
        out->hash_sort_ms += t[PH_SORT];
        out->reorder_ms += t[PH_REORDER];
        out->swap_ms += t[PH_SWAP];
        out->comm_ms += t[PH_COMM];
        out->interact_ms += t[PH_LIST] + t[PH_INTERACT];
        out->nbr_list_ms += t[PH_LIST];
        out->pair_ms += t[PH_INTERACT];
    }
    out->steps = c->timing_used;
    out->interact_launches = c->timing_used;
    return GSPH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Checkpoint / resume: a 64-byte header and the state arrays, each at a 256-byte aligned offset.
// ---------------------------------------------------------------------------------------------
namespace {
struct StateHeader {
    char magic[8];       // "GSPHSTA1"
    int64_t n;
    int32_t flags;       // bit 0: smoothing lengths present (variable_h)
    int32_t dt_valid;    // 1: dt is the next step's time step
    int64_t step;
    double dt;
    int64_t pad[3];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");
constexpr char kStateMagic[8] = {'G', 'S', 'P', 'H', 'S', 'T', 'A', '1'};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets of the arrays: 15 FP64 fields, material, label, id, h (variable_h). Returns the blob size.
size_t state_layout(int64_t n, bool varh, size_t off[19]) {
    size_t o = align256(sizeof(StateHeader));
    for (int k = 0; k < 15; ++k) { off[k] = o; o = align256(o + (size_t)n * 8); }
    off[15] = o; o = align256(o + (size_t)n);
    off[16] = o; o = align256(o + (size_t)n);
    off[17] = o; o = align256(o + (size_t)n * 4);
    off[18] = o;
    if (varh) o = align256(o + (size_t)n * 8);
    return o;
}

// The state arrays of A to (out = true) or from a blob, device or host, ordered on s.
cudaError_t copy_state_arrays(gsph_ctx *c, char *blob, bool on_device, bool out, cudaStream_t s) {
    size_t off[19];
    state_layout(c->n, c->cfg.variable_h != 0, off);
    const size_t N = (size_t)c->n;
    struct A_ { void *p; size_t bytes; };
    A_ arr[19];
    int na = 0;
    for (int k = 0; k < 15; ++k) arr[na++] = {c->A.f[k], N * 8};
    arr[na++] = {c->A.mat, N};
    arr[na++] = {c->A.label, N};
    arr[na++] = {c->A.id, N * 4};
    if (c->cfg.variable_h) arr[na++] = {c->A.h, N * 8};
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    for (int k = 0; k < na; ++k) {
        cudaError_t e = out ? cudaMemcpyAsync(blob + off[k], arr[k].p, arr[k].bytes, kind, s)
                            : cudaMemcpyAsync(arr[k].p, blob + off[k], arr[k].bytes, kind, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

size_t gsph_state_bytes(const gsph_ctx *c) {
    if (!c) return 0;
    size_t off[19];
    return state_layout(c->n, c->cfg.variable_h != 0, off);
}

gsph_status gsph_save_state(gsph_ctx *c, void *dst, size_t bytes, int32_t on_device, void *stream) {
    if (!c || !dst) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    if (bytes < gsph_state_bytes(c)) return GSPH_INVALID_ARG;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dt_dirty) {
        GSPH_CK(launch_dt_from_state(c->P, c->n, c->A, dt_args(c), c->dt, s));
        c->dt_dirty = false;
    }
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.n = c->n;
    h.flags = c->cfg.variable_h ? 1 : 0;
    h.dt_valid = 1;
    h.step = c->step;
    GSPH_CK(cudaMemcpyAsync(&h.dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    char *b = (char *)dst;
    if (on_device) GSPH_CK(cudaMemcpy(b, &h, sizeof(h), cudaMemcpyHostToDevice));
    else std::memcpy(b, &h, sizeof(h));
    GSPH_CK(copy_state_arrays(c, b, on_device != 0, true, s));
    if (!on_device) GSPH_CK(cudaStreamSynchronize(s));
    return GSPH_OK;
}

gsph_status gsph_load_state(gsph_ctx *c, const void *src, size_t bytes, int32_t on_device, void *stream) {
    if (!c || !src || bytes < sizeof(StateHeader)) return GSPH_INVALID_ARG;
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    StateHeader h{};
    if (on_device) {
        GSPH_CK(cudaStreamSynchronize(s));
        GSPH_CK(cudaMemcpy(&h, src, sizeof(h), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(&h, src, sizeof(h));
    }
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.n < 1 || h.n >= ((int64_t)1 << 26) ||
        ((h.flags & 1) != 0) != (c->cfg.variable_h != 0) || !(h.dt > 0.0 || !h.dt_valid))
        return GSPH_INVALID_ARG;
    size_t off[19];
    if (bytes < state_layout(h.n, c->cfg.variable_h != 0, off)) return GSPH_INVALID_ARG;
    if (h.n != c->n) {
        GSPH_CK(cudaStreamSynchronize(s));
        gsph_status st = realloc_for(c, h.n);
        if (st != GSPH_OK) return st;
        c->swap_passes = 0;
        c->launches = 0;
    }
    GSPH_CK(copy_state_arrays(c, (char *)src, on_device != 0, false, s));
    if (h.dt_valid) GSPH_CK(cudaMemcpyAsync(c->dt, &h.dt, sizeof(double), cudaMemcpyHostToDevice, s));
    GSPH_CK(cudaMemsetAsync(c->dtw, 0, offsetof(DtWords, last_ccount), s));
    GSPH_CK(cudaStreamSynchronize(s));
    c->step = h.step;
    c->dt_dirty = !h.dt_valid;
    c->have_step = false;
    c->rec_next_ok = false;
    return GSPH_OK;
}

// ---------------------------------------------------------------------------------------------
// Gradient of the impact observable: checkpointed forward, segment recompute, FP64 reverse sweep.
// ---------------------------------------------------------------------------------------------
namespace {
struct DevBufs {   // device allocations of one call, freed on every return path
    std::vector<void *> p;
    ~DevBufs() { for (void *q : p) cudaFree(q); }
    cudaError_t get(void **q, size_t bytes) {
        *q = nullptr;
        cudaError_t e = cudaMalloc(q, bytes);
        if (e == cudaSuccess) p.push_back(*q);
        return e;
    }
};
gsph_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return GSPH_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GSPH_OOM : GSPH_CUDA_ERROR;
}
}  // namespace

gsph_status gsph_adjoint(gsph_ctx *c, const gsph_adj_cfg *a, double grad[3], void *stream) {
    if (!c || !a || a->steps < 1 || a->every < 1 || a->n_obs < 1 || !a->obs_ids) return GSPH_INVALID_ARG;
    if (a->want_gradient && !grad) return GSPH_INVALID_ARG;
    if (c->cfg.reconstruction || c->cfg.variable_h || c->cfg.integrator) return GSPH_INVALID_ARG;
    for (int k = 0; k < c->cfg.n_materials; ++k)
        if (c->cfg.materials[k].eos != GSPH_EOS_LINEAR || !std::isinf(c->cfg.materials[k].p_min)) return GSPH_INVALID_ARG;
    if (c->n == 0) return GSPH_NOT_READY;
    const int64_t n = c->n;
    const int N = a->steps, every = a->every;
    if (a->dts)
        for (int k = 0; k < N; ++k)
            if (!(a->dts[k] > 0.0)) return GSPH_INVALID_ARG;
    std::vector<char> obs((size_t)n, 0);
    for (int64_t q = 0; q < a->n_obs; ++q) {
        if ((int64_t)a->obs_ids[q] >= n) return GSPH_INVALID_ARG;
        obs[a->obs_ids[q]] = 1;
    }
    GSPH_CK(cudaSetDevice(c->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sb = gsph_state_bytes(c);
    const int nck = (N + every - 1) / every;
    DevBufs mem;
    std::vector<char *> ck((size_t)nck), seg((size_t)every);
    char *fin = nullptr;
    for (int k = 0; k < nck; ++k) { gsph_status st = from_cuda(mem.get((void **)&ck[k], sb)); if (st) return st; }
    { gsph_status st = from_cuda(mem.get((void **)&fin, sb)); if (st) return st; }
    std::vector<double> dts((size_t)N);
    gsph_status st;
    // forward: checkpoints every `every` steps, the schedule given or recorded
    for (int k = 0; k < N; ++k) {
        if (k % every == 0 && (st = gsph_save_state(c, ck[k / every], sb, 1, stream)) != GSPH_OK) return st;
        if (a->dts) {
            if ((st = gsph_set_dt(c, a->dts[k], stream)) != GSPH_OK) return st;
            dts[k] = a->dts[k];
        } else if ((st = gsph_get_dt(c, stream, &dts[k])) != GSPH_OK) {
            return st;
        }
        if ((st = enqueue_step(c, s)) != GSPH_OK) return st;
    }
    if ((st = gsph_sync(c, stream)) != GSPH_OK) return st;
    if ((st = gsph_save_state(c, fin, sb, 1, stream)) != GSPH_OK) return st;
    if (a->dts_out) std::memcpy(a->dts_out, dts.data(), (size_t)N * sizeof(double));
    // J: mean z velocity of the observed particles, summed in slot order
    std::vector<uint32_t> ids((size_t)n);
    std::vector<double> vz((size_t)n);
    GSPH_CK(cudaMemcpyAsync(ids.data(), c->A.id, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaMemcpyAsync(vz.data(), c->A.f[FVZ], (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    GSPH_CK(cudaStreamSynchronize(s));
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        if (ids[i] < (uint32_t)n && obs[ids[i]]) { sum += vz[i]; ++cnt; }
    if (cnt == 0) return GSPH_INVALID_ARG;
    if (a->J) *a->J = sum / (double)cnt;
    if (!a->want_gradient) return GSPH_OK;
    // dJ/dy_N: 1 / count on the observed particles' v_z, in the final slot order
    double *lam = nullptr, *lamp = nullptr;
    if ((st = from_cuda(mem.get((void **)&lam, (size_t)n * 15 * 8))) != GSPH_OK) return st;
    if ((st = from_cuda(mem.get((void **)&lamp, (size_t)n * 15 * 8))) != GSPH_OK) return st;
    for (int k = 1; k < every && k < N; ++k)
        if ((st = from_cuda(mem.get((void **)&seg[k], sb))) != GSPH_OK) return st;
    {
        std::vector<double> l0((size_t)n, 0.0);
        for (int64_t i = 0; i < n; ++i)
            if (ids[i] < (uint32_t)n && obs[ids[i]]) l0[i] = 1.0 / (double)cnt;
        GSPH_CK(cudaMemsetAsync(lam, 0, (size_t)n * 15 * 8, s));
        GSPH_CK(cudaMemcpyAsync(lam + (size_t)FVZ * n, l0.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        GSPH_CK(cudaStreamSynchronize(s));
    }
    // the FP64 context of the reverse steps (diagnostics: the step's FP64 rates)
    gsph_config hc = c->cfg;
    hc.precision = GSPH_FP64;
    hc.diagnostics = 1;
    hc.overlap = 0;
    hc.swap_period = 0;
    gsph_ctx *hctx = nullptr;
    if ((st = gsph_create(&hc, &hctx)) != GSPH_OK) return st;
    struct Guard { gsph_ctx *h; ~Guard() { gsph_destroy(h); } } guard{hctx};
    {
        cudaError_t e = alloc_all(hctx, n);
        if (e != cudaSuccess) return from_cuda(e);
        hctx->n = n;
    }
    double gY = 0.0, gG = 0.0;
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
        const int k0 = sgi * every, k1 = k0 + every < N ? k0 + every : N;
        seg[0] = ck[sgi];
        if ((st = gsph_load_state(c, ck[sgi], sb, 1, stream)) != GSPH_OK) return st;
        for (int k = k0; k < k1 - 1; ++k) {   // recompute the segment's states with the schedule
            if ((st = gsph_set_dt(c, dts[k], stream)) != GSPH_OK) return st;
            if ((st = enqueue_step(c, s)) != GSPH_OK) return st;
            if ((st = gsph_save_state(c, seg[k - k0 + 1], sb, 1, stream)) != GSPH_OK) return st;
        }
        for (int k = k1 - 1; k >= k0; --k) {
            if ((st = gsph_load_state(hctx, seg[k - k0], sb, 1, stream)) != GSPH_OK) return st;
            double g2[2] = {0.0, 0.0};
            if ((st = gsph_adjoint_step(hctx, lam, lamp, dts[k], g2, stream)) != GSPH_OK) return st;
            gY += g2[0];
            gG += g2[1];
            double *t = lam; lam = lamp; lamp = t;
        }
    }
    // dJ/dv0 through the initial state: v_z = v0 and E = |v|^2 / 2 + e, dE/dv0 = v_z
    {
        std::vector<double> lvz((size_t)n), lE((size_t)n), vz0((size_t)n);
        size_t off[19];
        state_layout(n, false, off);
        GSPH_CK(cudaMemcpyAsync(lvz.data(), lam + (size_t)FVZ * n, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
        GSPH_CK(cudaMemcpyAsync(lE.data(), lam + (size_t)FE * n, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
        GSPH_CK(cudaMemcpyAsync(vz0.data(), ck[0] + off[FVZ], (size_t)n * 8, cudaMemcpyDeviceToHost, s));
        GSPH_CK(cudaStreamSynchronize(s));
        double gv = 0.0;
        for (int64_t i = 0; i < n; ++i) gv += lvz[i] + lE[i] * vz0[i];
        grad[0] = gY;
        grad[1] = gG;
        grad[2] = gv;
    }
    return gsph_load_state(c, fin, sb, 1, stream);
}

// ---------------------------------------------------------------------------------------------
// Failure-detection hooks (tests)
// ---------------------------------------------------------------------------------------------
gsph_status gsph_set_wait_limit(gsph_ctx *c, uint32_t spin_limit, uint32_t extra_blocks) {
    if (!c || extra_blocks > 1) return GSPH_INVALID_ARG;
    c->wait_spin = spin_limit;
    c->wait_extra = extra_blocks;
    return GSPH_OK;
}

void gsph_debug_fail_alloc(int32_t k) { g_alloc_fail_at = k > 0 ? k : 0; }
