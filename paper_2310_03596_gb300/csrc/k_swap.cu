// k_swap.cu - the communication-load-balancing heuristic (Sec. III.A, III.B) on K virtual labels.
//
// For each particle type (one pass over all particles when the scene has one material) and each
// label pair (a, b) in lexicographic order:
//   Cg of a and b from exact fixed-point sums (positions clamped to the grid box, scaled to
//   [0, 2^32] and truncated, summed in int64), biased towards the label's all-types Cg by alpha when
//   there are several types (Sec. III.B);
//   balancing hash of every particle of a w.r.t. b and of b w.r.t. a (0 on the own side of the
//   middle of the Cg segment, 1000 beyond the other Cg, floor(1000 t / half-distance) in between,
//   at least 1), with every product and sum rounded separately;
//   n = min(#positive on each side); the n largest hashes of each side swap labels, ties broken by
//   the lowest persistent id (a 1001-bin histogram finds the threshold hash, a 3 x 9-bit radix
//   select on ids finds the id threshold inside the threshold bin);
//   the fixed-point sums are updated with the moved particles (exactly, so the next pair sees the
//   same Cg as a recomputation).
// Everything stays on the device: no host synchronisation inside a pass.
#include "gsph_internal.cuh"

namespace gsph {

constexpr int SW_BINS = GSPH_BALANCE_HASH_MAX + 1;
constexpr int SW_ID_BITS = 9;
constexpr int SW_ID_BINS = 1 << SW_ID_BITS;
constexpr int SW_THREADS = 256;

struct SwapPair {
    double own[2][3];           // side 0 = label a, side 1 = label b: own Cg' and the other's Cg'
    double oth[2][3];
    int active;
    int a, b, type;             // type -1: all particles
    unsigned long long nsel;    // particles swapped each way
    uint32_t hist[2][SW_BINS];
    uint32_t idh[2][SW_ID_BINS];
    int T[2];                   // threshold hash
    uint32_t need[2];           // still to take from the threshold bin
    uint32_t idpre[2];          // id prefix found so far
    int idsel[2];               // 1: the threshold bin is split, ids decide
};

struct SwapScratch {
    long long sums[kMaxLabel][kMaxMat + 1][3];
    long long cnt[kMaxLabel][kMaxMat + 1];
    unsigned long long moved;
};

// Exact fixed-point coordinate: clamp to [lo, lo + ext], scale by 2^32 / ext, truncate.
__device__ __forceinline__ long long quantise(double x, double lo, double hi, double sc) {
    double xc = fmin(fmax(x, lo), hi);
    double t = __dmul_rn(__dsub_rn(xc, lo), sc);
    return (long long)t;
}

struct QuantParams {
    double lo[3], hi[3], sc[3], inv[3];
};

__global__ void k_cg_sums(int64_t n, QuantParams Q, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const uint8_t *__restrict__ lab,
                          const uint8_t *__restrict__ mat, int nt, SwapScratch *__restrict__ S) {
    __shared__ long long sh[kMaxLabel][kMaxMat + 1][4];
    for (int i = threadIdx.x; i < kMaxLabel * (kMaxMat + 1) * 4; i += blockDim.x) (&sh[0][0][0])[i] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int l = lab[i] & (kMaxLabel - 1);
        int t = nt > 0 ? (mat[i] < nt ? mat[i] : 0) : -1;
        long long q0 = quantise(x[i], Q.lo[0], Q.hi[0], Q.sc[0]);
        long long q1 = quantise(y[i], Q.lo[1], Q.hi[1], Q.sc[1]);
        long long q2 = quantise(z[i], Q.lo[2], Q.hi[2], Q.sc[2]);
        const int all = kMaxMat;
        atomicAdd((unsigned long long *)&sh[l][all][0], (unsigned long long)q0);
        atomicAdd((unsigned long long *)&sh[l][all][1], (unsigned long long)q1);
        atomicAdd((unsigned long long *)&sh[l][all][2], (unsigned long long)q2);
        atomicAdd((unsigned long long *)&sh[l][all][3], 1ull);
        if (t >= 0) {
            atomicAdd((unsigned long long *)&sh[l][t][0], (unsigned long long)q0);
            atomicAdd((unsigned long long *)&sh[l][t][1], (unsigned long long)q1);
            atomicAdd((unsigned long long *)&sh[l][t][2], (unsigned long long)q2);
            atomicAdd((unsigned long long *)&sh[l][t][3], 1ull);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kMaxLabel * (kMaxMat + 1); k += blockDim.x) {
        int l = k / (kMaxMat + 1), t = k % (kMaxMat + 1);
        if (sh[l][t][3] == 0) continue;
        for (int a = 0; a < 3; ++a) atomicAdd((unsigned long long *)&S->sums[l][t][a], (unsigned long long)sh[l][t][a]);
        atomicAdd((unsigned long long *)&S->cnt[l][t], (unsigned long long)sh[l][t][3]);
    }
}

__device__ __forceinline__ void cg_of(const QuantParams &Q, const long long *sum, long long cnt, double cg[3]) {
    for (int a = 0; a < 3; ++a) {
        double mean = __ddiv_rn((double)sum[a], (double)cnt);
        cg[a] = __dadd_rn(Q.lo[a], __dmul_rn(mean, Q.inv[a]));
    }
}

__global__ void k_pair_setup(QuantParams Q, double alpha, int multi, int a, int b, int type,
                             const SwapScratch *__restrict__ S, SwapPair *__restrict__ pr) {
    const int slot = type >= 0 ? type : kMaxMat;
    pr->a = a;
    pr->b = b;
    pr->type = type;
    pr->active = 0;
    long long na = S->cnt[a][slot], nb = S->cnt[b][slot];
    if (na == 0 || nb == 0) return;
    double ca[3], cb[3];
    cg_of(Q, S->sums[a][slot], na, ca);
    cg_of(Q, S->sums[b][slot], nb, cb);
    if (multi) {
        double aa[3], ab[3];
        cg_of(Q, S->sums[a][kMaxMat], S->cnt[a][kMaxMat], aa);
        cg_of(Q, S->sums[b][kMaxMat], S->cnt[b][kMaxMat], ab);
        double beta = __dsub_rn(1.0, alpha);
        for (int k = 0; k < 3; ++k) {
            ca[k] = __dadd_rn(__dmul_rn(alpha, aa[k]), __dmul_rn(beta, ca[k]));
            cb[k] = __dadd_rn(__dmul_rn(alpha, ab[k]), __dmul_rn(beta, cb[k]));
        }
    }
    for (int k = 0; k < 3; ++k) {
        pr->own[0][k] = ca[k]; pr->oth[0][k] = cb[k];
        pr->own[1][k] = cb[k]; pr->oth[1][k] = ca[k];
    }
    pr->active = 1;
}

// Balancing hash of position p for a particle owned by the label with Cg `own`, w.r.t. `oth`.
__device__ __forceinline__ int balancing_hash(const double own[3], const double oth[3], double p0, double p1,
                                              double p2) {
    double M[3], d[3];
    for (int k = 0; k < 3; ++k) {
        M[k] = __dmul_rn(__dadd_rn(own[k], oth[k]), 0.5);
        d[k] = __dsub_rn(oth[k], own[k]);
    }
    double dn = __dsqrt_rn(dist2_rn(d[0], d[1], d[2]));
    if (!(dn > 0.0)) return 0;
    double ell = __dmul_rn(dn, 0.5);
    double t = __dadd_rn(__dadd_rn(__dmul_rn(__dsub_rn(p0, M[0]), d[0]), __dmul_rn(__dsub_rn(p1, M[1]), d[1])),
                         __dmul_rn(__dsub_rn(p2, M[2]), d[2]));
    t = __ddiv_rn(t, dn);
    if (!(t > 0.0)) return 0;
    if (t >= ell) return GSPH_BALANCE_HASH_MAX;
    double k = floor(__ddiv_rn(__dmul_rn(1000.0, t), ell));
    int h = (int)k;
    h = h < 1 ? 1 : h;
    h = h > GSPH_BALANCE_HASH_MAX ? GSPH_BALANCE_HASH_MAX : h;
    return h;
}

__device__ __forceinline__ int side_of(const SwapPair &pr, uint8_t lab, uint8_t mat) {
    if (pr.type >= 0 && mat != pr.type) return -1;
    if (lab == pr.a) return 0;
    if (lab == pr.b) return 1;
    return -1;
}

__global__ void __launch_bounds__(SW_THREADS) k_bhash(int64_t n, const double *__restrict__ x,
                                                      const double *__restrict__ y, const double *__restrict__ z,
                                                      const uint8_t *__restrict__ lab, const uint8_t *__restrict__ mat,
                                                      SwapPair *__restrict__ pr, uint16_t *__restrict__ bh) {
    __shared__ uint32_t hs[2][SW_BINS];
    __shared__ double own[2][3], oth[2][3];
    __shared__ int act;
    if (threadIdx.x == 0) act = pr->active;
    if (threadIdx.x < 6) {
        int sd = threadIdx.x / 3, k = threadIdx.x % 3;
        own[sd][k] = pr->own[sd][k];
        oth[sd][k] = pr->oth[sd][k];
    }
    for (int i = threadIdx.x; i < 2 * SW_BINS; i += SW_THREADS) (&hs[0][0])[i] = 0;
    __syncthreads();
    if (!act) return;
    const int a = pr->a, b = pr->b, type = pr->type;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint8_t l = lab[i];
        int sd = -1;
        if (type < 0 || mat[i] == type) sd = (l == a) ? 0 : ((l == b) ? 1 : -1);
        if (sd >= 0) {
            int hv = balancing_hash(own[sd], oth[sd], x[i], y[i], z[i]);
            bh[i] = (uint16_t)hv;
            atomicAdd(&hs[sd][hv], 1u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * SW_BINS; k += SW_THREADS) {
        uint32_t v = (&hs[0][0])[k];
        if (v) atomicAdd(&(&pr->hist[0][0])[k], v);
    }
}

// One block: n = min(#positive), then for each side the threshold hash and how many to take from
// the threshold bin (histograms staged in shared memory, scanned by one thread).
__global__ void __launch_bounds__(1024) k_select(SwapPair *__restrict__ pr) {
    __shared__ uint32_t hs[2][SW_BINS];
    if (!pr->active) return;
    for (int k = threadIdx.x; k < 2 * SW_BINS; k += blockDim.x) (&hs[0][0])[k] = (&pr->hist[0][0])[k];
    __syncthreads();
    if (threadIdx.x != 0) return;
    uint64_t pos[2];
    for (int sd = 0; sd < 2; ++sd) {
        uint64_t c = 0;
        for (int hv = 1; hv < SW_BINS; ++hv) c += hs[sd][hv];
        pos[sd] = c;
    }
    uint64_t m = pos[0] < pos[1] ? pos[0] : pos[1];
    pr->nsel = m;
    if (m == 0) {
        pr->active = 0;
        return;
    }
    for (int sd = 0; sd < 2; ++sd) {
        uint64_t above = 0;
        int T = GSPH_BALANCE_HASH_MAX;
        for (; T >= 1; --T) {
            if (above + hs[sd][T] >= m) break;
            above += hs[sd][T];
        }
        pr->T[sd] = T;
        pr->need[sd] = (uint32_t)(m - above);
        pr->idsel[sd] = pr->need[sd] < hs[sd][T];
        pr->idpre[sd] = 0;
    }
}

// Radix select on persistent ids inside the threshold bin: histogram of id digit `pass` (9 bits,
// most significant first) among the candidates whose higher digits match the prefix so far.
__global__ void __launch_bounds__(SW_THREADS) k_idhist(int64_t n, const uint8_t *__restrict__ lab,
                                                       const uint8_t *__restrict__ mat,
                                                       const uint32_t *__restrict__ id,
                                                       const uint16_t *__restrict__ bh, SwapPair *__restrict__ pr,
                                                       int pass) {
    __shared__ uint32_t hs[2][SW_ID_BINS];
    __shared__ int need_any;
    if (threadIdx.x == 0) need_any = pr->active && (pr->idsel[0] || pr->idsel[1]);
    for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) (&hs[0][0])[k] = 0;
    __syncthreads();
    if (!need_any) return;
    const int shift = 18 - SW_ID_BITS * pass;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int sd = side_of(*pr, lab[i], mat[i]);
        if (sd >= 0 && pr->idsel[sd] && bh[i] == pr->T[sd]) {
            uint32_t v = id[i];
            if ((v >> (shift + SW_ID_BITS)) == (pr->idpre[sd] >> (shift + SW_ID_BITS)))
                atomicAdd(&hs[sd][(v >> shift) & (SW_ID_BINS - 1)], 1u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) {
        uint32_t v = (&hs[0][0])[k];
        if (v) atomicAdd(&(&pr->idh[0][0])[k], v);
    }
}

__global__ void __launch_bounds__(SW_ID_BINS) k_idselect(SwapPair *__restrict__ pr, int pass) {
    __shared__ uint32_t hs[2][SW_ID_BINS];
    if (!pr->active) return;
    for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += blockDim.x) {
        (&hs[0][0])[k] = (&pr->idh[0][0])[k];
        (&pr->idh[0][0])[k] = 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int shift = 18 - SW_ID_BITS * pass;
    for (int sd = 0; sd < 2; ++sd) {
        if (!pr->idsel[sd]) continue;
        uint32_t need = pr->need[sd], below = 0;
        int d = 0;
        for (; d < SW_ID_BINS - 1; ++d) {
            if (below + hs[sd][d] >= need) break;
            below += hs[sd][d];
        }
        pr->idpre[sd] |= (uint32_t)d << shift;
        pr->need[sd] = need - below;
    }
}

// Label exchange and exact update of the fixed-point sums.
__global__ void __launch_bounds__(SW_THREADS) k_apply(int64_t n, QuantParams Q, const double *__restrict__ x,
                                                      const double *__restrict__ y, const double *__restrict__ z,
                                                      uint8_t *__restrict__ lab, const uint8_t *__restrict__ mat,
                                                      const uint32_t *__restrict__ id,
                                                      const uint16_t *__restrict__ bh, SwapPair *__restrict__ pr,
                                                      SwapScratch *__restrict__ S, int nt) {
    if (!pr->active) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int sd = side_of(*pr, lab[i], mat[i]);
    if (sd < 0) return;
    int hv = bh[i];
    bool take = hv > pr->T[sd] || (hv == pr->T[sd] && (!pr->idsel[sd] || id[i] <= pr->idpre[sd]));
    if (hv == 0 || !take) return;
    int from = sd == 0 ? pr->a : pr->b, to = sd == 0 ? pr->b : pr->a;
    lab[i] = (uint8_t)to;
    long long q[3] = {quantise(x[i], Q.lo[0], Q.hi[0], Q.sc[0]), quantise(y[i], Q.lo[1], Q.hi[1], Q.sc[1]),
                      quantise(z[i], Q.lo[2], Q.hi[2], Q.sc[2])};
    int t = nt > 0 ? (mat[i] < nt ? mat[i] : 0) : -1;
    for (int k = 0; k < 3; ++k) {
        atomicAdd((unsigned long long *)&S->sums[from][kMaxMat][k], (unsigned long long)(-q[k]));
        atomicAdd((unsigned long long *)&S->sums[to][kMaxMat][k], (unsigned long long)q[k]);
        if (t >= 0) {
            atomicAdd((unsigned long long *)&S->sums[from][t][k], (unsigned long long)(-q[k]));
            atomicAdd((unsigned long long *)&S->sums[to][t][k], (unsigned long long)q[k]);
        }
    }
    atomicAdd((unsigned long long *)&S->cnt[from][kMaxMat], (unsigned long long)(-1ll));
    atomicAdd((unsigned long long *)&S->cnt[to][kMaxMat], 1ull);
    if (t >= 0) {
        atomicAdd((unsigned long long *)&S->cnt[from][t], (unsigned long long)(-1ll));
        atomicAdd((unsigned long long *)&S->cnt[to][t], 1ull);
    }
    atomicAdd(&S->moved, 1ull);
}

// ---------------------------------------------------------------------------------------------
// Host side: one full pass.
// ---------------------------------------------------------------------------------------------
size_t swap_scratch_bytes(int K, int nmat) {
    int ntype = nmat > 1 ? nmat : 1;
    size_t npairs = (size_t)ntype * (size_t)(K * (K - 1) / 2);
    return sizeof(SwapScratch) + (npairs > 0 ? npairs : 1) * sizeof(SwapPair);
}

QuantParams quant_params(const DevParams &P) {
    QuantParams Q;
    for (int a = 0; a < 3; ++a) {
        double ext = (double)P.dims[a] * P.cell;
        Q.lo[a] = P.lo[a];
        Q.hi[a] = P.lo[a] + ext;
        Q.sc[a] = 4294967296.0 / ext;
        Q.inv[a] = ext / 4294967296.0;
    }
    return Q;
}

// scratch: swap_scratch_bytes() device bytes; bh: n uint16. moved_out (device) receives the number of
// particles that changed label.
cudaError_t launch_swap_pass(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                             uint8_t *lab, const uint8_t *mat, const uint32_t *id, void *scratch, uint16_t *bh,
                             cudaStream_t s) {
    if (n <= 0 || P.K_labels < 2) return cudaSuccess;
    const int K = P.K_labels;
    const int multi = P.nmat > 1;
    const int ntype = multi ? P.nmat : 1;
    const size_t bytes = swap_scratch_bytes(K, P.nmat);
    cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e != cudaSuccess) return e;
    SwapScratch *S = (SwapScratch *)scratch;
    SwapPair *pairs = (SwapPair *)((char *)scratch + sizeof(SwapScratch));
    QuantParams Q = quant_params(P);
    unsigned g = (unsigned)((n + SW_THREADS - 1) / SW_THREADS);
    k_cg_sums<<<g, SW_THREADS, 0, s>>>(n, Q, x, y, z, lab, mat, multi ? P.nmat : 0, S);
    int idx = 0;
    for (int T = 0; T < ntype; ++T) {
        int type = multi ? T : -1;
        for (int a = 0; a < K - 1; ++a)
            for (int b = a + 1; b < K; ++b, ++idx) {
                SwapPair *pr = pairs + idx;
                k_pair_setup<<<1, 1, 0, s>>>(Q, P.alpha, multi, a, b, type, S, pr);
                k_bhash<<<g, SW_THREADS, 0, s>>>(n, x, y, z, lab, mat, pr, bh);
                k_select<<<1, 1024, 0, s>>>(pr);
                for (int pass = 0; pass < 3; ++pass) {
                    k_idhist<<<g, SW_THREADS, 0, s>>>(n, lab, mat, id, bh, pr, pass);
                    k_idselect<<<1, SW_ID_BINS, 0, s>>>(pr, pass);
                }
                k_apply<<<g, SW_THREADS, 0, s>>>(n, Q, x, y, z, lab, mat, id, bh, pr, S, multi ? P.nmat : 0);
            }
    }
    return cudaGetLastError();
}

// Number of particles moved by the last pass (device pointer into the scratch).
unsigned long long *swap_moved_ptr(void *scratch) { return &((SwapScratch *)scratch)->moved; }

}  // namespace gsph
