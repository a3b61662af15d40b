// k_swap.cu - the communication-load-balancing heuristic (Sec. III.A, III.B) on K virtual labels.
//
// One swap pass is two streaming kernels (the fixed-point sums; the speculative counts, each block
// forming the pass-start pair geometries itself) and one cooperative kernel (all blocks resident) for the
// sequential pair loop, whose phases are
// separated by a bounded grid barrier; a barrier that does not complete within about a second records a
// timeout in the error word and the pass returns. For each particle type (one pass over all particles when the scene
// has one material) and each label pair (a, b) in lexicographic order:
//   Cg of a and b from exact fixed-point sums (per axis the nearest integer to (x - lo) 2^32 / L of the
//   FP64 position, L the grid extent, clamped to [0, 2^32 - 1] and summed in int64; Cg = lo + mean L 2^-32),
//   biased towards the label's all-types Cg by alpha when there are several types (Sec. III.B). Every
//   block derives the pair's geometry (FP64) from the sums itself, a few threads in parallel, with the
//   same operations, so no block waits for another to publish it;
//   balancing hash of every particle of a w.r.t. b and of b w.r.t. a (0 on the own side of the
//   middle of the Cg segment, 1000 beyond the other Cg, floor(1000 t / half-distance) in between, at
//   least 1), defined in FP64. Each particle evaluates it first in FP32 from the FP32 roundings of its
//   position and of the pair geometry, with a bound of the FP32 value's distance from the FP64 one; only
//   a particle whose interval reaches a decision boundary (an integer hash, the middle, the other Cg)
//   evaluates the FP64 sequence from its FP64 position;
//   n = min(#positive on each side); the n largest hashes of each side swap labels, ties broken by
//   the lowest persistent id. A 1001-bin histogram finds the threshold hash. When the threshold bin
//   holds more particles than are needed, the exchange pass collects that bin into a short list, and
//   every block finds the id threshold by a 3 x 9-bit radix select over the list in shared memory
//   (the block owning a listed slot applies its swap); a bin larger than the list capacity is split
//   by the same radix select run over all particles with a grid barrier per digit;
//   the fixed-point sums are updated with the moved particles (exactly, so the next pair sees the
//   same Cg as a recomputation).
// Before the pairs, one speculative sweep counts every pair's positive hashes at the pass-start
// state; the pairs before the first one with positives on both sides change nothing and are skipped.
// With 8 or more labels the same sweep groups the slots by label, and each pair then visits only its
// two labels' slots (the segments keep their sizes since a pair's swaps are 1:1; the moved particles
// exchange their segment positions after the pair).
#include <cuda/atomic>

#include "gsph_internal.cuh"

namespace gsph {

constexpr int SW_BINS = GSPH_BALANCE_HASH_MAX + 1;
constexpr int SW_ID_BITS = 9;
constexpr int SW_ID_BINS = 1 << SW_ID_BITS;
constexpr int SW_THREADS = 512;
constexpr int SW_NT = kMaxMat + 1;   // per-type slots + the all-types slot
constexpr int SW_TCAP = 2048;        // threshold-bin list capacity per side
constexpr int SW_MAXCOMBO = kMaxMat * (kMaxLabel * (kMaxLabel - 1) / 2);   // (type, label pair) combinations
constexpr int SW_SBUF = 2 * SW_TCAP * 4;

struct SwapPair {
    uint32_t hist[2][SW_BINS];
    uint32_t npos[2];                // particles with a positive hash per side
    uint32_t spec[2];                // the same at the pass-start labels and sums (speculative pass)
    uint32_t idh[3][2][SW_ID_BINS];
    uint32_t tcnt[2];                // threshold-bin list fill per side
    uint32_t mvcnt[2];               // particles moved per side (their label-segment positions listed)
    unsigned long long moved;
};

struct SwapScratch {
    long long sums[kMaxLabel][SW_NT][3];
    long long cnt[kMaxLabel][SW_NT];
    unsigned long long lcur[kMaxLabel];   // fill of each label's segment (pass start)
    unsigned long long moved;
    unsigned long long fp64;              // balancing hashes the FP32 bound left to the FP64 sequence
    unsigned int bar_count;
    unsigned int bar_gen;
};

// Fixed-point Cg per axis: q = nearest integer (ties to even) to (x - lo) s, s = 2^32 / L, clamped to
// [0, 2^32 - 1]; Cg = lo + (sum / count) step, step = L 2^-32 (L: the grid extent).
struct QuantParams {
    double lo[3], s[3], step[3];
};

// Pair geometry for one side, FP64 (the definition) and its FP32 roundings (the fast path): middle M,
// direction d from the own Cg' to the other, |d| and the half-distance ell; unit direction u = d / |d|
// and scale 1000 / ell in FP32.
struct SideF {
    float M[3];
    float u[3];
    float scale;
};
struct Side {
    SideF f;
    double M[3], d[3], dn, ell;
};

// Geometry of label pair (a, b) of one type from the current sums, by one thread with the operations of
// the per-pair code (every rounding explicit, so the values are the same bits), for side a. Returns false
// when a side is empty or the two Cgs coincide.
__device__ bool combo_geometry(const SwapScratch *S, const QuantParams &Q, double alpha, bool multi, int slot, int a,
                               int b, Side &sd) {
    const int lab[2] = {a, b};
    double cg[4][3];
    long long cn[4];
    for (int w = 0; w < 4; ++w) {
        const int l = lab[w & 1], sl = w < 2 ? slot : kMaxMat;
        cn[w] = ((volatile const long long *)&S->cnt[l][sl])[0];
        if ((w < 2 || multi) && cn[w] > 0)
            for (int ax = 0; ax < 3; ++ax) {
                const long long sm = ((volatile const long long *)&S->sums[l][sl][ax])[0];
                const double mean = __ddiv_rn(__ll2double_rn(sm), __ll2double_rn(cn[w]));
                cg[w][ax] = __dadd_rn(Q.lo[ax], __dmul_rn(mean, Q.step[ax]));
            }
    }
    if (!(cn[0] > 0 && cn[1] > 0)) return false;
    for (int ax = 0; ax < 3; ++ax) {
        double ca = cg[0][ax], cb = cg[1][ax];
        if (multi) {
            const double beta = __dsub_rn(1.0, alpha);
            ca = __dadd_rn(__dmul_rn(alpha, cg[2][ax]), __dmul_rn(beta, ca));
            cb = __dadd_rn(__dmul_rn(alpha, cg[3][ax]), __dmul_rn(beta, cb));
        }
        sd.M[ax] = __dmul_rn(__dadd_rn(ca, cb), 0.5);
        sd.f.M[ax] = (float)sd.M[ax];
        sd.d[ax] = __dsub_rn(cb, ca);
    }
    sd.dn = __dsqrt_rn(dist2_rn(sd.d[0], sd.d[1], sd.d[2]));
    if (!(sd.dn > 0.0)) return false;
    sd.ell = __dmul_rn(sd.dn, 0.5);
    for (int ax = 0; ax < 3; ++ax) sd.f.u[ax] = (float)__ddiv_rn(sd.d[ax], sd.dn);
    sd.f.scale = (float)__ddiv_rn(1000.0, sd.ell);
    return true;
}

// The balancing hash in FP64, each operation rounded: t = ((e0 d0 + e1 d1) + e2 d2) / |d| with e = x - M;
// 0 when t <= 0, 1000 when t >= ell, else floor(1000 t / ell) clamped to [1, 1000].
__device__ int balancing_hash64(const double M[3], const double d[3], double dn, double ell, double X, double Y,
                                double Z) {
    const double a0 = __dmul_rn(__dsub_rn(X, M[0]), d[0]);
    const double a1 = __dmul_rn(__dsub_rn(Y, M[1]), d[1]);
    const double a2 = __dmul_rn(__dsub_rn(Z, M[2]), d[2]);
    const double t = __ddiv_rn(__dadd_rn(__dadd_rn(a0, a1), a2), dn);
    if (!(t > 0.0)) return 0;
    if (t >= ell) return GSPH_BALANCE_HASH_MAX;
    const double k = floor(__ddiv_rn(__dmul_rn(1000.0, t), ell));
    if (k < 1.0) return 1;
    if (k >= (double)GSPH_BALANCE_HASH_MAX) return GSPH_BALANCE_HASH_MAX;
    return (int)k;
}

// The balancing hash from the FP32 roundings, or -1 when FP32 cannot decide it. v = t scale carries the
// roundings of the position, the middle, the direction and the scale and of each operation; B bounds
// |v - V| for the FP64 value V = 1000 t / ell (twice the first-order bound plus 8 ulp of v, which covers
// the second-order terms, the FP64 sequence's own roundings and those of the bound). V lies in
// [v - B, v + B]: below 0 the hash is 0, above 1000.5 it is 1000 (V <= 1000 (1 + 2^-52) while t < ell),
// and inside [k, k + 1) with k <= 998 it is max(k, 1) (V < 999 means t < ell).
__device__ __forceinline__ int balancing_hash_fast(const SideF &g, float p0, float p1, float p2) {
    const float e0 = __fsub_rn(p0, g.M[0]), e1 = __fsub_rn(p1, g.M[1]), e2 = __fsub_rn(p2, g.M[2]);
    const float a0 = __fmul_rn(e0, g.u[0]), a1 = __fmul_rn(e1, g.u[1]), a2 = __fmul_rn(e2, g.u[2]);
    const float t = __fadd_rn(__fadd_rn(a0, a1), a2);
    const float v = __fmul_rn(t, g.scale);
    const float S = fabsf(a0) + fabsf(a1) + fabsf(a2);
    const float X = fabsf(g.u[0]) * (fabsf(p0) + fabsf(g.M[0])) + fabsf(g.u[1]) * (fabsf(p1) + fabsf(g.M[1])) +
                    fabsf(g.u[2]) * (fabsf(p2) + fabsf(g.M[2]));
    const float B = 0x1p-23f * g.scale * (X + 5.0f * S) + 0x1p-21f * fabsf(v);
    const float lo = v - B, hi = v + B;
    if (hi < 0.0f) return 0;
    if (lo > 1000.5f) return GSPH_BALANCE_HASH_MAX;
    if (lo > 0.0f && hi < 999.0f) {
        const float k = floorf(lo);
        if (k == floorf(hi)) return k < 1.0f ? 1 : (int)k;
    }
    return -1;
}

// Sum of a non-negative 33-bit value over the lanes of `peers` (lanes sharing one key), exact: the
// low 16 and high 17 bits are reduced separately in 32-bit arithmetic (at most 32 lanes).
__device__ __forceinline__ long long group_sum33(unsigned peers, long long v) {
    const unsigned lo = __reduce_add_sync(peers, (unsigned)(v & 0xffff));
    const unsigned hi = __reduce_add_sync(peers, (unsigned)(v >> 16));
    return (long long)lo + ((long long)hi << 16);
}

// Adds (q0, q1, q2, 1) of every lane to sh[key] with one shared atomic per distinct key in the warp.
// Lanes with valid = false contribute nothing (their key may be anything).
__device__ __forceinline__ void warp_add_sums(long long (*sh)[4], int key, bool valid, long long q0, long long q1,
                                              long long q2) {
    const unsigned peers = __match_any_sync(kFullMask, valid ? key : -1);
    const long long s0 = group_sum33(peers, valid ? q0 : 0), s1 = group_sum33(peers, valid ? q1 : 0);
    const long long s2 = group_sum33(peers, valid ? q2 : 0);
    if (valid && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) {
        atomicAdd((unsigned long long *)&sh[key][0], (unsigned long long)s0);
        atomicAdd((unsigned long long *)&sh[key][1], (unsigned long long)s1);
        atomicAdd((unsigned long long *)&sh[key][2], (unsigned long long)s2);
        atomicAdd((unsigned long long *)&sh[key][3], (unsigned long long)__popc(peers));
    }
}

// Moves the sums of the particles that changed label (dsum[side] = q0 q1 q2 count; side 0 went a -> b,
// side 1 b -> a) into the global per-label (and per-type) fixed-point sums. Threads 0 and 1.
__device__ __forceinline__ void flush_moved(SwapScratch *S, const long long (*dsum)[4], int a, int b, int type) {
    if (threadIdx.x >= 2) return;
    const int sd = threadIdx.x;
    const int from = sd == 0 ? a : b, to = sd == 0 ? b : a;
    const long long c = dsum[sd][3];
    if (!c) return;
    for (int k = 0; k < 3; ++k) {
        const long long q = dsum[sd][k];
        atomicAdd((unsigned long long *)&S->sums[from][kMaxMat][k], (unsigned long long)(-q));
        atomicAdd((unsigned long long *)&S->sums[to][kMaxMat][k], (unsigned long long)q);
        if (type >= 0) {
            atomicAdd((unsigned long long *)&S->sums[from][type][k], (unsigned long long)(-q));
            atomicAdd((unsigned long long *)&S->sums[to][type][k], (unsigned long long)q);
        }
    }
    atomicAdd((unsigned long long *)&S->cnt[from][kMaxMat], (unsigned long long)(-c));
    atomicAdd((unsigned long long *)&S->cnt[to][kMaxMat], (unsigned long long)c);
    if (type >= 0) {
        atomicAdd((unsigned long long *)&S->cnt[from][type], (unsigned long long)(-c));
        atomicAdd((unsigned long long *)&S->cnt[to][type], (unsigned long long)c);
    }
    atomicAdd(&S->moved, (unsigned long long)c);
}

// In-place inclusive scan of a[0..nv) in shared memory by the whole block (nv <= 2 * SW_THREADS).
__device__ void block_inclusive_scan(uint32_t *a, int nv) {
    __shared__ uint32_t wt[SW_THREADS / 32];
    const int t = threadIdx.x, l = t & 31, w = t >> 5;
    const uint32_t x0 = 2 * t < nv ? a[2 * t] : 0u, x1 = 2 * t + 1 < nv ? a[2 * t + 1] : 0u;
    const uint32_t s2 = x0 + x1;
    uint32_t inc = s2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, inc, o);
        if (l >= o) inc += y;
    }
    if (l == 31) wt[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t v = l < SW_THREADS / 32 ? wt[l] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, v, o);
            if (l >= o) v += y;
        }
        if (l < SW_THREADS / 32) wt[l] = v;
    }
    __syncthreads();
    const uint32_t base = (w > 0 ? wt[w - 1] : 0u) + inc - s2;
    if (2 * t < nv) a[2 * t] = base + x0;
    if (2 * t + 1 < nv) a[2 * t + 1] = base + x0 + x1;
    __syncthreads();
}

// Bounded grid barrier (generation counter). Returns false, with the timeout bit set, when the
// other blocks do not arrive within the spin limit.
// Bounded wait of the swap pass's grid barrier: spin limit (iterations of about 64 ns) and blocks the
// barrier expects beyond those launched (0 in normal use; a failure-detection test makes the wait run
// out with 1 and a short limit).
struct WaitCfg {
    unsigned spin_limit;
    unsigned extra_blocks;
};

__device__ bool grid_barrier(SwapScratch *S, unsigned nblocks, int *err, const WaitCfg &wc) {
    nblocks += wc.extra_blocks;
    __shared__ int ok_sh;
    __threadfence();   // this thread's writes of the phase are visible device-wide before arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(S->bar_gen);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(S->bar_count);
        const unsigned g = gen.load(cuda::memory_order_acquire);
        int ok = 1;
        if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == nblocks - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.fetch_add(1u, cuda::memory_order_release);
        } else {
            unsigned it = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (++it > wc.spin_limit) {   // default 2^24: about a second with the back-off below
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// The pass's two streaming phases run as separate kernels at full occupancy; the cooperative kernel
// starts from their results and returns at once when no label pair can swap (the usual case once the
// labels have settled).
// Phase 1: exact fixed-point sums per (label, type) and per label (warp-aggregated shared atomics, one
// global atomic per non-zero entry and block).
__global__ void __launch_bounds__(SW_THREADS) k_swap_sums(int64_t n, int nmat, const SwapPos pos,
                                                          const uint8_t *__restrict__ lab,
                                                          const uint8_t *__restrict__ mat, SwapScratch *__restrict__ S) {
    pdl_wait();      // launched after the reorder as a programmatic dependent launch
    pdl_release();
    __shared__ long long shs[kMaxLabel][SW_NT][4];
    const bool multi = nmat > 1;
    const int64_t gstride = (int64_t)gridDim.x * SW_THREADS;
    for (int i = threadIdx.x; i < kMaxLabel * SW_NT * 4; i += SW_THREADS) (&shs[0][0][0])[i] = 0;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * SW_THREADS; base < n; base += gstride) {
        const int64_t i = base + threadIdx.x;
        const bool v = i < n;
        const int l = v ? (lab[i] & (kMaxLabel - 1)) : 0;
        const int t = (v && multi) ? (mat[i] < nmat ? mat[i] : 0) : 0;
        long long q0 = 0, q1 = 0, q2 = 0;
        if (v) {
            q0 = pos.qx[i];
            q1 = pos.qy[i];
            q2 = pos.qz[i];
        }
        long long(*flat)[4] = &shs[0][0];
        warp_add_sums(flat, l * SW_NT + kMaxMat, v, q0, q1, q2);
        if (multi) warp_add_sums(flat, l * SW_NT + t, v, q0, q1, q2);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kMaxLabel * SW_NT; k += SW_THREADS) {
        const int l = k / SW_NT, t = k % SW_NT;
        if (shs[l][t][3] == 0) continue;
        for (int a = 0; a < 3; ++a) atomicAdd((unsigned long long *)&S->sums[l][t][a], (unsigned long long)shs[l][t][a]);
        atomicAdd((unsigned long long *)&S->cnt[l][t], (unsigned long long)shs[l][t][3]);
    }
}

// The balancing hash of one particle by the FP64 sequence: the pair's FP64 geometry from the sums, the
// direction flipped for a particle of label b.
__device__ __forceinline__ int spec_hash64(const SwapScratch *S, const QuantParams &Q, double alpha, bool multi, int T,
                                        int a, int b, bool flip, double X, double Y, double Z) {
    Side G;
    combo_geometry(S, Q, alpha, multi, T, a, b, G);
    if (flip) { G.d[0] = -G.d[0]; G.d[1] = -G.d[1]; G.d[2] = -G.d[2]; }
    atomicAdd((unsigned long long *)&S->fp64, 1ull);
    return balancing_hash64(G.M, G.d, G.dn, G.ell, X, Y, Z);
}

// Phase 2 (exact speculative pass): positive-hash counts of every (type, label pair) at the pass-start
// labels and sums. A pair with no positive hash on one side swaps nothing and changes nothing, so the
// sequential loop starts at the first pair with positive hashes on both sides: until then the labels and
// sums each pair sees are the pass-start ones, the state this pass evaluates. With 8 or more labels the
// same sweep groups the slots by label (the label segments of the pair loop).
__global__ void __launch_bounds__(SW_THREADS, 2) k_swap_spec(int64_t n, QuantParams Q, double alpha, int K, int nmat,
                                                          const SwapPos pos, const uint8_t *__restrict__ lab,
                                                          const uint8_t *__restrict__ mat, SwapScratch *__restrict__ S,
                                                          SwapPair *__restrict__ pairs, uint32_t *__restrict__ sidx) {
    pdl_wait();      // launched after the sums as a programmatic dependent launch
    __shared__ SideF spec[SW_MAXCOMBO];
    __shared__ uint32_t scnt[2 * SW_MAXCOMBO];
    __shared__ long long loff_sh[kMaxLabel + 1];
    const bool multi = nmat > 1;
    const int npairs = K * (K - 1) / 2, ncombo = (multi ? nmat : 1) * npairs;
    const int64_t gstride = (int64_t)gridDim.x * SW_THREADS;
    const bool seg = K >= 8;
    // the pass-start geometry of every (type, label pair) from the sums, formed by each block (a few FP64
    // operations per pair) rather than by a separate one-block kernel
    for (int q = threadIdx.x; q < ncombo; q += SW_THREADS) {
        const int T = q / npairs;
        int a = 0, rem = q % npairs;
        while (rem >= K - 1 - a) { rem -= K - 1 - a; ++a; }
        Side g;
        SideF f;
        if (combo_geometry(S, Q, alpha, multi, multi ? T : kMaxMat, a, a + 1 + rem, g)) f = g.f;
        else f.scale = -1.0f;
        spec[q] = f;
        scnt[2 * q] = 0u;
        scnt[2 * q + 1] = 0u;
    }
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int l = 0; l < kMaxLabel; ++l) {
            loff_sh[l] = o;
            if (l < K) o += S->cnt[l][kMaxMat];
        }
        loff_sh[kMaxLabel] = o;
    }
    __syncthreads();
    uint32_t *const byl = sidx;
    for (int64_t base = (int64_t)blockIdx.x * SW_THREADS; base < n; base += gstride) {
        const int64_t i = base + threadIdx.x;
        const bool v = i < n;
        const int l = v ? (lab[i] & (kMaxLabel - 1)) : 0;
        const int T = (v && multi) ? (mat[i] < nmat ? mat[i] : 0) : 0;
        const float px = v ? pos.x[i] : 0.0f, py = v ? pos.y[i] : 0.0f, pz = v ? pos.z[i] : 0.0f;
        if (seg) {   // the slot's place in its label's segment (one atomic per label and warp)
            const unsigned peers = __match_any_sync(kFullMask, v ? l : -1);
            unsigned long long at = 0;
            if (v && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
                at = atomicAdd(&S->lcur[l], (unsigned long long)__popc(peers));
            at = __shfl_sync(kFullMask, at, __ffs(peers) - 1);
            if (v) byl[loff_sh[l] + (long long)at + __popc(peers & lanemask_lt())] = (uint32_t)i;
        }
        for (int o = 0; o < K; ++o) {   // the K - 1 pairs of the particle's label (warp-uniform loop)
            const int a = l < o ? l : o, b = l < o ? o : l;
            const int q = T * npairs + a * (2 * K - a - 1) / 2 + (b - a - 1);
            int key = -1;
            if (v && o != l) {
                SideF g = spec[q];
                if (g.scale >= 0.0f) {
                    if (l == b) { g.u[0] = -g.u[0]; g.u[1] = -g.u[1]; g.u[2] = -g.u[2]; }
                    int hv = balancing_hash_fast(g, px, py, pz);
                    if (hv < 0)   // rare: the FP64 sequence
                        hv = spec_hash64(S, Q, alpha, multi, multi ? T : kMaxMat, a, b, l == b, pos.X[i], pos.Y[i],
                                         pos.Z[i]);
                    if (hv > 0) key = 2 * q + (l == a ? 0 : 1);
                }
            }
            if (__any_sync(kFullMask, key >= 0)) {   // positives are rare once labels have settled
                const unsigned peers = __match_any_sync(kFullMask, key);
                if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
                    atomicAdd(&scnt[key], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * ncombo; q += SW_THREADS)
        if (scnt[q]) atomicAdd(&pairs[q >> 1].spec[q & 1], scnt[q]);
}

// Two blocks per SM (64 registers): the phases between grid barriers are latency-bound streams over the
// pair's particles, which more resident warps cover better (measured faster than one block per SM at
// 109 registers, with the same labels).
__global__ void __launch_bounds__(SW_THREADS, 2) k_swap_pass(int64_t n, QuantParams Q, double alpha, int K, int nmat,
                                                          const SwapPos pos, uint8_t *__restrict__ lab,
                                                          const uint8_t *__restrict__ mat,
                                                          const uint32_t *__restrict__ id, uint16_t *__restrict__ bh,
                                                          SwapScratch *__restrict__ S, SwapPair *__restrict__ pairs,
                                                          uint2 *__restrict__ tl, uint32_t *__restrict__ sidx,
                                                          int *__restrict__ err, const WaitCfg wc) {
    __shared__ uint32_t hs[2][SW_BINS];
    __shared__ uint32_t ids[2][SW_ID_BINS];
    __shared__ Side side_sh[2];
    __shared__ int act_sh;
    __shared__ long long gn_sh[4];       // counts of a, b (this type) and of a, b (all types)
    __shared__ uint32_t npos_sh[2];      // this block's positive hashes per side
    __shared__ double gcg_sh[4][3];      // their Cgs
    __shared__ double gd_sh[3], gdn_sh;  // Cg_b - Cg_a, its length
    __shared__ int T_sh[2], idsel_sh[2];
    __shared__ uint32_t need_sh[2], idpre_sh[2];
    __shared__ long long dsum[2][4];   // per side: moved q0 q1 q2, count
    __shared__ uint32_t cntT_sh[2];    // particles in the threshold bin
    __shared__ int list_sh;            // threshold bins split through the list (else the grid select)
    // tkey (tie-break select)
    __shared__ __align__(16) unsigned char sbuf[SW_SBUF];
    uint32_t(*tkey)[SW_TCAP] = (uint32_t(*)[SW_TCAP])sbuf;
    const unsigned nb = gridDim.x;
    const int64_t gstride = (int64_t)gridDim.x * SW_THREADS;
    const int64_t g0 = (int64_t)blockIdx.x * SW_THREADS + threadIdx.x;
    const bool multi = nmat > 1;
    const int ntype = multi ? nmat : 1;

    // the fixed-point sums and the speculative counts come from k_swap_sums and k_swap_spec
    const int npairs = K * (K - 1) / 2;
    const int ncombo = ntype * npairs;
    __shared__ int first_sh;
    // label segments (K >= 8): sidx[0, n) holds the slots grouped by label (segment l at
    // [loff[l], loff[l + 1]), built by k_swap_spec). A pair's swaps exchange equally many particles each
    // way, so the segments keep their sizes; the moved particles exchange their segment positions after
    // each pair (mv lists at sidx[n, 2n)), and a pair visits only its two labels' particles, 2n/K
    // instead of n. Order within a segment is free: every use is a count, an exact sum or a select by
    // persistent id. With fewer labels the segments cost more (their build, one more barrier per pair)
    // than they save, and the pairs visit every slot.
    const bool seg = K >= 8;
    __shared__ long long loff_sh[kMaxLabel + 1];
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int l = 0; l < kMaxLabel; ++l) {
            loff_sh[l] = o;
            if (l < K) o += ((volatile long long *)&S->cnt[l][kMaxMat])[0];
        }
        loff_sh[kMaxLabel] = o;
        // the first pair with positive hashes on both sides at the pass-start state; the pairs before
        // it swap nothing and change nothing
        int f = ncombo;
        for (int q = 0; q < ncombo && f == ncombo; ++q)
            if (((volatile uint32_t *)&pairs[q].spec[0])[0] > 0u && ((volatile uint32_t *)&pairs[q].spec[1])[0] > 0u) f = q;
        first_sh = f;
    }
    uint32_t *const byl = sidx;
    uint32_t *const mvl = sidx + n;                      // side 0 at [0, n/2), side 1 at [n/2, n)
    const int64_t mvh = (n + 1) / 2;
    __syncthreads();
    const int first = first_sh;   // the same in every block
    if (first >= ncombo) return;

    // labels whose particles or sums a pair of this pass has changed (the same in every thread: every
    // block takes the same decisions). A pair of two unchanged labels sees the pass-start state, so its
    // speculative counts are its own: an empty side means the pair swaps nothing and changes nothing.
    uint32_t dirty = 0u;
    int idx = 0;
    for (int T = 0; T < ntype; ++T) {
        const int type = multi ? T : -1;
        const int slot = multi ? T : kMaxMat;
        for (int a = 0; a < K - 1; ++a)
            for (int b = a + 1; b < K; ++b, ++idx) {
                SwapPair *pr = pairs + idx;
                if (idx < first) continue;   // no positive hashes on a side: nothing to do
                if (!(dirty & ((1u << a) | (1u << b))) && (pr->spec[0] == 0u || pr->spec[1] == 0u)) continue;
                // this pair's particles: the segments of a and b (their labels read from L2: another
                // block may have written them in an earlier pair)
                const long long oa = loff_sh[a], na = loff_sh[a + 1] - oa, ob = loff_sh[b];
                const long long tot = seg ? na + (loff_sh[b + 1] - ob) : n;
                // position k of the pair's iteration -> its segment position (without segments: the slot)
                auto segpos = [&](long long k) { return !seg ? k : (k < na ? oa + k : ob + (k - na)); };
                auto slot_at = [&](long long sp) { return seg ? __ldcg(&byl[sp]) : (uint32_t)sp; };
                // -- pair geometry (every block, identical operations on the same sums): counts, then the
                // Cg components in parallel, the Cg' blend and the segment, its length, then the direction
                // and scale. Side b's direction is the exact negation of side a's (d_b = -d_a bit for bit).
                // counts and sums in one round trip: thread 3w + ax reads count w and sum component ax
                if (threadIdx.x < 12) {
                    const int w = threadIdx.x / 3, ax = threadIdx.x % 3, l = (w & 1) ? b : a, sl = w < 2 ? slot : kMaxMat;
                    const long long cn = ((volatile long long *)&S->cnt[l][sl])[0];
                    if (ax == 0) gn_sh[w] = cn;
                    if ((w < 2 || multi) && cn > 0) {
                        const long long sm = ((volatile long long *)&S->sums[l][sl][ax])[0];
                        const double mean = __ddiv_rn(__ll2double_rn(sm), __ll2double_rn(cn));
                        gcg_sh[w][ax] = __dadd_rn(Q.lo[ax], __dmul_rn(mean, Q.step[ax]));
                    }
                }
                __syncthreads();
                const bool have = gn_sh[0] > 0 && gn_sh[1] > 0;
                if (have && threadIdx.x < 3) {
                    const int ax = threadIdx.x;
                    double ca = gcg_sh[0][ax], cb = gcg_sh[1][ax];
                    if (multi) {   // Sec. III.B: Cg' = alpha Cg_all + (1 - alpha) Cg_type
                        const double beta = __dsub_rn(1.0, alpha);
                        ca = __dadd_rn(__dmul_rn(alpha, gcg_sh[2][ax]), __dmul_rn(beta, ca));
                        cb = __dadd_rn(__dmul_rn(alpha, gcg_sh[3][ax]), __dmul_rn(beta, cb));
                    }
                    const double M = __dmul_rn(__dadd_rn(ca, cb), 0.5);
                    const double d = __dsub_rn(cb, ca);
                    side_sh[0].M[ax] = M;
                    side_sh[1].M[ax] = M;
                    side_sh[0].f.M[ax] = (float)M;
                    side_sh[1].f.M[ax] = (float)M;
                    side_sh[0].d[ax] = d;
                    side_sh[1].d[ax] = -d;
                    gd_sh[ax] = d;
                }
                __syncthreads();
                if (threadIdx.x == 0) gdn_sh = have ? __dsqrt_rn(dist2_rn(gd_sh[0], gd_sh[1], gd_sh[2])) : 0.0;
                __syncthreads();
                const bool act_g = have && gdn_sh > 0.0;
                if (act_g && threadIdx.x < 4) {
                    if (threadIdx.x < 3) {
                        const float u = (float)__ddiv_rn(gd_sh[threadIdx.x], gdn_sh);
                        side_sh[0].f.u[threadIdx.x] = u;
                        side_sh[1].f.u[threadIdx.x] = -u;
                    } else {
                        const double ell = __dmul_rn(gdn_sh, 0.5);
                        const float sc = (float)__ddiv_rn(1000.0, ell);
                        side_sh[0].f.scale = sc;
                        side_sh[1].f.scale = sc;
                        side_sh[0].dn = gdn_sh;
                        side_sh[1].dn = gdn_sh;
                        side_sh[0].ell = ell;
                        side_sh[1].ell = ell;
                    }
                }
                if (threadIdx.x == 0) act_sh = act_g;
                for (int k = threadIdx.x; k < 2 * SW_BINS; k += SW_THREADS) (&hs[0][0])[k] = 0;
                if (threadIdx.x < 2) npos_sh[threadIdx.x] = 0u;
                __syncthreads();
                const bool act = act_sh != 0;
                // -- balancing hashes and their histograms
                if (act) {
                    const SideF s0 = side_sh[0].f, s1 = side_sh[1].f;
                    for (int64_t base = (int64_t)blockIdx.x * SW_THREADS; base < tot; base += gstride) {
                        const int64_t k = base + threadIdx.x;
                        int key = -1;
                        if (k < tot) {
                            const uint32_t i = slot_at(segpos(k));
                            const uint8_t l = __ldcg(&lab[i]);
                            if ((l == a || l == b) && (type < 0 || mat[i] == type)) {
                                const int sd = l == a ? 0 : 1;
                                int hv = balancing_hash_fast(sd == 0 ? s0 : s1, pos.x[i], pos.y[i], pos.z[i]);
                                if (hv < 0) {   // within the FP32 bound of a decision boundary
                                    const Side &G = side_sh[sd];
                                    hv = balancing_hash64(G.M, G.d, G.dn, G.ell, pos.X[i], pos.Y[i], pos.Z[i]);
                                    atomicAdd(&S->fp64, 1ull);
                                }
                                bh[i] = (uint16_t)hv;
                                if (hv > 0) key = sd * SW_BINS + hv;   // only positive hashes are counted
                            }
                        }
                        // warps without a positive hash (most of them once labels have settled) skip the
                        // histogram; the others count per side and add per bin
                        const unsigned pos0 = __ballot_sync(kFullMask, key >= 0 && key < SW_BINS);
                        const unsigned pos1 = __ballot_sync(kFullMask, key >= SW_BINS);
                        if (pos0 | pos1) {
                            if ((threadIdx.x & 31) == 0) {
                                if (pos0) atomicAdd(&npos_sh[0], (uint32_t)__popc(pos0));
                                if (pos1) atomicAdd(&npos_sh[1], (uint32_t)__popc(pos1));
                            }
                            const unsigned peers = __match_any_sync(kFullMask, key);
                            if (key >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
                                atomicAdd(&(&hs[0][0])[key], (uint32_t)__popc(peers));
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x < 2 && npos_sh[threadIdx.x]) atomicAdd(&pr->npos[threadIdx.x], npos_sh[threadIdx.x]);
                    for (int k = threadIdx.x; k < 2 * SW_BINS; k += SW_THREADS) {
                        const uint32_t v = (&hs[0][0])[k];
                        if (v) atomicAdd(&(&pr->hist[0][0])[k], v);
                    }
                }
                if (!grid_barrier(S, nb, err, wc)) return;
                if (!act) continue;
                // n = min(#positive): no scans when a side has none (the same decision in every block)
                if (((volatile uint32_t *)&pr->npos[0])[0] == 0u || ((volatile uint32_t *)&pr->npos[1])[0] == 0u) continue;
                // -- n = min(#positive), threshold hash and the count to take from the threshold bin:
                // cum[sd][r] = particles of side sd with hash >= 1000 - r (block scans, every block)
                __shared__ uint32_t cum[2][SW_BINS - 1];
                for (int k = threadIdx.x; k < 2 * (SW_BINS - 1); k += SW_THREADS) {
                    const int sd = k / (SW_BINS - 1), r = k % (SW_BINS - 1);
                    cum[sd][r] = ((volatile uint32_t *)&pr->hist[sd][0])[GSPH_BALANCE_HASH_MAX - r];
                }
                __syncthreads();
                block_inclusive_scan(cum[0], SW_BINS - 1);
                block_inclusive_scan(cum[1], SW_BINS - 1);
                const uint32_t m = min(cum[0][SW_BINS - 2], cum[1][SW_BINS - 2]);
                if (m == 0) continue;    // the same decision in every block: no barrier is skipped unevenly
                dirty |= (1u << a) | (1u << b);
                for (int k = threadIdx.x; k < 2 * (SW_BINS - 1); k += SW_THREADS) {
                    const int sd = k / (SW_BINS - 1), r = k % (SW_BINS - 1);
                    const uint32_t above = r > 0 ? cum[sd][r - 1] : 0u;
                    if (cum[sd][r] >= m && above < m) {
                        const int Tb = GSPH_BALANCE_HASH_MAX - r;
                        T_sh[sd] = Tb;
                        need_sh[sd] = m - above;
                        cntT_sh[sd] = cum[sd][r] - above;
                        idsel_sh[sd] = (m - above) < (cum[sd][r] - above);
                        idpre_sh[sd] = 0;
                    }
                }
                if (blockIdx.x == 0 && threadIdx.x == 0) pr->moved = 2ull * m;
                __syncthreads();
                if (threadIdx.x == 0)
                    list_sh = (!idsel_sh[0] || cntT_sh[0] <= (uint32_t)SW_TCAP) &&
                              (!idsel_sh[1] || cntT_sh[1] <= (uint32_t)SW_TCAP);
                __syncthreads();
                const bool use_list = list_sh != 0;
                // -- radix select on persistent ids inside split threshold bins, over all particles
                if (!use_list && (idsel_sh[0] || idsel_sh[1])) {
                    for (int pass = 0; pass < 3; ++pass) {
                        const int shift = 18 - SW_ID_BITS * pass;
                        for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) (&ids[0][0])[k] = 0;
                        __syncthreads();
                        for (int64_t k = g0; k < tot; k += gstride) {
                            const uint32_t i = slot_at(segpos(k));
                            const uint8_t l = __ldcg(&lab[i]);
                            if ((l != a && l != b) || (type >= 0 && mat[i] != type)) continue;
                            const int sd = l == a ? 0 : 1;
                            if (!idsel_sh[sd] || __ldcg(&bh[i]) != T_sh[sd]) continue;
                            const uint32_t v = id[i];
                            if ((v >> (shift + SW_ID_BITS)) == (idpre_sh[sd] >> (shift + SW_ID_BITS)))
                                atomicAdd(&ids[sd][(v >> shift) & (SW_ID_BINS - 1)], 1u);
                        }
                        __syncthreads();
                        for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) {
                            const uint32_t v = (&ids[0][0])[k];
                            if (v) atomicAdd(&(&pr->idh[pass][0][0])[k], v);
                        }
                        if (!grid_barrier(S, nb, err, wc)) return;
                        for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS)
                            (&ids[0][0])[k] = ((volatile uint32_t *)&pr->idh[pass][0][0])[k];
                        __syncthreads();
                        block_inclusive_scan(ids[0], SW_ID_BINS);
                        block_inclusive_scan(ids[1], SW_ID_BINS);
                        __shared__ uint32_t upd[2][2];
                        for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) {
                            const int sd = k / SW_ID_BINS, d = k % SW_ID_BINS;
                            if (!idsel_sh[sd]) continue;
                            const uint32_t below = d > 0 ? ids[sd][d - 1] : 0u;
                            if (ids[sd][d] >= need_sh[sd] && below < need_sh[sd]) {
                                upd[sd][0] = (uint32_t)d;
                                upd[sd][1] = below;
                            }
                        }
                        __syncthreads();
                        if (threadIdx.x < 2 && idsel_sh[threadIdx.x]) {
                            idpre_sh[threadIdx.x] |= upd[threadIdx.x][0] << shift;
                            need_sh[threadIdx.x] -= upd[threadIdx.x][1];
                        }
                        __syncthreads();
                    }
                }
                // -- label exchange and exact update of the fixed-point sums; the threshold bins that the
                // list splits are collected instead
                if (threadIdx.x < 8) (&dsum[0][0])[threadIdx.x] = 0;
                __syncthreads();
                for (int64_t base = (int64_t)blockIdx.x * SW_THREADS; base < tot; base += gstride) {
                    const int64_t k = base + threadIdx.x;
                    int sd = -1, ap = -1;
                    long long q0 = 0, q1 = 0, q2 = 0;
                    uint32_t i = 0;
                    const long long sp = k < tot ? segpos(k) : 0;
                    if (k < tot) {
                        i = slot_at(sp);
                        const uint8_t l = __ldcg(&lab[i]);
                        if ((l == a || l == b) && (type < 0 || mat[i] == type)) {
                            const int side = l == a ? 0 : 1;
                            const int hv = __ldcg(&bh[i]);
                            bool take = false;
                            if (hv > 0 && hv > T_sh[side]) {
                                take = true;
                            } else if (hv > 0 && hv == T_sh[side]) {
                                if (!idsel_sh[side]) take = true;
                                else if (!use_list) take = id[i] <= idpre_sh[side];
                                else ap = side;
                            }
                            if (take) {
                                sd = side;
                                lab[i] = (uint8_t)(side == 0 ? b : a);
                                q0 = pos.qx[i];
                                q1 = pos.qy[i];
                                q2 = pos.qz[i];
                            }
                        }
                    }
                    if (__any_sync(kFullMask, sd >= 0)) warp_add_sums(dsum, sd < 0 ? 0 : sd, sd >= 0, q0, q1, q2);
                    // the moved particles' segment positions, per side
#pragma unroll
                    for (int side = 0; side < 2 && seg; ++side) {
                        const unsigned mm = __ballot_sync(kFullMask, sd == side);
                        if (!mm) continue;
                        const int lane = threadIdx.x & 31, ld = __ffs(mm) - 1;
                        uint32_t pos = 0;
                        if (lane == ld) pos = atomicAdd(&pr->mvcnt[side], (uint32_t)__popc(mm));
                        pos = __shfl_sync(kFullMask, pos, ld) + (uint32_t)__popc(mm & lanemask_lt());
                        if (seg && sd == side) mvl[side * mvh + pos] = (uint32_t)sp;
                    }
                    // warp-aggregated append of (id, segment position) to the side's threshold-bin list
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const unsigned am = __ballot_sync(kFullMask, ap == side);
                        if (!am) continue;
                        const int lane = threadIdx.x & 31, ld = __ffs(am) - 1;
                        uint32_t pos = 0;
                        if (lane == ld) pos = atomicAdd(&pr->tcnt[side], (uint32_t)__popc(am));
                        pos = __shfl_sync(kFullMask, pos, ld) + (uint32_t)__popc(am & lanemask_lt());
                        if (ap == side && pos < (uint32_t)SW_TCAP)
                            tl[side * SW_TCAP + pos] = make_uint2(id[i], (uint32_t)sp);
                    }
                }
                __syncthreads();
                flush_moved(S, dsum, a, b, type);
                if (!grid_barrier(S, nb, err, wc)) return;
                // (the moved particles exchange their segment positions once all of the pair's moves are in)
                auto exchange_positions = [&]() -> bool {
                    if (!seg) return true;
                    for (int64_t r = g0; r < (int64_t)m; r += gstride) {
                        const uint32_t ka = __ldcg(&mvl[r]), kb = __ldcg(&mvl[mvh + r]);
                        const uint32_t ia = __ldcg(&byl[ka]), ib = __ldcg(&byl[kb]);
                        byl[ka] = ib;
                        byl[kb] = ia;
                    }
                    return grid_barrier(S, nb, err, wc);
                };
                if (!use_list || !(idsel_sh[0] || idsel_sh[1])) {
                    if (!exchange_positions()) return;
                    continue;
                }
                // -- id threshold of each listed bin: radix select in shared memory, every block
                for (int sd = 0; sd < 2; ++sd) {
                    if (!idsel_sh[sd]) continue;
                    for (uint32_t k = threadIdx.x; k < cntT_sh[sd]; k += SW_THREADS)
                        tkey[sd][k] = __ldcg(&tl[sd * SW_TCAP + k].x);
                }
                __syncthreads();
                for (int pass = 0; pass < 3; ++pass) {
                    const int shift = 18 - SW_ID_BITS * pass;
                    for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) (&ids[0][0])[k] = 0;
                    __syncthreads();
                    for (int sd = 0; sd < 2; ++sd) {
                        if (!idsel_sh[sd]) continue;
                        for (uint32_t k = threadIdx.x; k < cntT_sh[sd]; k += SW_THREADS) {
                            const uint32_t v = tkey[sd][k];
                            if ((v >> (shift + SW_ID_BITS)) == (idpre_sh[sd] >> (shift + SW_ID_BITS)))
                                atomicAdd(&ids[sd][(v >> shift) & (SW_ID_BINS - 1)], 1u);
                        }
                    }
                    __syncthreads();
                    block_inclusive_scan(ids[0], SW_ID_BINS);
                    block_inclusive_scan(ids[1], SW_ID_BINS);
                    __shared__ uint32_t upd2[2][2];
                    for (int k = threadIdx.x; k < 2 * SW_ID_BINS; k += SW_THREADS) {
                        const int sd = k / SW_ID_BINS, d = k % SW_ID_BINS;
                        if (!idsel_sh[sd]) continue;
                        const uint32_t below = d > 0 ? ids[sd][d - 1] : 0u;
                        if (ids[sd][d] >= need_sh[sd] && below < need_sh[sd]) {
                            upd2[sd][0] = (uint32_t)d;
                            upd2[sd][1] = below;
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x < 2 && idsel_sh[threadIdx.x]) {
                        idpre_sh[threadIdx.x] |= upd2[threadIdx.x][0] << shift;
                        need_sh[threadIdx.x] -= upd2[threadIdx.x][1];
                    }
                    __syncthreads();
                }
                // -- swaps of the listed particles up to the id threshold, each applied by the block that
                // owns its slot in the strided partition (so no block reads a label another block wrote)
                if (threadIdx.x < 8) (&dsum[0][0])[threadIdx.x] = 0;
                __syncthreads();
                for (int sd = 0; sd < 2; ++sd) {
                    if (!idsel_sh[sd]) continue;
                    const uint32_t c = cntT_sh[sd];
                    for (uint32_t k0 = 0; k0 < c; k0 += SW_THREADS) {
                        const uint32_t k = k0 + threadIdx.x;
                        bool mv = false;
                        long long q0 = 0, q1 = 0, q2 = 0;
                        if (k < c) {
                            const uint2 e = __ldcg(&tl[sd * SW_TCAP + k]);
                            const uint32_t i = slot_at(e.y);
                            if ((k / SW_THREADS) % nb == blockIdx.x && e.x <= idpre_sh[sd]) {
                                mv = true;
                                // (append the segment position to the side's moved list)
                                if (seg) mvl[sd * mvh + atomicAdd(&pr->mvcnt[sd], 1u)] = e.y;
                                lab[i] = (uint8_t)(sd == 0 ? b : a);
                                q0 = pos.qx[i];
                                q1 = pos.qy[i];
                                q2 = pos.qz[i];
                            }
                        }
                        if (__any_sync(kFullMask, mv)) warp_add_sums(dsum, sd, mv, q0, q1, q2);
                    }
                }
                __syncthreads();
                flush_moved(S, dsum, a, b, type);
                if (!grid_barrier(S, nb, err, wc)) return;
                if (!exchange_positions()) return;
            }
    }
}

// ---------------------------------------------------------------------------------------------
// Host side: one full pass, three streaming launches and one cooperative launch.
// ---------------------------------------------------------------------------------------------
size_t swap_scratch_bytes(int K, int nmat) {
    const int ntype = nmat > 1 ? nmat : 1;
    const size_t npairs = (size_t)ntype * (size_t)(K * (K - 1) / 2);
    return sizeof(SwapScratch) + (npairs > 0 ? npairs : 1) * sizeof(SwapPair) + 2 * SW_TCAP * sizeof(uint2);
}

static QuantParams quant_params(const DevParams &P) {
    QuantParams Q;
    for (int a = 0; a < 3; ++a) {
        Q.lo[a] = P.lo[a];
        Q.s[a] = P.q_s[a];
        Q.step[a] = P.q_step[a];
    }
    return Q;
}

// Blocks of the cooperative swap pass: two per SM when they fit (all must be resident at once).
int swap_grid_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_swap_pass, SW_THREADS, 0) != cudaSuccess) return 0;
    return sms * (per < 2 ? per : 2);
}

// pos: the particles' FP32 and FP64 positions and fixed-point coordinates (launch_round_positions, or the
// reorder). scratch: swap_scratch_bytes() device bytes, cleared here unless scratch_clear says that an
// earlier kernel on the stream has cleared it; bh: n uint16; sidx: 2n uint32 (label segments and moved
// lists); grid from swap_grid_blocks(). The sums and the speculative pass are programmatic dependent
// launches.
cudaError_t launch_swap_pass(const DevParams &P, int64_t n, const SwapPos &pos, uint8_t *lab, const uint8_t *mat,
                             const uint32_t *id, void *scratch, uint16_t *bh, uint32_t *sidx, int *err, int grid,
                             unsigned spin_limit, unsigned extra_blocks, bool scratch_clear, cudaStream_t s) {
    if (n <= 0 || P.K_labels < 2) return cudaSuccess;
    if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
    const size_t bytes = swap_scratch_bytes(P.K_labels, P.nmat);
    cudaError_t e = cudaSuccess;
    if (!scratch_clear && (e = cudaMemsetAsync(scratch, 0, bytes, s)) != cudaSuccess) return e;
    SwapScratch *S = (SwapScratch *)scratch;
    SwapPair *pairs = (SwapPair *)((char *)scratch + sizeof(SwapScratch));
    const int ntype = P.nmat > 1 ? P.nmat : 1;
    const size_t npairs = (size_t)ntype * (size_t)(P.K_labels * (P.K_labels - 1) / 2);
    uint2 *tl = (uint2 *)(pairs + (npairs > 0 ? npairs : 1));
    QuantParams Q = quant_params(P);
    double alpha = P.alpha;
    int K = P.K_labels, nmat = P.nmat;
    SwapPos ps = pos;
    // the streaming phases: two blocks per cooperative block, at most one thread per particle
    const int64_t want = (n + SW_THREADS - 1) / SW_THREADS;
    const unsigned sgrid = (unsigned)(want < 2 * (int64_t)grid ? want : 2 * (int64_t)grid);
    const uint8_t *labc = lab;
    if ((e = pdl_launch(k_swap_sums, dim3(sgrid), dim3(SW_THREADS), s, n, nmat, ps, labc, mat, S)) != cudaSuccess)
        return e;
    if ((e = pdl_launch(k_swap_spec, dim3(sgrid), dim3(SW_THREADS), s, n, Q, alpha, K, nmat, ps, labc, mat, S, pairs,
                        sidx)) != cudaSuccess)
        return e;
    WaitCfg wc{spin_limit > 0 ? spin_limit : (1u << 24), extra_blocks};
    void *args[] = {(void *)&n, (void *)&Q, (void *)&alpha, (void *)&K, (void *)&nmat, (void *)&ps, (void *)&lab,
                    (void *)&mat, (void *)&id, (void *)&bh, (void *)&S, (void *)&pairs, (void *)&tl, (void *)&sidx,
                    (void *)&err, (void *)&wc};
    return cudaLaunchCooperativeKernel((const void *)k_swap_pass, dim3(grid), dim3(SW_THREADS), args, 0, s);
}

// The swap pass's position inputs from FP64 positions (a pass outside a step): FP32 roundings and the
// fixed-point coordinates of the Cg sums.
__global__ void k_round_positions(DevParams P, int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                  const double *__restrict__ z, float *__restrict__ xf, float *__restrict__ yf,
                                  float *__restrict__ zf, uint32_t *__restrict__ qx, uint32_t *__restrict__ qy,
                                  uint32_t *__restrict__ qz, QuantParams Q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double X = x[i], Y = y[i], Z = z[i];
    xf[i] = __double2float_rn(X);
    yf[i] = __double2float_rn(Y);
    zf[i] = __double2float_rn(Z);
    qx[i] = quantise64(X, Q.lo[0], Q.s[0]);
    qy[i] = quantise64(Y, Q.lo[1], Q.s[1]);
    qz[i] = quantise64(Z, Q.lo[2], Q.s[2]);
}

cudaError_t launch_round_positions(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                                   float *xf, float *yf, float *zf, uint32_t *qx, uint32_t *qy, uint32_t *qz,
                                   cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_round_positions<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, x, y, z, xf, yf, zf, qx, qy, qz,
                                                                  quant_params(P));
    return cudaGetLastError();
}

// Number of particles moved by the last pass (device pointer into the scratch).
unsigned long long *swap_moved_ptr(void *scratch) { return &((SwapScratch *)scratch)->moved; }
// Balancing hashes of the last pass that the FP64 sequence decided (the next word).
static_assert(offsetof(SwapScratch, fp64) == offsetof(SwapScratch, moved) + 8, "moved, fp64 adjacent");
static_assert(kMaxLabel <= 32, "the pair loop keeps its changed labels in one 32-bit mask");

}  // namespace gsph
