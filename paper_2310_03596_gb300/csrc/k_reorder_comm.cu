// k_reorder_comm.cu - reorder into hash order with bucket ranges and interaction records (Sec. I),
// communication hash, MGPU boundary flags and boundary set (Sec. II steps b-d, K virtual labels),
// particle initialisation and the FP64 reductions (time step, conserved sums).
#include "gsph_internal.cuh"

namespace gsph {

// ---------------------------------------------------------------------------------------------
// Reorder: sorted slot s takes old slot o = perm[s]. Writes the sorted FP64 positions (and their FP32
// roundings when xf is given: the swap pass's inputs), label, material and id, the bucket range of each
// occupied bucket (ranges of empty buckets stay 0,0 from the memset), and the interaction record of the
// particle.
// ---------------------------------------------------------------------------------------------
// Interaction record of one particle in slot s with bucket hash k: split path, the position relative
// to the own bucket corner and the FP32 state with the stress diagonal as sigma = -p I + S; FP64 path,
// the FP64 position and state. Pressure and impedance from the equation of state.
// Split-path position record: the position relative to the particle's own bucket corner (|.| < 2h, so
// FP32 keeps it to about 2^-24 * 2h) and the FP32 volume. The corners come from per-axis tables
// (fma(c, 2h, lo), formed once per buffer set), which saves the FP64 product of every particle.
__device__ __forceinline__ float4 pos_split(const DevParams &P, uint32_t k, double x, double y, double z, double w) {
    float4 p4 = make_float4(0.f, 0.f, 0.f, (float)w);
    if (k < P.ncell) {
        int cx, cy, cz;
        decode_cell(P, k, cx, cy, cz);
        p4.x = (float)(x - P.corner[0][cx]);
        p4.y = (float)(y - P.corner[1][cy]);
        p4.z = (float)(z - P.corner[2][cz]);
    }
    return p4;
}

template <bool SPLIT>
__device__ __forceinline__ void write_record(const DevParams &P, int64_t s, uint32_t k, double x, double y, double z,
                                             double w, double m, double vx, double vy, double vz, double E,
                                             double sxx, double syy, double szz, double sxy, double sxz,
                                             double syz, int mat, void *__restrict__ pos_out,
                                             void *__restrict__ rec_out) {
    if (SPLIT) {
        RecF r;
        ((float4 *)pos_out)[s] = pos_split(P, k, x, y, z, w);
        if (P.eos[mat] == 0) {
            r = record_split_linear(P, mat, w, m, vx, vy, vz, E, sxx, syy, sxy, sxz, syz);
        } else {   // Mie-Gruneisen in FP64 (its Hugoniot terms cancel as well), rounded once
            const float rho = (float)m / (float)w;
            double pd, cd;
            const double rd = m / w;
            eos_pc(P, mat, rd, E - 0.5 * (vx * vx + vy * vy + vz * vz), pd, cd);
            const float pf = (float)pd, Zf = (float)(rd * cd);
            // the diagonal of the full stress sigma = -p I + S (S traceless in FP32: S_zz = -(S_xx + S_yy))
            const float fxx = (float)sxx, fyy = (float)syy, fzz = -(fxx + fyy);
            r.a = make_float4((float)vx, (float)vy, (float)vz, rho);
            r.b = make_float4(fzz - pf, Zf, (float)E, fxx - pf);
            r.c = make_float4(fyy - pf, (float)sxy, (float)sxz, (float)syz);
        }
        ((RecF *)rec_out)[s] = r;
        (void)szz;
    } else {
        RecD r;
        double rho = m / w;
        double pr, c;
        eos_pc(P, mat, rho, E - 0.5 * (vx * vx + vy * vy + vz * vz), pr, c);
        r.a = make_d4(vx, vy, vz, rho);
        r.b = make_d4(pr, rho * c, E, sxx);
        r.c = make_d4(syy, szz, sxy, sxz);
        r.d = make_d4(syz, 0.0, 0.0, 0.0);
        ((D4 *)pos_out)[s] = make_d4(x, y, z, w);
        ((RecD *)rec_out)[s] = r;
    }
}

template <bool SPLIT>
__global__ void __launch_bounds__(256) k_reorder(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                                                 const uint32_t *__restrict__ perm, State A,
                                                 double *__restrict__ xs, double *__restrict__ ys,
                                                 double *__restrict__ zs, uint8_t *__restrict__ lab_s,
                                                 uint8_t *__restrict__ mat_s, uint32_t *__restrict__ id_s,
                                                 uint2 *__restrict__ cellr, float *__restrict__ cxs,
                                                 void *__restrict__ pos_out, void *__restrict__ rec_out,
                                                 float *__restrict__ xf, float *__restrict__ yf,
                                                 float *__restrict__ zf, uint32_t *__restrict__ qx,
                                                 uint32_t *__restrict__ qy, uint32_t *__restrict__ qz,
                                                 double *__restrict__ hs, float *__restrict__ hsf,
                                                 const RecF *__restrict__ rec_in, float4 *__restrict__ posf,
                                                 int *__restrict__ err, unsigned long long *__restrict__ garbage) {
    pdl_wait();      // launched after the sort as a programmatic dependent launch
    pdl_release();
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t k = skey[s];
    uint32_t o = perm[s];
    if (garbage) {   // particles outside the grid sort last (key ncell): their count from where they start
        if (k >= P.ncell && (s == 0 || skey[s - 1] < P.ncell)) *garbage = (unsigned long long)(n - s);
        if (s == n - 1 && k < P.ncell) *garbage = 0ull;
    }
    if (hs) {   // variable h: the sorted smoothing lengths, FP64 and their FP32 roundings
        const double hh = A.h[o];
        hs[s] = hh;
        hsf[s] = __double2float_rn(hh);
    }
    double x = A.f[FX][o], y = A.f[FY][o], z = A.f[FZ][o];
    xs[s] = x; ys[s] = y; zs[s] = z;
    if (xf) {   // the swap pass's inputs: FP32 roundings and fixed-point coordinates
        xf[s] = __double2float_rn(x);
        yf[s] = __double2float_rn(y);
        zf[s] = __double2float_rn(z);
        qx[s] = quantise64(x, P.lo[0], P.q_s[0]);
        qy[s] = quantise64(y, P.lo[1], P.q_s[1]);
        qz[s] = quantise64(z, P.lo[2], P.q_s[2]);
    }
    uint8_t lab = A.label[o], mat = A.mat[o];
    // invalid values are reported and clamped so that no later kernel indexes out of range
    if (lab >= P.K_labels) { atomicOr(err, kErrLabel); lab = 0; }
    if (mat >= P.nmat) { atomicOr(err, kErrMaterial); mat = 0; }
    lab_s[s] = lab;
    mat_s[s] = mat;
    id_s[s] = A.id[o];
    if (k < P.ncell) {
        if (s == 0 || skey[s - 1] != k) cellr[k].x = (uint32_t)s;
        if (s == n - 1 || skey[s + 1] != k) cellr[k].y = (uint32_t)(s + 1);
        cxs[s] = (float)(k % (uint32_t)P.dims[0]);
    } else {
        cxs[s] = -1.0e9f;
    }
    if (!SPLIT && posf) {   // FP64 path: the FP32 bucket-relative positions of the neighbour-list build
        posf[s] = pos_split(P, k, x, y, z, A.f[FW][o]);
    }
    if (SPLIT && rec_in) {   // the record the previous step's integration wrote from the same state
        ((float4 *)pos_out)[s] = pos_split(P, k, x, y, z, A.f[FW][o]);
        ((RecF *)rec_out)[s] = rec_in[o];
        return;
    }
    write_record<SPLIT>(P, s, k, x, y, z, A.f[FW][o], A.f[FM][o], A.f[FVX][o], A.f[FVY][o], A.f[FVZ][o],
                        A.f[FE][o], A.f[FSXX][o], A.f[FSYY][o], A.f[FSZZ][o], A.f[FSXY][o], A.f[FSXZ][o],
                        A.f[FSYZ][o], mat, pos_out, rec_out);
}

// Records of the predicted state of the Heun step (state B in slot order), relative to the bucket
// corners of the step's hash; the sorted view and the bucket ranges stay those of the step's start.
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_refresh(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                                                 State B, void *__restrict__ pos_out, void *__restrict__ rec_out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int mat = B.mat[s] < P.nmat ? B.mat[s] : 0;
    write_record<SPLIT>(P, s, skey[s], B.f[FX][s], B.f[FY][s], B.f[FZ][s], B.f[FW][s], B.f[FM][s], B.f[FVX][s],
                        B.f[FVY][s], B.f[FVZ][s], B.f[FE][s], B.f[FSXX][s], B.f[FSYY][s], B.f[FSZZ][s],
                        B.f[FSXY][s], B.f[FSXZ][s], B.f[FSYZ][s], mat, pos_out, rec_out);
}

cudaError_t launch_refresh(bool split, const DevParams &P, int64_t n, const uint32_t *skey, const State &B,
                           void *pos, void *rec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    unsigned g = (unsigned)((n + 255) / 256);
    if (split) k_refresh<true><<<g, 256, 0, s>>>(P, n, skey, B, pos, rec);
    else k_refresh<false><<<g, 256, 0, s>>>(P, n, skey, B, pos, rec);
    return cudaGetLastError();
}

cudaError_t launch_reorder(bool split, const DevParams &P, int64_t n, const uint32_t *skey, const uint32_t *perm,
                           const State &A, double *xs, double *ys, double *zs, uint8_t *lab_s, uint8_t *mat_s,
                           uint32_t *id_s, uint2 *cellr, float *cxs, void *pos, void *rec, float *xf, float *yf,
                           float *zf, uint32_t *qx, uint32_t *qy, uint32_t *qz, double *hs, float *hsf,
                           const void *rec_in, float4 *posf, int *err, unsigned long long *garbage,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    unsigned g = (unsigned)((n + 255) / 256);
    const uint32_t *key = skey, *pm = perm;
    if (split)
        return pdl_launch(k_reorder<true>, dim3(g), dim3(256), s, P, n, key, pm, A, xs, ys, zs, lab_s, mat_s, id_s,
                          cellr, cxs, pos, rec, xf, yf, zf, qx, qy, qz, hs, hsf, (const RecF *)rec_in,
                          (float4 *)nullptr, err, garbage);
    return pdl_launch(k_reorder<false>, dim3(g), dim3(256), s, P, n, key, pm, A, xs, ys, zs, lab_s, mat_s, id_s,
                      cellr, cxs, pos, rec, xf, yf, zf, qx, qy, qz, hs, hsf, (const RecF *)nullptr, posf, err, garbage);
}

// ---------------------------------------------------------------------------------------------
// Communication hash (Sec. II steps b-c with K virtual labels). On one device the hash broadcast of
// step b becomes a per-bucket OR of label bits: mask[c] has bit k set when a particle of label k
// is in bucket c. A particle is an MGPU boundary particle when the 27 buckets around it hold a
// label other than its own.
// ---------------------------------------------------------------------------------------------
__global__ void k_label_mask(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                             const uint8_t *__restrict__ lab_s, uint32_t *__restrict__ mask) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t k = s < n ? skey[s] : 0xffffffffu;
    uint32_t bit = (s < n && k < P.ncell) ? (1u << (lab_s[s] & 31)) : 0u;
    // sorted keys: lanes of one bucket combine their bits first, one atomic per bucket and warp
    unsigned peers = __match_any_sync(kFullMask, k);
    uint32_t acc = __reduce_or_sync(peers, bit);
    if (s < n && k < P.ncell && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicOr(&mask[k], acc);
}

// Flags, communication hash and per-block counts per label (block_counts[label * nblk + block]).
constexpr int CM_THREADS = 512;
__global__ void __launch_bounds__(CM_THREADS) k_comm(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                                                     const uint8_t *__restrict__ lab_s,
                                                     const uint32_t *__restrict__ mask, uint8_t *__restrict__ flag,
                                                     uint32_t *__restrict__ comm, uint32_t *__restrict__ block_counts,
                                                     int nblk) {
    __shared__ uint32_t cnt[kMaxLabel];
    if (threadIdx.x < kMaxLabel) cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t k = s < n ? skey[s] : P.ncell;
    const bool in = s < n && k < P.ncell;
    // the 27-bucket OR of each distinct bucket of the warp (sorted keys: a few per warp), its 27 masks
    // fetched by 27 lanes at once and combined by one warp reduction
    uint32_t acc = 0;
    unsigned todo = __ballot_sync(kFullMask, in);
    while (todo) {
        const uint32_t kb = __shfl_sync(kFullMask, k, __ffs(todo) - 1);
        int cx, cy, cz;
        decode_cell(P, kb, cx, cy, cz);
        uint32_t m = 0;
        if (lane < 27) {
            const int X = cx + lane % 3 - 1, Y = cy + (lane / 3) % 3 - 1, Z = cz + lane / 9 - 1;
            if (X >= 0 && X < P.dims[0] && Y >= 0 && Y < P.dims[1] && Z >= 0 && Z < P.dims[2])
                m = __ldg(mask + (uint32_t)X + (uint32_t)P.dims[0] * ((uint32_t)Y + (uint32_t)P.dims[1] * (uint32_t)Z));
        }
        const uint32_t orr = __reduce_or_sync(kFullMask, m);
        const bool mine = in && k == kb;
        if (mine) acc = orr;
        todo &= ~__ballot_sync(kFullMask, mine);
    }
    if (s < n) {
        uint8_t f = 0;
        if (in) {
            const uint32_t lab = lab_s[s];
            f = (acc & ~(1u << lab)) != 0u;
            if (f) atomicAdd(&cnt[lab], 1u);
        }
        flag[s] = f;
        comm[s] = f ? k : P.ncell;
    }
    __syncthreads();
    if (threadIdx.x < P.K_labels) block_counts[(size_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of the label-major block counts (single block of 1024 threads; K * nblk entries), total
// per label into label_total[0..K) and the overall total into label_total[K]. Each thread sums a chunk
// of consecutive entries, one block-wide scan offsets the chunks, and each thread writes its chunk's
// prefixes: one pass over the counts.
__global__ void __launch_bounds__(1024) k_comm_scan(uint32_t *__restrict__ block_counts, int64_t entries,
                                                    int nblk, int K, unsigned long long *__restrict__ label_total) {
    __shared__ uint32_t warp_tmp[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t chunk = (entries + 1023) / 1024;
    const int64_t b0 = (int64_t)threadIdx.x * chunk, b1 = b0 + chunk < entries ? b0 + chunk : entries;
    uint32_t v = 0;
    for (int64_t i = b0; i < b1; ++i) v += block_counts[i];
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) warp_tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = warp_tmp[l];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, t, o);
            if (l >= o) t += y;
        }
        warp_tmp[l] = t;
    }
    __syncthreads();
    uint32_t e = (w > 0 ? warp_tmp[w - 1] : 0u) + x - v;   // exclusive prefix of this chunk
    for (int64_t i = b0; i < b1; ++i) {
        const uint32_t c = block_counts[i];
        block_counts[i] = e;
        // the first entry of each label row starts that label's list
        if (i % nblk == 0) label_total[i / nblk] = e;
        e += c;
    }
    if (threadIdx.x == 1023) label_total[K] = warp_tmp[31];
}

// Stable compaction of the flagged slots into label-major lists (slot order = communication-hash
// order within a label, since slots are sorted by hash and flagged particles keep their hash).
__global__ void __launch_bounds__(CM_THREADS) k_boundary_scatter(int64_t n, const uint8_t *__restrict__ lab_s,
                                                                 const uint8_t *__restrict__ flag,
                                                                 const uint32_t *__restrict__ block_offsets,
                                                                 int nblk, uint32_t *__restrict__ out,
                                                                 uint32_t *__restrict__ hidx) {
    constexpr int W = CM_THREADS / 32;
    __shared__ uint32_t wc[W][kMaxLabel];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool f = s < n && flag[s];
    uint32_t lab = f ? lab_s[s] : 0xffffffffu;
    unsigned peers = __match_any_sync(kFullMask, lab);
    uint32_t rank = __popc(peers & lanemask_lt());
    for (int i = threadIdx.x; i < W * kMaxLabel; i += CM_THREADS) (&wc[0][0])[i] = 0;
    __syncthreads();
    if (f && (__ffs(peers) - 1) == l) wc[w][lab] = __popc(peers);
    __syncthreads();
    if (f) {
        uint32_t before = 0;
        for (int k = 0; k < w; ++k) before += wc[k][lab];
        const uint32_t at = block_offsets[(size_t)lab * nblk + blockIdx.x] + before + rank;
        out[at] = (uint32_t)s;
        if (hidx) hidx[s] = at;   // halo index of the two-pass interaction order
    }
}

// Large count arrays (many blocks, many labels): a two-level scan. Chunks of SC_CHUNK entries: the
// chunk sums (one block each), their exclusive scan (one block), then every chunk's prefixes offset by
// its chunk's prefix (one block each), all loads and stores coalesced.
constexpr int SC_THREADS = 1024, SC_PER = 4, SC_CHUNK = SC_THREADS * SC_PER;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &total) {
    __shared__ uint32_t wsum[SC_THREADS / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = wsum[l];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, t, o);
            if (l >= o) t += y;
        }
        wsum[l] = t;
    }
    __syncthreads();
    total = wsum[31];
    const uint32_t r = (w > 0 ? wsum[w - 1] : 0u) + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_partial(const uint32_t *__restrict__ a, int64_t entries,
                                                             uint32_t *__restrict__ part) {
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    uint32_t v = 0;
    for (int k = 0; k < SC_PER; ++k) {
        const int64_t i = base + (int64_t)k * SC_THREADS + threadIdx.x;
        if (i < entries) v += a[i];
    }
    uint32_t tot;
    block_exclusive_scan(v, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_chunks(uint32_t *__restrict__ part, int nchunk, int K,
                                                            unsigned long long *__restrict__ label_total) {
    const uint32_t v = threadIdx.x < nchunk ? part[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t e = block_exclusive_scan(v, tot);
    if (threadIdx.x < nchunk) part[threadIdx.x] = e;
    if (threadIdx.x == 0) label_total[K] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(uint32_t *__restrict__ a, int64_t entries,
                                                           const uint32_t *__restrict__ part, int nblk,
                                                           unsigned long long *__restrict__ label_total) {
    const int64_t i0 = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_PER;
    uint32_t c[SC_PER], v = 0;
    for (int k = 0; k < SC_PER; ++k) {
        c[k] = i0 + k < entries ? a[i0 + k] : 0u;
        v += c[k];
    }
    uint32_t tot;
    uint32_t e = block_exclusive_scan(v, tot) + part[blockIdx.x];
    for (int k = 0; k < SC_PER; ++k) {
        const int64_t i = i0 + k;
        if (i < entries) {
            a[i] = e;
            if (i % nblk == 0) label_total[i / nblk] = e;   // the first entry of each label row
        }
        e += c[k];
    }
}

cudaError_t launch_comm(const DevParams &P, int64_t n, const uint32_t *skey, const uint8_t *lab_s, uint32_t *mask,
                        uint8_t *flag, uint32_t *comm, uint32_t *block_counts, unsigned long long *label_total,
                        uint32_t *blist, uint32_t *hidx, uint32_t *scan_part, int *launches, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(mask, 0, (size_t)P.ncell * 4, s);
    if (e != cudaSuccess) return e;
    unsigned g = (unsigned)((n + CM_THREADS - 1) / CM_THREADS);
    k_label_mask<<<g, CM_THREADS, 0, s>>>(P, n, skey, lab_s, mask);
    k_comm<<<g, CM_THREADS, 0, s>>>(P, n, skey, lab_s, mask, flag, comm, block_counts, (int)g);
    const int64_t entries = (int64_t)P.K_labels * g;
    if (entries <= 8 * SC_CHUNK) {   // a few chunks: the one-block scan
        k_comm_scan<<<1, 1024, 0, s>>>(block_counts, entries, (int)g, P.K_labels, label_total);
        *launches = 4;
    } else {
        const int nchunk = (int)((entries + SC_CHUNK - 1) / SC_CHUNK);
        k_scan_partial<<<nchunk, SC_THREADS, 0, s>>>(block_counts, entries, scan_part);
        k_scan_chunks<<<1, SC_THREADS, 0, s>>>(scan_part, nchunk, P.K_labels, label_total);
        k_scan_apply<<<nchunk, SC_THREADS, 0, s>>>(block_counts, entries, scan_part, (int)g, label_total);
        *launches = 6;
    }
    k_boundary_scatter<<<g, CM_THREADS, 0, s>>>(n, lab_s, flag, block_counts, (int)g, blist, hidx);
    return cudaGetLastError();
}

int comm_blocks(int64_t n) { return (int)((n + CM_THREADS - 1) / CM_THREADS); }
// chunk sums of the two-level scan (K = 16 labels and 2^26 particles: 512 chunks)
int comm_scan_chunks(int64_t n) {
    return (int)(((int64_t)kMaxLabel * comm_blocks(n) + SC_CHUNK - 1) / SC_CHUNK) + 1;
}

// ---------------------------------------------------------------------------------------------
// Initialisation from user arrays (pos/vel n x 3 row-major).
// ---------------------------------------------------------------------------------------------
__global__ void k_init_state(DevParams P, int64_t n, const double *__restrict__ pos, const double *__restrict__ vel,
                             const double *__restrict__ vol, const uint8_t *__restrict__ mat,
                             const uint8_t *__restrict__ lab, State A, int *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
    A.f[FX][i] = pos[3 * i];
    A.f[FY][i] = pos[3 * i + 1];
    A.f[FZ][i] = pos[3 * i + 2];
    A.f[FVX][i] = vx;
    A.f[FVY][i] = vy;
    A.f[FVZ][i] = vz;
    uint8_t m = mat[i], l = lab[i];
    if (m >= P.nmat) { atomicOr(err, kErrMaterial); m = 0; }
    if (l >= P.K_labels) atomicOr(err, kErrLabel);
    A.f[FW][i] = vol[i];
    A.f[FM][i] = __dmul_rn(P.rho0[m], vol[i]);
    A.f[FE][i] = __dmul_rn(0.5, dist2_rn(vx, vy, vz));
    for (int k = FSXX; k <= FSYZ; ++k) A.f[k][i] = 0.0;
    A.mat[i] = m;
    A.label[i] = l;
    A.id[i] = (uint32_t)i;
    if (A.h) A.h[i] = P.h;   // variable h: every particle starts at the largest length
}

cudaError_t launch_init(const DevParams &P, int64_t n, const double *pos, const double *vel, const double *vol,
                        const uint8_t *mat, const uint8_t *lab, const State &A, int *err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_init_state<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, pos, vel, vol, mat, lab, A, err);
    return cudaGetLastError();
}

// Time step of the state A (slot order): every particle goes through the warp candidate filter, then
// k_dt_exact takes the exact FP64 maximum over the candidates.
__global__ void k_signal_max(DevParams P, int64_t n, State A, DtArgs d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < n;
    const int m = ok && A.mat[i] < P.nmat ? A.mat[i] : 0;
    dt_candidate(P, d, ok, m, ok ? A.f[FM][i] : 0.0, ok ? A.f[FW][i] : 1.0,
                 ok ? A.f[FVX][i] : 0.0, ok ? A.f[FVY][i] : 0.0, ok ? A.f[FVZ][i] : 0.0, ok ? A.f[FE][i] : 0.0,
                 (ok && P.variable_h) ? A.h[i] : 1.0);
}

// Exact FP64 maximum of the candidates' signal speeds (those whose upper bound reaches the largest
// lower bound), then dt = cfl h / max (variable h: cfl / max) by the last block to finish, which also
// clears the reduction words for the next step. A block loads its candidates, drops those equal bit for
// bit to the previous candidate (neighbouring warps of a uniform region list the same inputs), compacts
// the rest in shared memory and evaluates them densely. A list that overflowed its capacity falls back
// to every particle of S.
constexpr int DT_THREADS = 256;
__device__ __forceinline__ double dt_value(const DevParams &P, int mat, double m, double w, double vx, double vy,
                                           double vz, double E, double h) {
    double v = signal_speed64(P, mat, m, w, vx, vy, vz, E);
    if (P.variable_h) v = __ddiv_rn(v, h);
    return v;
}
__device__ __forceinline__ bool same_inputs(const DtCand &a, const DtCand &b) {
    return __double_as_longlong(a.m) == __double_as_longlong(b.m) && __double_as_longlong(a.w) == __double_as_longlong(b.w) &&
           __double_as_longlong(a.vx) == __double_as_longlong(b.vx) && __double_as_longlong(a.vy) == __double_as_longlong(b.vy) &&
           __double_as_longlong(a.vz) == __double_as_longlong(b.vz) && __double_as_longlong(a.E) == __double_as_longlong(b.E) &&
           __double_as_longlong(a.h) == __double_as_longlong(b.h) && a.mat == b.mat;
}
__global__ void __launch_bounds__(DT_THREADS) k_dt_exact(DevParams P, DtArgs d, int64_t n, State S,
                                                         double *__restrict__ dt) {
    __shared__ bool last;
    __shared__ unsigned nev, nq;
    __shared__ unsigned short q[DT_THREADS];
    __shared__ DtCand prev_sh;
    __shared__ unsigned long long wmax_sh[DT_THREADS / 32];
    const unsigned T = *(volatile unsigned *)&d.w->sig;
    const unsigned ncount = *(volatile unsigned *)&d.w->ccount;
    const unsigned hint = *(volatile unsigned *)&d.w->hint;
    // the largest signal speed this thread evaluates, as the bits of a non-NaN double (the maximum of the
    // bit patterns, which is what the global word keeps): one atomic per block instead of one per value,
    // and the same maximum whatever the grouping
    unsigned long long vmax = 0ull;
    if (threadIdx.x == 0) nev = 0u;
    if (ncount <= d.cap && T >= hint) {
        for (unsigned base = blockIdx.x * DT_THREADS; base < ncount; base += gridDim.x * DT_THREADS) {
            const unsigned k = base + threadIdx.x;
            if (threadIdx.x == 0) {
                nq = 0u;
                if (base > 0) prev_sh = d.cand[base - 1];
            }
            __syncthreads();
            DtCand c{};
            bool take = false;
            if (k < ncount) {
                c = d.cand[k];
                take = c.hi >= T;
                if (take && k > 0) {   // a run of equal candidates is evaluated once, at its start
                    const DtCand p = threadIdx.x > 0 ? d.cand[k - 1] : prev_sh;
                    take = !(p.hi >= T && same_inputs(p, c));
                }
            }
            if (take) q[atomicAdd(&nq, 1u)] = (unsigned short)threadIdx.x;
            __syncthreads();
            const unsigned m = nq;
            if (threadIdx.x < m) {
                const DtCand e = d.cand[base + q[threadIdx.x]];
                const double v = dt_value(P, e.mat, e.m, e.w, e.vx, e.vy, e.vz, e.E, e.h);
                if (v == v) vmax = max(vmax, (unsigned long long)__double_as_longlong(v));   // v >= 0
            }
            if (threadIdx.x == 0) nev += m;
            __syncthreads();
        }
    } else {   // overflow, or a listing threshold above this step's lower bound: every particle
        for (int64_t i = (int64_t)blockIdx.x * DT_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DT_THREADS) {
            const int m = S.mat[i] < P.nmat ? S.mat[i] : 0;
            const double v = dt_value(P, m, S.f[FM][i], S.f[FW][i], S.f[FVX][i], S.f[FVY][i], S.f[FVZ][i],
                                      S.f[FE][i], P.variable_h ? S.h[i] : 1.0);
            if (v == v) vmax = max(vmax, (unsigned long long)__double_as_longlong(v));
        }
        if (threadIdx.x == 0 && blockIdx.x == 0) nev = (unsigned)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(kFullMask, vmax, o));
    if ((threadIdx.x & 31) == 0) wmax_sh[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bm = 0ull;
        for (int w = 0; w < DT_THREADS / 32; ++w) bm = max(bm, wmax_sh[w]);
        if (bm) atomicMax(&d.w->sigd, bm);
        if (nev) atomicAdd(&d.w->eval, nev);
        __threadfence();
        last = atomicAdd(&d.w->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double mx = __longlong_as_double((long long)atomicAdd(&d.w->sigd, 0ull));
        *dt = P.variable_h ? __ddiv_rn(P.cfl, mx) : __ddiv_rn(__dmul_rn(P.cfl, P.h), mx);
        d.w->last_ccount = d.w->ccount;
        d.w->last_eval = atomicAdd(&d.w->eval, 0u);
        float delta = d.w->delta > 0.0f ? d.w->delta : 0x1p-10f;
        if (T < hint) delta = fminf(2.0f * delta, 0.5f);                   // the threshold was too tight
        else if (d.w->ccount > d.cap / 2) delta = fmaxf(0.5f * delta, 0x1p-16f);   // too wide
        d.w->delta = delta;
        d.w->hint = __float_as_uint(__fmul_rn(__uint_as_float(T), 1.0f - delta));
        d.w->sigd = 0ull;
        d.w->sig = 0u;
        d.w->ccount = 0u;
        d.w->done = 0u;
        d.w->eval = 0u;
    }
}

static unsigned dt_grid(int64_t n) {
    const int64_t g = (n + DT_THREADS - 1) / DT_THREADS;
    return (unsigned)(g < 1 ? 1 : (g > 304 ? 304 : g));
}

cudaError_t launch_dt_from_state(const DevParams &P, int64_t n, const State &A, const DtArgs &d, double *dt,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d.w, 0, offsetof(DtWords, last_ccount), s);
    if (e != cudaSuccess) return e;
    if (n > 0) k_signal_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, A, d);
    k_dt_exact<<<dt_grid(n), DT_THREADS, 0, s>>>(P, d, n, A, dt);
    return cudaGetLastError();
}

cudaError_t launch_finalize_dt(const DevParams &P, int64_t n, const DtArgs &d, const State &S, double *dt,
                               cudaStream_t s) {
    k_dt_exact<<<dt_grid(n), DT_THREADS, 0, s>>>(P, d, n, S, dt);
    return cudaGetLastError();
}

// FP64 conserved sums {m, m vx, m vy, m vz, m E, w}: per-block partials, then one block adds the
// partials in block order (deterministic).
__global__ void __launch_bounds__(256) k_conserved_partial(int64_t n, State A, double *__restrict__ part) {
    __shared__ double sh[6][256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (i < n) {
        double m = A.f[FM][i];
        v[0] = m;
        v[1] = m * A.f[FVX][i];
        v[2] = m * A.f[FVY][i];
        v[3] = m * A.f[FVZ][i];
        v[4] = m * A.f[FE][i];
        v[5] = A.f[FW][i];
    }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 6) part[(size_t)blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_conserved_final(int nblk, const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * 6 + threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

cudaError_t launch_conserved(int64_t n, const State &A, double *part, double *out, cudaStream_t s) {
    int nblk = (int)((n + 255) / 256);
    if (nblk < 1) nblk = 1;
    k_conserved_partial<<<nblk, 256, 0, s>>>(n, A, part);
    k_conserved_final<<<1, 32, 0, s>>>(nblk, part, out);
    return cudaGetLastError();
}

}  // namespace gsph
