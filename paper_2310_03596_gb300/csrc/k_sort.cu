// k_sort.cu - bucket hash (Sec. I) and the LSD radix sort of (hash, slot) pairs (Sec. I).
//
// Radix sort: ceil(bits / 9) passes of equal digits of at most 9 bits (18-bit bucket hashes: two passes
// of 9), the last digit masked to the requested bits. Each pass is three launches:
//   k_rs_hist    per-tile digit histogram (tile = 2048 keys), warp-aggregated shared atomics;
//   k_rs_rowscan one block per digit value: exclusive scan of its per-tile counts, digit total;
//   k_rs_scatter reloads the tile, ranks each key among equal digits in tile order (warp match_any,
//                per-warp counters, cross-warp prefix), scatters keys and values.
// The ranking follows tile order, so every pass is stable and the sort is stable overall. In a step the
// bucket hash (k_hash_hist) builds the first pass's tile histogram as it writes the keys. The hash and
// the launches after it are programmatic dependent launches (pdl_launch): each kernel's blocks may be
// scheduled while its predecessor drains and wait for it in pdl_wait(), which hides the launch gaps of
// these short kernels. In a step the hash counts no particles outside the grid (garbage = null): the
// reorder reads their count off the sorted keys.
// Bytes per key per pass: 4 (hist) + 8 read + 8 written (scatter) + 2*4*bins/2048 (counts).
#include <mutex>

#include "gsph_internal.cuh"

namespace gsph {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_MAX_DIGIT = 9;
constexpr int RS_BINS = 1 << RS_MAX_DIGIT;   // histogram rows allocated per tile (the widest digit)

// Item order inside a tile: warp-major, then round, then lane (each round reads 32 consecutive
// keys, so loads are coalesced and the item order is the key order).
__device__ __forceinline__ int64_t rs_item(int64_t tile_base, int w, int r, int l) {
    return tile_base + (int64_t)w * (32 * RS_IPT) + r * 32 + l;
}

template <int DIG>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                        uint32_t dmask, uint32_t *__restrict__ hist, int nblk) {
    pdl_wait();
    pdl_release();
    constexpr int BINS = 1 << DIG;
    __shared__ uint32_t sh[BINS];
    for (int i = threadIdx.x; i < BINS; i += RS_THREADS) sh[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t idx = rs_item(base, w, r, l);
        bool valid = idx < n;
        uint32_t d = valid ? (__ldg(keys + idx) >> shift) & dmask : 0xffffffffu;
        unsigned peers = __match_any_sync(kFullMask, d);
        if (valid && (__ffs(peers) - 1) == l) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BINS; i += RS_THREADS) hist[(size_t)i * nblk + blockIdx.x] = sh[i];
}

// Block-wide exclusive scan helper (blockDim.x == 1024); returns the exclusive prefix of v and
// the block total in *total.
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *warp_tmp, uint32_t *total) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) warp_tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = warp_tmp[l];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, s, o);
            if (l >= o) s += y;
        }
        warp_tmp[l] = s;  // inclusive over warps
    }
    __syncthreads();
    uint32_t before = (w > 0 ? warp_tmp[w - 1] : 0u) + x - v;
    *total = warp_tmp[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(1024) k_rs_rowscan(uint32_t *__restrict__ hist, int nblk,
                                                     uint32_t *__restrict__ tot) {
    pdl_wait();
    pdl_release();
    __shared__ uint32_t warp_tmp[32];
    uint32_t *row = hist + (size_t)blockIdx.x * nblk;
    uint32_t carry = 0;
    for (int b = 0; b < nblk; b += 1024) {
        int i = b + threadIdx.x;
        uint32_t v = i < nblk ? row[i] : 0u;
        uint32_t t;
        uint32_t e = block_excl_scan_1024(v, warp_tmp, &t);
        if (i < nblk) row[i] = carry + e;
        carry += t;
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

template <int DIG>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin,
                                                           uint32_t *__restrict__ kout,
                                                           uint32_t *__restrict__ vout, int64_t n, int shift,
                                                           uint32_t dmask, const uint32_t *__restrict__ hist,
                                                           const uint32_t *__restrict__ tot, int nblk) {
    pdl_wait();
    pdl_release();
    constexpr int BINS = 1 << DIG;
    constexpr int DPT = BINS / RS_THREADS;   // digit values per thread in the per-digit phases
    static_assert(DPT >= 1 && BINS % RS_THREADS == 0, "digit width");
    __shared__ uint32_t wcnt[RS_WARPS][BINS];
    __shared__ uint32_t base_sh[BINS];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    // digit bases: exclusive scan of the digit totals plus this tile's exclusive offset; thread t
    // holds digits t*DPT .. t*DPT + DPT - 1
    {
        const int d0 = threadIdx.x * DPT;
        uint32_t loc[DPT], sum = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            loc[q] = sum;
            sum += tot[d0 + q];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, x, o);
            if (l >= o) x += y;
        }
        __shared__ uint32_t ws[RS_WARPS];
        if (l == 31) ws[w] = x;
#pragma unroll
        for (int q = 0; q < DPT; ++q)
            for (int k = 0; k < RS_WARPS; ++k) wcnt[k][d0 + q] = 0;
        __syncthreads();
        uint32_t pre = 0;
        for (int k = 0; k < w; ++k) pre += ws[k];
        pre += x - sum;
#pragma unroll
        for (int q = 0; q < DPT; ++q) base_sh[d0 + q] = pre + loc[q] + hist[(size_t)(d0 + q) * nblk + blockIdx.x];
    }
    __syncthreads();
    uint32_t key[RS_IPT], val[RS_IPT], rank[RS_IPT];
#pragma unroll
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t idx = rs_item(base, w, r, l);
        bool valid = idx < n;
        key[r] = valid ? __ldg(kin + idx) : 0xffffffffu;
        val[r] = valid ? __ldg(vin + idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_IPT; ++r) {
        uint32_t d = (key[r] >> shift) & dmask;
        unsigned peers = __match_any_sync(kFullMask, d);
        uint32_t before = wcnt[w][d];
        rank[r] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if ((__ffs(peers) - 1) == l) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = threadIdx.x * DPT + q;
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < RS_WARPS; ++k) {
            uint32_t t = wcnt[k][d];
            wcnt[k][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t idx = rs_item(base, w, r, l);
        if (idx < n) {
            uint32_t d = (key[r] >> shift) & dmask;
            uint32_t pos = base_sh[d] + wcnt[w][d] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// Sec. I: bucket hash of every slot fused with the first sort pass's tile histogram: the same tiles
// and item order as k_rs_hist, so the histogram is the one k_rs_hist would build from the keys written
// here (the first digit: shift 0, mask dmask). val = slot; particles outside the grid are counted.
template <int DIG>
__global__ void __launch_bounds__(RS_THREADS) k_hash_hist(DevParams P, int64_t n, const double *__restrict__ x,
                                                          const double *__restrict__ y, const double *__restrict__ z,
                                                          uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                                          unsigned long long *__restrict__ garbage, uint32_t dmask,
                                                          uint32_t *__restrict__ hist, int nblk,
                                                          uint2 *__restrict__ zero8, int64_t nzero8,
                                                          uint32_t *__restrict__ zero4, int64_t nzero4) {
    pdl_wait();
    pdl_release();
    constexpr int BINS = 1 << DIG;
    __shared__ uint32_t sh[BINS];
    for (int i = threadIdx.x; i < BINS; i += RS_THREADS) sh[i] = 0;
    // buffers that later kernels of the step fill (the bucket ranges, the swap pass's sums) cleared here,
    // so that no separate clearing breaks the launch chain; nothing reads them before the sort ends
    const int64_t gstride = (int64_t)gridDim.x * RS_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < nzero8; i += gstride) zero8[i] = make_uint2(0u, 0u);
    for (int64_t i = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < nzero4; i += gstride) zero4[i] = 0u;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    unsigned gc = 0;
#pragma unroll 4
    for (int r = 0; r < RS_IPT; ++r) {
        const int64_t idx = rs_item(base, w, r, l);
        const bool valid = idx < n;
        uint32_t k = 0u;
        if (valid) {
            k = hash_of(P, x[idx], y[idx], z[idx]);
            key[idx] = k;
            val[idx] = (uint32_t)idx;
        }
        gc += (unsigned)__popc(__ballot_sync(kFullMask, valid && k == P.ncell));
        const uint32_t d = valid ? (k & dmask) : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFullMask, d);
        if (valid && (__ffs(peers) - 1) == l) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    if (garbage && l == 0 && gc) atomicAdd(garbage, (unsigned long long)gc);
    __syncthreads();
    for (int i = threadIdx.x; i < BINS; i += RS_THREADS) hist[(size_t)i * nblk + blockIdx.x] = sh[i];
}

// Sec. I: bucket hash of every slot; val = slot. Counts particles outside the grid.
__global__ void k_hash(DevParams P, int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                       unsigned long long *__restrict__ garbage) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool g = false;
    if (i < n) {
        uint32_t k = hash_of(P, x[i], y[i], z[i]);
        key[i] = k;
        val[i] = (uint32_t)i;
        g = (k == P.ncell);
    }
    unsigned b = __ballot_sync(kFullMask, g);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(garbage, (unsigned long long)__popc(b));
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
static inline int rs_nblk(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

size_t radix_hist_words(int64_t n) { return (size_t)RS_BINS * (size_t)(rs_nblk(n) > 0 ? rs_nblk(n) : 1); }

// Sorts (k0, v0) by the low `bits` bits using (k1, v1) as the other buffer. Returns true when the
// result ends in (k1, v1).
int radix_passes(int bits) { return (bits + RS_MAX_DIGIT - 1) / RS_MAX_DIGIT; }

// first_hist: the first pass's tile histogram is already in hist (k_hash_hist).
cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t *hist,
                             uint32_t *tot, int64_t n, int bits, cudaStream_t s, bool *in_alt, bool first_hist) {
    *in_alt = false;
    if (n <= 0) return cudaSuccess;
    int nblk = rs_nblk(n);
    const int passes = radix_passes(bits);
    const int dig = (bits + passes - 1) / passes;   // <= 9
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < passes; ++p) {
        const int shift = dig * p;
        const int width = bits - shift < dig ? bits - shift : dig;
        const uint32_t dmask = (1u << width) - 1u;
        const bool hist_done = first_hist && p == 0;
        if (dig > 8) {
            if (!hist_done && (e = pdl_launch(k_rs_hist<9>, dim3(nblk), dim3(RS_THREADS), s, (const uint32_t *)ki, n,
                                              shift, dmask, hist, nblk)) != cudaSuccess)
                return e;
            if ((e = pdl_launch(k_rs_rowscan, dim3(1u << 9), dim3(1024), s, hist, nblk, tot)) != cudaSuccess) return e;
            if ((e = pdl_launch(k_rs_scatter<9>, dim3(nblk), dim3(RS_THREADS), s, (const uint32_t *)ki,
                                (const uint32_t *)vi, ko, vo, n, shift, dmask, (const uint32_t *)hist,
                                (const uint32_t *)tot, nblk)) != cudaSuccess)
                return e;
        } else {
            if (!hist_done && (e = pdl_launch(k_rs_hist<8>, dim3(nblk), dim3(RS_THREADS), s, (const uint32_t *)ki, n,
                                              shift, dmask, hist, nblk)) != cudaSuccess)
                return e;
            if ((e = pdl_launch(k_rs_rowscan, dim3(1u << 8), dim3(1024), s, hist, nblk, tot)) != cudaSuccess) return e;
            if ((e = pdl_launch(k_rs_scatter<8>, dim3(nblk), dim3(RS_THREADS), s, (const uint32_t *)ki,
                                (const uint32_t *)vi, ko, vo, n, shift, dmask, (const uint32_t *)hist,
                                (const uint32_t *)tot, nblk)) != cudaSuccess)
                return e;
        }
        uint32_t *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    *in_alt = (passes & 1) != 0;
    return cudaGetLastError();
}

// The hash with the first pass's histogram of a sort by the low `bits` bits (radix_sort_pairs with
// first_hist = true follows). It also clears zero8[0, nzero8) and zero4[0, nzero4) (either may be empty),
// buffers that kernels after the sort fill.
cudaError_t launch_hash_hist(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                             uint32_t *key, uint32_t *val, unsigned long long *garbage, uint32_t *hist, int bits,
                             uint2 *zero8, int64_t nzero8, uint32_t *zero4, int64_t nzero4, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nblk = rs_nblk(n);
    const int passes = radix_passes(bits);
    const int dig = (bits + passes - 1) / passes;
    const int width = bits < dig ? bits : dig;
    const uint32_t dmask = (1u << width) - 1u;
    if (dig > 8)
        return pdl_launch(k_hash_hist<9>, dim3(nblk), dim3(RS_THREADS), s, P, n, x, y, z, key, val, garbage, dmask,
                          hist, nblk, zero8, nzero8, zero4, nzero4);
    return pdl_launch(k_hash_hist<8>, dim3(nblk), dim3(RS_THREADS), s, P, n, x, y, z, key, val, garbage, dmask, hist,
                      nblk, zero8, nzero8, zero4, nzero4);
    return cudaGetLastError();
}

cudaError_t launch_hash(const DevParams &P, int64_t n, const double *x, const double *y, const double *z,
                        uint32_t *key, uint32_t *val, unsigned long long *garbage, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int th = 256;
    k_hash<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(P, n, x, y, z, key, val, garbage);
    return cudaGetLastError();
}

}  // namespace gsph

// ---------------------------------------------------------------------------------------------
// Stateless C-ABI sort
// ---------------------------------------------------------------------------------------------
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" size_t gsph_radix_sort_workspace(int64_t n, int32_t key_bits) {
    (void)key_bits;
    if (n < 0) return 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    return align256(nn * 4) * 2 + align256(gsph::radix_hist_words(n) * 4) + align256(gsph::RS_BINS * 4);
}

extern "C" gsph_status gsph_radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int32_t key_bits,
                                             void *workspace, size_t workspace_bytes, void *stream) {
    if (n < 0 || n >= ((int64_t)1 << 31) || key_bits < 1 || key_bits > 32) return GSPH_INVALID_ARG;
    if (n == 0) return GSPH_OK;
    if (!keys || !vals || !workspace) return GSPH_INVALID_ARG;
    if (workspace_bytes < gsph_radix_sort_workspace(n, key_bits)) return GSPH_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *p = (char *)workspace;
    uint32_t *k1 = (uint32_t *)p;
    p += align256((size_t)n * 4);
    uint32_t *v1 = (uint32_t *)p;
    p += align256((size_t)n * 4);
    uint32_t *hist = (uint32_t *)p;
    p += align256(gsph::radix_hist_words(n) * 4);
    uint32_t *tot = (uint32_t *)p;
    bool alt = false;
    cudaError_t e = gsph::radix_sort_pairs(keys, vals, k1, v1, hist, tot, n, key_bits, s, &alt, false);
    if (e == cudaSuccess && alt) {
        e = cudaMemcpyAsync(keys, k1, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, v1, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    }
    return e == cudaSuccess ? GSPH_OK : GSPH_CUDA_ERROR;
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the stateless sort. The scratch lives in a fixed device array of this
// library (held on every GPU that loads the library until the process exits), so the call needs no
// cudaMalloc/cudaFree and no caller-provided workspace.
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocMaxN = (int64_t)1 << 20;
constexpr size_t kNoAllocKeyBytes = (size_t)kNoAllocMaxN * 4;
constexpr size_t kNoAllocHistBytes = (size_t)gsph::RS_BINS * (size_t)(kNoAllocMaxN / gsph::RS_TILE) * 4;
constexpr size_t kNoAllocBytes = 2 * kNoAllocKeyBytes + kNoAllocHistBytes + gsph::RS_BINS * 4;
static_assert(kNoAllocBytes == (size_t)GSPH_SORT_NOALLOC_BYTES, "GSPH_SORT_NOALLOC_BYTES in gsph.h");
static_assert(kNoAllocKeyBytes % 256 == 0 && kNoAllocHistBytes % 256 == 0, "256-byte aligned sections");

static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_sort_scratch on the current device, looked up once per device. In host code
// the array's name only stands for it; the address that kernels may use comes from the runtime.
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" gsph_status gsph_radix_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t key_bits,
                                                     void *stream) {
    if (n < 0 || n > kNoAllocMaxN || key_bits < 1 || key_bits > 32) return GSPH_INVALID_ARG;
    if (n == 0) return GSPH_OK;
    if (!keys || !vals) return GSPH_INVALID_ARG;
    void *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return GSPH_CUDA_ERROR;
    cudaStream_t s = (cudaStream_t)stream;
    char *p = (char *)base;
    uint32_t *k1 = (uint32_t *)p;
    uint32_t *v1 = (uint32_t *)(p + kNoAllocKeyBytes);
    uint32_t *hist = (uint32_t *)(p + 2 * kNoAllocKeyBytes);
    uint32_t *tot = (uint32_t *)(p + 2 * kNoAllocKeyBytes + kNoAllocHistBytes);
    // every scratch word the sort reads is written earlier in the same call (per-tile histograms,
    // their scans, the other key/value buffer), so nothing has to be cleared between calls
    bool alt = false;
    cudaError_t e = gsph::radix_sort_pairs(keys, vals, k1, v1, hist, tot, n, key_bits, s, &alt, false);
    if (e == cudaSuccess && alt) {
        e = cudaMemcpyAsync(keys, k1, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, v1, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    }
    return e == cudaSuccess ? GSPH_OK : GSPH_CUDA_ERROR;
}
