// gsph_internal.cuh - device-side layout and helpers shared by the CUDA translation units of libgsph.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsph.h"

namespace gsph {

constexpr int kMaxMat = GSPH_MAX_MATERIALS;
constexpr int kMaxWall = GSPH_MAX_WALLS;
constexpr int kMaxLabel = GSPH_MAX_LABELS;
constexpr int kNRate = GSPH_NRATE;
constexpr uint32_t kFullMask = 0xffffffffu;

// Device error bits (OR-ed into Ctx::d_err).
constexpr int kErrLabel = 1;      // a label >= K
constexpr int kErrMaterial = 2;   // a material >= n_materials
constexpr int kErrTimeout = 4;    // a bounded device wait gave up

// Parameters every kernel receives by value.
struct DevParams {
    double lo[3];
    double cell;         // bucket side 2h
    double R2;           // (2h)^2, the strict support predicate r^2 < R2
    double h;
    double cfl;
    double g[3];
    double wall_pos[kMaxWall];
    double rho0[kMaxMat], K[kMaxMat], G[kMaxMat], Y[kMaxMat];
    double Mmod[kMaxMat];    // K + (4 G) / 3, the longitudinal modulus
    double kdw;              // 5 * 21 / (16 pi h^3) / h: |dW/dr| = kdw * q (1 - q/2)^3
    double alpha;
    int dims[3];
    uint32_t ncell;          // grid product; the garbage hash
    int nwalls;
    int wall_axis[kMaxWall];
    int nmat;
    int K_labels;
    int has_gravity;         // g != 0
    // FP32 copies for the split path
    float f_cell, f_inv_h, f_kdw, f_R2lo, f_R2hi;
    float f_inv_cell;        // FP32 rounding of the FP64 reciprocal of the bucket side
    float f_lo[3];           // FP32 roundings of the grid's lower corner (the hash's fast path)
    float f_rho0[kMaxMat], f_K[kMaxMat], f_G[kMaxMat], f_Mmod[kMaxMat];
    // FP32 roundings for the time step's signal-speed bounds: c0, s - 1, gamma0, 4G/3
    float f_c0[kMaxMat], f_sm1[kMaxMat], f_g0[kMaxMat], f_G43[kMaxMat];
    // equation of state per material (0 linear, 1 Mie-Gruneisen) and pressure cut-off
    int eos[kMaxMat];
    double c0[kMaxMat], s_hug[kMaxMat], gamma0[kMaxMat], p_min[kMaxMat];
    double inv_rho0[kMaxMat], k0[kMaxMat], inv_2rho0[kMaxMat];   // 1/rho0, rho0 c0^2, 1/(2 rho0)
    // variable smoothing lengths: support r^2 < (h_i + h_j)^2; the FP32 list test decides outside the
    // relative band [1 - d, 1 + d] around it (d = kVarBand, wide enough for size ratios up to 4)
    int variable_h;
    float f_vlo, f_vhi;      // 1 - d, 1 + d
    float f_k5;              // |dW/dr| = k5 (1 / (h_i + h_j))^5 r (1 - r / (h_i + h_j))^3: 210 / pi
    double k5;
    // fixed-point Cg of the swap pass (Sec. III.A): q = nearest integer to (x - lo) q_s, q_s = 2^32 / L,
    // Cg = lo + mean(q) q_step, q_step = L 2^-32, L = dims * 2h the grid extent per axis
    double q_s[3], q_step[3];
    double wall_reach;       // (2h)(1 + 1e-6): beyond this distance from a wall plane no image is in the support
    // bucket corners per axis, fma(c, 2h, lo) for c in [0, dims): device tables of the buffer set
    const double *corner[3];
};
constexpr double kVarBand = 1.0e-3;

// Buffers, stream and events of the two-pass interaction order (Sec. II steps d-f), host side.
struct OverlapBufs {
    const uint8_t *flag;                 // MGPU boundary flag per slot
    const uint32_t *blist;               // boundary list (halo index -> slot)
    const unsigned long long *btotal;    // boundary set size (device)
    const uint32_t *hidx;                // slot -> halo index
    void *hpos, *hrec;                   // halo records (interaction record layout of the path)
    float *hcx;                          // halo bucket x
    void *part;                          // parked partial sums, 120 bytes per particle
    int32_t *part_cnt;                   // parked neighbour counts, 2 per particle
    cudaStream_t aux;                    // the second stream (halo gather)
    cudaEvent_t ev_fork, ev_join;        // launch stream -> aux, aux -> launch stream
    cudaEvent_t ev_halo0, ev_halo1, ev_local;   // timing only (null when not timing)
    unsigned gather_grid, boundary_grid;
};

// FP64 state in structure-of-arrays form.
struct State {
    double *f[15];           // x y z vx vy vz w m E sxx syy szz sxy sxz syz
    uint8_t *mat, *label;
    uint32_t *id;
    double *h;               // per-particle smoothing length (variable h), else null
};
enum { FX = 0, FY, FZ, FVX, FVY, FVZ, FW, FM, FE, FSXX, FSYY, FSZZ, FSXY, FSXZ, FSYZ };

// Positions of the swap pass (Sec. III.A): FP32 roundings (the balancing hash's fast path), FP64 (its
// exact fallback) and the fixed-point coordinates of the Cg sums (quantise64).
struct SwapPos {
    const float *x, *y, *z;
    const double *X, *Y, *Z;
    const uint32_t *qx, *qy, *qz;
};

// Interaction records of sorted particles.
// Split path: pos4 = (x, y, z relative to the particle's own bucket corner, w) in FP32 and
// rec = {(vx, vy, vz, rho), (p, Z, E, sxx), (syy, sxy, sxz, syz)}; szz = -(sxx + syy).
struct RecF { float4 a, b, c; };
// 32-byte aligned FP64 4-vector (loads as one 256-bit or two 128-bit transactions).
struct __align__(32) D4 { double x, y, z, w; };
__host__ __device__ __forceinline__ D4 make_d4(double x, double y, double z, double w) { return D4{x, y, z, w}; }
// FP64 path: pos = (x, y, z, w) absolute and rec = {(vx, vy, vz, rho), (p, Z, E, sxx),
// (syy, szz, sxy, sxz), (syz, -, -, -)}.
struct RecD { D4 a, b, c, d; };

// ---------------------------------------------------------------------------------------------
// Exactly rounded FP64 helpers: every product and sum rounded separately (no contraction), so that
// the integer decisions made from them (hash, support predicate, balancing hash) are the same on
// any IEEE machine that evaluates the same operation sequence.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double dist2_rn(double dx, double dy, double dz) {
    double a = __dmul_rn(dx, dx);
    double b = __dmul_rn(dy, dy);
    double c = __dmul_rn(dz, dz);
    return __dadd_rn(__dadd_rn(a, b), c);
}

// Bucket coordinate along one axis: -1 below the grid, dim at or beyond the top.
__device__ __forceinline__ int bucket_coord(double x, double lo, double cell, int dim) {
    double t = __ddiv_rn(__dsub_rn(x, lo), cell);
    if (!(t >= 0.0)) return -1;
    if (t >= (double)dim) return dim;
    return (int)t;
}

// FP32 value of x with the FP64 significand truncated (|x - f| < 2^-23 |x|), formed with integer
// operations from the bits; false when x is zero, infinite, NaN or outside the FP32 normal range.
__device__ __forceinline__ bool trunc_to_f32(double x, float &f) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e < 1023 - 126 || e > 1023 + 127) return false;
    f = __uint_as_float((hi & 0x80000000u) | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    return true;
}

// bucket_coord without an FP64 operation in the common case. With xt the truncated FP32 value of x
// (below 2^-23 |x| away), lof the FP32 rounding of lo (2^-24 |lo|), and three FP32 roundings (the
// difference, the reciprocal 1/cell and the product), the FP32 quotient tf lies within
// 2^-23 |x| / cell + 2^-24 |lo| / cell + 3.01 * 2^-24 |tf| of the exact (x - lo) / cell, and the
// correctly rounded FP64 quotient t within another 2^-52 |t|. When tf is farther than
// 2^-22 (|tf| + 1 + (|xt| + |lof|) / cell) from every integer, t lies strictly between the same two
// integers and floor(tf) = floor(t). Otherwise (near a bucket face, x zero, NaN, infinite or beyond the
// FP32 normal range, a difference below that range, a reciprocal that is not a normal FP32 number -
// passed as NaN) the FP64 division decides.
__device__ __forceinline__ int bucket_coord_fast(double x, double lo, float lof, double cell, float inv_cell, int dim) {
    float xt;
    if (trunc_to_f32(x, xt)) {
        const float df = __fsub_rn(xt, lof);
        const float tf = __fmul_rn(df, inv_cell);
        const float fl = floorf(tf);
        const float fr = __fsub_rn(tf, fl);   // exact
        const float span = __fmul_rn(__fadd_rn(fabsf(xt), fabsf(lof)), inv_cell);
        const float eps = __fmul_rn(0x1p-22f, __fadd_rn(__fadd_rn(fabsf(tf), 1.0f), span));
        if (fr > eps && fr < __fsub_rn(1.0f, eps) && fabsf(df) >= 0x1p-126f) {
            if (fl < 0.0f) return -1;
            if (fl >= (float)dim) return dim;
            return (int)fl;
        }
    }
    return bucket_coord(x, lo, cell, dim);
}

__device__ __forceinline__ int bucket_coord_signed(double x, double lo, double cell) {
    return (int)floor(__ddiv_rn(__dsub_rn(x, lo), cell));
}

__device__ __forceinline__ uint32_t hash_of(const DevParams &P, double x, double y, double z) {
    int cx = bucket_coord_fast(x, P.lo[0], P.f_lo[0], P.cell, P.f_inv_cell, P.dims[0]);
    int cy = bucket_coord_fast(y, P.lo[1], P.f_lo[1], P.cell, P.f_inv_cell, P.dims[1]);
    int cz = bucket_coord_fast(z, P.lo[2], P.f_lo[2], P.cell, P.f_inv_cell, P.dims[2]);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= P.dims[0] || cy >= P.dims[1] || cz >= P.dims[2]) return P.ncell;
    return (uint32_t)cx + (uint32_t)P.dims[0] * ((uint32_t)cy + (uint32_t)P.dims[1] * (uint32_t)cz);
}

// Fixed-point coordinate of the swap pass's Cg sums: nearest integer (ties to even) to (x - lo) s, clamped
// to [0, 2^32 - 1] (NaN gives 0).
__device__ __forceinline__ uint32_t quantise64(double x, double lo, double s) {
    const double t = __dmul_rn(__dsub_rn(x, lo), s);
    const long long b = __double_as_longlong(t);
    if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) return 0u;   // NaN
    long long q = __double2ll_rn(t);                                   // saturates beyond the int64 range
    q = q < 0 ? 0 : (q > 4294967295LL ? 4294967295LL : q);
    return (uint32_t)q;
}

__device__ __forceinline__ void decode_cell(const DevParams &P, uint32_t c, int &cx, int &cy, int &cz) {
    cx = (int)(c % (uint32_t)P.dims[0]);
    uint32_t r = c / (uint32_t)P.dims[0];
    cy = (int)(r % (uint32_t)P.dims[1]);
    cz = (int)(r / (uint32_t)P.dims[1]);
}

// ---------------------------------------------------------------------------------------------
// CFL time step (Sec. II step g): dt = cfl h / max_i s_i with the signal speed s_i = c_i + |v_i| in FP64
// (variable h: dt = cfl / max_i (s_i / h_i)). The FP64 sequence below is the definition; a step never
// evaluates it for every particle (GB300's FP64 units are scarce). Each particle first evaluates s in
// FP32 together with a bound of the FP32 value's distance from the FP64 one (a running error bound,
// below), giving an interval [lo, hi] that contains the FP64 value. The largest lo over all particles is
// a lower bound of the FP64 maximum, so only particles whose hi reaches it can attain the maximum. A warp
// first keeps its lanes whose hi reaches the warp's largest lo, drops the lanes whose FP64 inputs equal
// bit for bit those of the lane holding that lo (same inputs, same FP64 value), and appends the rest to
// a candidate list; a second kernel keeps the candidates whose hi reaches the grid's largest lo,
// evaluates their FP64 signal speed, takes the exact maximum and forms dt.
// ---------------------------------------------------------------------------------------------

// FP64 signal speed of one particle, each operation rounded (no contraction): rho = m / w,
// |v|^2 = (vx^2 + vy^2) + vz^2; linear EOS c = sqrt(M / rho), M = K + 4G/3; Mie-Gruneisen
// c = sqrt(cb2 + (4G/3) / rho) with cb2 the isentropic bulk term at e = E - |v|^2 / 2, floored at 0.
__device__ __forceinline__ double signal_speed64(const DevParams &P, int mat, double m, double w, double vx,
                                                 double vy, double vz, double E) {
    const double rho = __ddiv_rn(m, w);
    const double v2 = dist2_rn(vx, vy, vz);
    double c;
    if (P.eos[mat] == 0) {
        c = __dsqrt_rn(__ddiv_rn(P.Mmod[mat], rho));
    } else {
        const double rho0 = P.rho0[mat], c0 = P.c0[mat], g0 = P.gamma0[mat];
        const double e = __dsub_rn(E, __dmul_rn(v2, 0.5));
        const double mu = __dsub_rn(__ddiv_rn(rho, rho0), 1.0);
        const double k0 = __dmul_rn(__dmul_rn(rho0, c0), c0);
        const double q = __dadd_rn(1.0, mu);
        double pH, dpH;
        if (mu > 0.0) {
            const double sm1 = __dsub_rn(P.s_hug[mat], 1.0);
            const double D = __dsub_rn(1.0, __dmul_rn(sm1, mu));
            pH = __ddiv_rn(__dmul_rn(__dmul_rn(k0, mu), q), __dmul_rn(D, D));
            const double a1 = __dmul_rn(__dadd_rn(1.0, __dmul_rn(2.0, mu)), D);
            const double a2 = __dmul_rn(__dmul_rn(__dmul_rn(2.0, sm1), mu), q);
            dpH = __ddiv_rn(__dmul_rn(k0, __dadd_rn(a1, a2)), __dmul_rn(__dmul_rn(D, D), D));
        } else {
            pH = __dmul_rn(k0, mu);
            dpH = k0;
        }
        const double r2 = __dmul_rn(2.0, rho0);
        const double eH = __ddiv_rn(__dmul_rn(pH, mu), __dmul_rn(r2, q));
        const double deH = __ddiv_rn(__dadd_rn(__dmul_rn(__dmul_rn(dpH, mu), q), pH), __dmul_rn(__dmul_rn(r2, q), q));
        const double gr = __dmul_rn(g0, rho0);
        const double p = __dadd_rn(pH, __dmul_rn(gr, __dsub_rn(e, eH)));
        double cb2 = __dadd_rn(__ddiv_rn(__dsub_rn(dpH, __dmul_rn(gr, deH)), rho0),
                               __ddiv_rn(__dmul_rn(__dmul_rn(p, g0), rho0), __dmul_rn(rho, rho)));
        if (cb2 < 0.0) cb2 = 0.0;
        const double G43 = __ddiv_rn(__dmul_rn(4.0, P.G[mat]), 3.0);
        c = __dsqrt_rn(__dadd_rn(cb2, __ddiv_rn(G43, rho)));
    }
    return __dadd_rn(c, __dsqrt_rn(v2));
}

// FP32 value with a bound e of its absolute distance from the exact value of the same expression on the
// exact inputs. Each operation adds the propagated bounds of its operands and its own rounding (at most
// 2^-24 of the result); a division by an operand whose bound reaches its magnitude, or an overflow,
// gives an infinite bound.
struct FErr { float v, e; };
constexpr float kU32 = 0x1p-24f;
__device__ __forceinline__ FErr fe_in(double x) {   // FP32 rounding of an exact FP64 input
    const float v = __double2float_rn(x);
    return FErr{v, __fmul_rn(kU32, fabsf(v))};
}
__device__ __forceinline__ FErr fe_add(FErr a, FErr b) {
    const float v = __fadd_rn(a.v, b.v);
    return FErr{v, __fadd_rn(__fadd_rn(a.e, b.e), __fmul_rn(kU32, fabsf(v)))};
}
__device__ __forceinline__ FErr fe_sub(FErr a, FErr b) {
    const float v = __fsub_rn(a.v, b.v);
    return FErr{v, __fadd_rn(__fadd_rn(a.e, b.e), __fmul_rn(kU32, fabsf(v)))};
}
__device__ __forceinline__ FErr fe_mul(FErr a, FErr b) {
    const float v = __fmul_rn(a.v, b.v);
    const float e = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(a.v), b.e), __fmul_rn(fabsf(b.v), a.e)), __fmul_rn(a.e, b.e));
    return FErr{v, __fadd_rn(e, __fmul_rn(kU32, fabsf(v)))};
}
__device__ __forceinline__ FErr fe_div(FErr a, FErr b) {
    const float v = __fdiv_rn(a.v, b.v);
    const float den = __fsub_rn(fabsf(b.v), b.e);
    float e = den > 0.0f ? __fdiv_rn(__fadd_rn(a.e, __fmul_rn(fabsf(v), b.e)), den) : __int_as_float(0x7f800000);
    return FErr{v, __fadd_rn(e, __fmul_rn(kU32, fabsf(v)))};
}
__device__ __forceinline__ FErr fe_sqrt(FErr a) {   // of a non-negative exact value
    const float v = __fsqrt_rn(fmaxf(a.v, 0.0f));
    const float r = __fsqrt_rn(a.e);
    const float e = v > 0.0f ? fminf(__fdiv_rn(a.e, v), r) : r;
    return FErr{v, __fadd_rn(e, __fmul_rn(kU32, v))};
}
__device__ __forceinline__ FErr fe_scale(FErr a, float k) {   // by an exact power of two
    return FErr{a.v * k, a.e * fabsf(k)};
}
__device__ __forceinline__ FErr fe_c(float v) {   // FP32 rounding of an FP64 constant
    return FErr{v, __fmul_rn(kU32, fabsf(v))};
}

// Interval [lo, hi] containing the FP64 signal speed of signal_speed64 (divided by h for variable h). The
// bound covers the FP32 roundings; the factor 1 + 2^-8 covers the FP64 sequence's own roundings (2^-29
// times the FP32 ones, through the same operations) and the roundings of the bound's evaluation.
__device__ __forceinline__ void signal_bounds32(const DevParams &P, int mat, double m, double w, double vx,
                                                double vy, double vz, double E, double h, float &lo, float &hi) {
    if (P.eos[mat] == 0) {
        // Linear EOS: every quantity is non-negative, so relative errors compose. The roundings of m, w
        // and the quotient give rho within 3u, M / rho within 5u (M's rounding), the root within 3.5u; each
        // v component and its square within 3u, the sums within 5u, the root within 3.5u; their sum
        // within 4.5u (u = 2^-24, first order); the quotient by h adds 2u. 2^-20 = 16u covers these, the
        // second-order terms and the FP64 sequence's own roundings, when m, w (and h) are normal positive
        // FP32 numbers; otherwise the interval is unbounded.
        const float mf = __double2float_rn(m), wf = __double2float_rn(w);
        const float fx = __double2float_rn(vx), fy = __double2float_rn(vy), fz = __double2float_rn(vz);
        const float rho = __fdiv_rn(mf, wf);
        const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz));
        float sv = __fadd_rn(__fsqrt_rn(__fdiv_rn(P.f_Mmod[mat], rho)), __fsqrt_rn(v2));
        bool good = mf >= 0x1p-126f && wf >= 0x1p-126f && mf < 0x1p127f && wf < 0x1p127f;
        if (P.variable_h) {
            const float hf = __double2float_rn(h);
            good = good && hf >= 0x1p-126f;
            sv = __fdiv_rn(sv, hf);
        }
        if (good && sv > 0.0f && sv < 0x1p120f) {
            lo = __fmul_rn(sv, 1.0f - 0x1p-20f);
            hi = __fmul_rn(sv, 1.0f + 0x1p-20f);
        } else {
            lo = 0.0f;
            hi = __int_as_float(0x7f800000);
        }
        return;
    }
    const FErr rho = fe_div(fe_in(m), fe_in(w));
    const FErr fx = fe_in(vx), fy = fe_in(vy), fz = fe_in(vz);
    const FErr v2 = fe_add(fe_add(fe_mul(fx, fx), fe_mul(fy, fy)), fe_mul(fz, fz));
    const FErr vn = fe_sqrt(v2);
    FErr s1, s2;
    {
        const FErr rho0 = fe_c(P.f_rho0[mat]), c0 = fe_c(P.f_c0[mat]), g0 = fe_c(P.f_g0[mat]);
        const FErr sm1 = fe_c(P.f_sm1[mat]);
        const FErr one{1.0f, 0.0f};
        const FErr e = fe_sub(fe_in(E), fe_scale(v2, 0.5f));
        const FErr mu = fe_sub(fe_div(rho, rho0), one);
        const FErr k0 = fe_mul(fe_mul(rho0, c0), c0);
        const FErr q = fe_add(one, mu);
        const FErr r2 = fe_scale(rho0, 2.0f);
        const FErr gr = fe_mul(g0, rho0);
        const FErr G43 = fe_c(P.f_G43[mat]);
        // both branches of the reference curve when the sign of mu is not certain
        auto branch = [&](bool comp) {
            FErr pH, dpH;
            if (comp) {
                const FErr D = fe_sub(one, fe_mul(sm1, mu));
                const FErr D2 = fe_mul(D, D);
                pH = fe_div(fe_mul(fe_mul(k0, mu), q), D2);
                const FErr a1 = fe_mul(fe_add(one, fe_scale(mu, 2.0f)), D);
                const FErr a2 = fe_mul(fe_mul(fe_scale(sm1, 2.0f), mu), q);
                dpH = fe_div(fe_mul(k0, fe_add(a1, a2)), fe_mul(D2, D));
            } else {
                pH = fe_mul(k0, mu);
                dpH = k0;
            }
            const FErr eH = fe_div(fe_mul(pH, mu), fe_mul(r2, q));
            const FErr deH = fe_div(fe_add(fe_mul(fe_mul(dpH, mu), q), pH), fe_mul(fe_mul(r2, q), q));
            const FErr p = fe_add(pH, fe_mul(gr, fe_sub(e, eH)));
            FErr cb2 = fe_add(fe_div(fe_sub(dpH, fe_mul(gr, deH)), rho0), fe_div(fe_mul(p, gr), fe_mul(rho, rho)));
            cb2.v = fmaxf(cb2.v, 0.0f);   // the floor at 0 does not widen the bound
            return fe_add(fe_sqrt(fe_add(cb2, fe_div(G43, rho))), vn);
        };
        const bool pos = mu.v > mu.e, neg = mu.v < -mu.e;
        s1 = branch(!neg);
        s2 = (pos || neg) ? s1 : branch(false);
    }
    if (P.variable_h) {
        const FErr hh = fe_in(h);
        s1 = fe_div(s1, hh);
        s2 = fe_div(s2, hh);
    }
    const float k = 1.00390625f;   // 1 + 2^-8
    const float e1 = __fmul_rn(s1.e, k), e2 = __fmul_rn(s2.e, k);
    float l = fminf(__fmul_rn(__fsub_rn(s1.v, e1), 1.0f - 0x1p-20f), __fmul_rn(__fsub_rn(s2.v, e2), 1.0f - 0x1p-20f));
    float u = fmaxf(__fmul_rn(__fadd_rn(s1.v, e1), 1.0f + 0x1p-20f), __fmul_rn(__fadd_rn(s2.v, e2), 1.0f + 0x1p-20f));
    if (!(l > 0.0f)) l = 0.0f;                                       // also NaN
    if (!(u >= l) || isinf(e1) || isinf(e2)) u = __int_as_float(0x7f800000);
    lo = l;
    hi = u;
}

// Words of the time-step reduction (zero between steps). sig: bits of the largest lo (non-negative
// floats order like their bit patterns); sigd: bits of the largest FP64 signal speed of the candidates;
// ccount: candidates listed; done: blocks of the final kernel that finished.
struct DtWords {
    unsigned long long sigd;
    unsigned int sig, ccount, done, eval;
    // bits of a listing threshold from the previous step: 2^-10 below its largest lower end (0: none).
    // Lanes below it are not listed; if this step's largest lower end falls below it, a dropped lane
    // might have mattered, and the final kernel evaluates every particle instead
    unsigned int hint;
    unsigned int last_ccount, last_eval;   // the last completed reduction's counts (statistics)
    // relative width of the threshold (0: 2^-10); doubled after a step whose lower bound fell below
    // the threshold, halved after a step that listed more candidates than half the capacity
    float delta;
};
// A listed candidate: its FP64 inputs, material and the upper end of its interval.
struct __align__(16) DtCand {
    double m, w, vx, vy, vz, E, h;
    unsigned int hi;
    int mat;
};
struct DtArgs {
    DtWords *w;
    DtCand *cand;
    uint32_t cap;     // list capacity; a step that lists more evaluates every particle in FP64 instead
};

// ---------------------------------------------------------------------------------------------
// Programmatic dependent launch: a chain of kernels on one stream whose successors are launched with
// pdl_launch may have a successor's blocks scheduled while its predecessor drains, which hides the
// launch latency between short kernels. Every kernel launched with pdl_launch calls pdl_wait() first,
// in every block and before any access to device memory: it returns once the previous kernel on the
// stream has completed and its writes are visible (at once for a normal launch), so each kernel of the
// chain completes after everything before it. pdl_release() then allows the next kernel's launch.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-collective (all 32 lanes): the candidate filter of one warp. ok: the lane has a particle whose
// signal speed counts; its FP64 inputs and slot.
__device__ __forceinline__ void dt_candidate(const DevParams &P, const DtArgs &d, bool ok, int mat,
                                             double m, double w, double vx, double vy, double vz, double E,
                                             double h) {
    const unsigned full = 0xffffffffu;
    float lo = 0.0f, hi = 0.0f;
    if (ok) signal_bounds32(P, mat, m, w, vx, vy, vz, E, h, lo, hi);
    const unsigned lob = __float_as_uint(lo);
    const unsigned wmax = __reduce_max_sync(full, ok ? lob : 0u);
    const unsigned lead = __ballot_sync(full, ok && lob == wmax);
    if (lead == 0u) return;   // no particle in this warp
    const int lane = threadIdx.x & 31, ld = __ffs(lead) - 1;
    if (lane == ld) atomicMax(&d.w->sig, wmax);
    const unsigned hint = *(volatile unsigned *)&d.w->hint;
    bool cand = ok && __float_as_uint(hi) >= (wmax > hint ? wmax : hint);
    if (__ballot_sync(full, cand) != (1u << ld)) {
    // the leader's FP64 inputs: identical inputs give the identical FP64 value
    const long long lm = __shfl_sync(full, __double_as_longlong(m), ld);
    const long long lw = __shfl_sync(full, __double_as_longlong(w), ld);
    const long long lx = __shfl_sync(full, __double_as_longlong(vx), ld);
    const long long ly = __shfl_sync(full, __double_as_longlong(vy), ld);
    const long long lz = __shfl_sync(full, __double_as_longlong(vz), ld);
    const long long lE = __shfl_sync(full, __double_as_longlong(E), ld);
    const long long lh = __shfl_sync(full, __double_as_longlong(h), ld);
    const int lmat = __shfl_sync(full, mat, ld);
    const bool same = lane != ld && lm == __double_as_longlong(m) && lw == __double_as_longlong(w) &&
                      lx == __double_as_longlong(vx) && ly == __double_as_longlong(vy) &&
                      lz == __double_as_longlong(vz) && lE == __double_as_longlong(E) &&
                      lh == __double_as_longlong(h) && lmat == mat;
    cand = cand && !same;
    }
    const unsigned cm = __ballot_sync(full, cand);
    const int first = __ffs(cm) - 1;
    unsigned base = 0u;
    if (lane == first) base = atomicAdd(&d.w->ccount, (unsigned)__popc(cm));
    base = __shfl_sync(full, base, first);
    if (cand) {
        const unsigned idx = base + (unsigned)__popc(cm & lanemask_lt());
        if (idx < d.cap) {
            DtCand c;
            c.m = m; c.w = w; c.vx = vx; c.vy = vy; c.vz = vz; c.E = E; c.h = h;
            c.hi = __float_as_uint(hi);
            c.mat = mat;
            d.cand[idx] = c;
        }
    }
}

// Pressure (with the cut-off) and sound speed (bulk part from the isentropic derivative of the uncut
// pressure, plus the shear part 4G/3rho) of material mat at density rho and specific internal energy
// e, FP64. Linear EOS: p = K (rho/rho0 - 1), c^2 = (K + 4G/3) / rho.
__device__ __forceinline__ void eos_pc(const DevParams &P, int mat, double rho, double e, double &p, double &c) {
    if (P.eos[mat] == 0) {
        p = P.K[mat] * (rho / P.rho0[mat] - 1.0);
        c = sqrt(P.Mmod[mat] / rho);
    } else {
        // the reference's formulas with three divisions (1/D, 1/(1 + mu), 1/rho); FP64 scarce on GB300
        const double sm1 = P.s_hug[mat] - 1.0, gr = P.gamma0[mat] * P.rho0[mat], k0 = P.k0[mat];
        const double mu = rho * P.inv_rho0[mat] - 1.0;
        const double q = 1.0 + mu, iq = 1.0 / q;
        double pH, dpH;
        if (mu > 0.0) {
            const double D = 1.0 - sm1 * mu, iD = 1.0 / D;
            pH = k0 * mu * q * iD * iD;
            dpH = k0 * ((1.0 + 2.0 * mu) * D + 2.0 * sm1 * mu * q) * iD * iD * iD;
        } else {
            pH = k0 * mu;
            dpH = k0;
        }
        const double eH = pH * mu * iq * P.inv_2rho0[mat];
        const double deH = (dpH * mu * q + pH) * iq * iq * P.inv_2rho0[mat];
        p = pH + gr * (e - eH);
        const double irho = 1.0 / rho;
        double cb2 = (dpH - gr * deH) * P.inv_rho0[mat] + p * gr * irho * irho;
        if (!(cb2 > 0.0)) cb2 = 0.0;
        c = sqrt(cb2 + 4.0 * P.G[mat] / 3.0 * irho);
    }
    if (p < P.p_min[mat]) p = P.p_min[mat];
}

// Split-path interaction record of a state, the position part aside: FP32 velocity and density, the
// diagonal of the full stress sigma = -p I + S (S traceless in FP32: S_zz = -(S_xx + S_yy)), impedance
// and energy; linear EOS, p = K (rho/rho0 - 1) = K (m - rho0 w) / (rho0 w) with the cancelling difference
// in FP64. Every operation is an explicitly rounded intrinsic, so the reorder (from the gathered FP64
// state) and the integration (from the new state it has just formed) produce the same bits.
__device__ __forceinline__ RecF record_split_linear(const DevParams &P, int mat, double w, double m, double vx,
                                                    double vy, double vz, double E, double sxx, double syy,
                                                    double sxy, double sxz, double syz) {
    const float rho = __fdiv_rn(__double2float_rn(m), __double2float_rn(w));
    const double rw = __dmul_rn(P.rho0[mat], w);
    float pf = __fdiv_rn(__fmul_rn(P.f_K[mat], __double2float_rn(__dsub_rn(m, rw))), __double2float_rn(rw));
    const float pmin = __double2float_rn(P.p_min[mat]);
    if (pf < pmin) pf = pmin;
    const float Zf = __fmul_rn(rho, __fsqrt_rn(__fdiv_rn(P.f_Mmod[mat], rho)));
    const float fxx = __double2float_rn(sxx), fyy = __double2float_rn(syy), fzz = -__fadd_rn(fxx, fyy);
    RecF r;
    r.a = make_float4(__double2float_rn(vx), __double2float_rn(vy), __double2float_rn(vz), rho);
    r.b = make_float4(__fsub_rn(fzz, pf), Zf, __double2float_rn(E), __fsub_rn(fxx, pf));
    r.c = make_float4(__fsub_rn(fyy, pf), __double2float_rn(sxy), __double2float_rn(sxz), __double2float_rn(syz));
    return r;
}

}  // namespace gsph
