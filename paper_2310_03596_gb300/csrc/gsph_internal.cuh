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
    float f_rho0[kMaxMat], f_K[kMaxMat], f_G[kMaxMat], f_Mmod[kMaxMat];
    // equation of state per material (0 linear, 1 Mie-Gruneisen) and pressure cut-off
    int eos[kMaxMat];
    double c0[kMaxMat], s_hug[kMaxMat], gamma0[kMaxMat], p_min[kMaxMat];
    double inv_rho0[kMaxMat], k0[kMaxMat], inv_2rho0[kMaxMat];   // 1/rho0, rho0 c0^2, 1/(2 rho0)
    // FP32 roundings for the signal speed: c0, s - 1, gamma0, 4G/3
    float f_c0[kMaxMat], f_sm1[kMaxMat], f_g0[kMaxMat], f_G43[kMaxMat];
    // variable smoothing lengths: support r^2 < (h_i + h_j)^2; the FP32 list test decides outside the
    // relative band [1 - d, 1 + d] around it (d = kVarBand, wide enough for size ratios up to 4)
    int variable_h;
    float f_vlo, f_vhi;      // 1 - d, 1 + d
    float f_k5;              // |dW/dr| = k5 (1 / (h_i + h_j))^5 r (1 - r / (h_i + h_j))^3: 210 / pi
    double k5;
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

// bucket_coord without the FP64 division in the common case. The FP32 quotient tf of the FP32 rounding
// of d = x - lo by the FP32 reciprocal carries three FP32 roundings, so it lies within 3.01 * 2^-24 |t|
// of the exact d / cell, and the correctly rounded FP64 quotient t within another 2^-53 |t|. When tf
// is farther than 2^-22 (|tf| + 1) from every integer, t lies strictly between the same two integers
// and floor(tf) = floor(t). Otherwise (near a bucket face, NaN, infinities, differences beyond the
// FP32 range or below its normal range, a reciprocal that is not a normal FP32 number - passed as NaN)
// the FP64 division decides.
__device__ __forceinline__ int bucket_coord_fast(double x, double lo, double cell, float inv_cell, int dim) {
    const double d = __dsub_rn(x, lo);
    const float df = __double2float_rn(d);
    const float tf = __fmul_rn(df, inv_cell);
    const float fl = floorf(tf);
    const float fr = __fsub_rn(tf, fl);   // exact
    const float eps = __fmul_rn(0x1p-22f, __fadd_rn(fabsf(tf), 1.0f));
    if (fr > eps && fr < __fsub_rn(1.0f, eps) && fabsf(df) >= 0x1p-126f) {
        if (fl < 0.0f) return -1;
        if (fl >= (float)dim) return dim;
        return (int)fl;
    }
    return bucket_coord(x, lo, cell, dim);
}

__device__ __forceinline__ int bucket_coord_signed(double x, double lo, double cell) {
    return (int)floor(__ddiv_rn(__dsub_rn(x, lo), cell));
}

__device__ __forceinline__ uint32_t hash_of(const DevParams &P, double x, double y, double z) {
    int cx = bucket_coord_fast(x, P.lo[0], P.cell, P.f_inv_cell, P.dims[0]);
    int cy = bucket_coord_fast(y, P.lo[1], P.cell, P.f_inv_cell, P.dims[1]);
    int cz = bucket_coord_fast(z, P.lo[2], P.cell, P.f_inv_cell, P.dims[2]);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= P.dims[0] || cy >= P.dims[1] || cz >= P.dims[2]) return P.ncell;
    return (uint32_t)cx + (uint32_t)P.dims[0] * ((uint32_t)cy + (uint32_t)P.dims[1] * (uint32_t)cz);
}

__device__ __forceinline__ void decode_cell(const DevParams &P, uint32_t c, int &cx, int &cy, int &cz) {
    cx = (int)(c % (uint32_t)P.dims[0]);
    uint32_t r = c / (uint32_t)P.dims[0];
    cy = (int)(r % (uint32_t)P.dims[1]);
    cz = (int)(r / (uint32_t)P.dims[1]);
}

// CFL signal speed c + |v| of one particle, evaluated in FP32 with correctly rounded operations on
// the FP32 roundings of m, w, v (the max over particles is order independent, so the time step is
// reproducible bit for bit on any IEEE machine evaluating the same sequence).
__device__ __forceinline__ float signal_speed32(const DevParams &P, int mat, double m, double w,
                                                double vx, double vy, double vz, double E) {
    const float rho = __fdiv_rn((float)m, (float)w);
    const float fx = (float)vx, fy = (float)vy, fz = (float)vz;
    const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz));
    float c;
    if (P.eos[mat] == 0) {
        c = __fsqrt_rn(__fdiv_rn(P.f_Mmod[mat], rho));
    } else {
        // Mie-Gruneisen sound speed: the same FP32 sequence as the host reference, each operation
        // correctly rounded (no contraction)
        const float rho0 = P.f_rho0[mat], c0 = P.f_c0[mat], sm1 = P.f_sm1[mat], g0 = P.f_g0[mat];
        const float e = __fsub_rn((float)E, __fmul_rn(0.5f, v2));
        const float mu = __fsub_rn(__fdiv_rn(rho, rho0), 1.0f);
        const float k0 = __fmul_rn(__fmul_rn(rho0, c0), c0);
        float pH, dpH;
        if (mu > 0.0f) {
            const float D = __fsub_rn(1.0f, __fmul_rn(sm1, mu));
            const float D2 = __fmul_rn(D, D);
            const float q = __fadd_rn(1.0f, mu);
            pH = __fdiv_rn(__fmul_rn(__fmul_rn(k0, mu), q), D2);
            const float t1 = __fmul_rn(__fadd_rn(1.0f, __fmul_rn(2.0f, mu)), D);
            const float t2 = __fmul_rn(__fmul_rn(2.0f, sm1), __fmul_rn(mu, q));
            dpH = __fdiv_rn(__fmul_rn(k0, __fadd_rn(t1, t2)), __fmul_rn(D2, D));
        } else {
            pH = __fmul_rn(k0, mu);
            dpH = k0;
        }
        const float q = __fadd_rn(1.0f, mu);
        const float r2q = __fmul_rn(__fmul_rn(2.0f, rho0), q);
        const float eH = __fdiv_rn(__fmul_rn(pH, mu), r2q);
        const float deH = __fdiv_rn(__fadd_rn(__fmul_rn(__fmul_rn(dpH, mu), q), pH), __fmul_rn(r2q, q));
        const float gr = __fmul_rn(g0, rho0);
        const float p = __fadd_rn(pH, __fmul_rn(gr, __fsub_rn(e, eH)));
        float cb2 = __fadd_rn(__fdiv_rn(__fsub_rn(dpH, __fmul_rn(gr, deH)), rho0),
                              __fdiv_rn(__fmul_rn(p, gr), __fmul_rn(rho, rho)));
        if (!(cb2 > 0.0f)) cb2 = 0.0f;
        c = __fsqrt_rn(__fadd_rn(cb2, __fdiv_rn(P.f_G43[mat], rho)));
    }
    return __fadd_rn(c, __fsqrt_rn(v2));
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

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace gsph
