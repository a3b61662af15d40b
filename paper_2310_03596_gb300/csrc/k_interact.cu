// k_interact.cu - the interaction loop (Sec. II step f) fused with the integration (step g), as two
// kernels.
//
// k_nbr_list: one lane per sorted particle i; a warp holds 32 consecutive particles of the hash order,
//   which share most of their 27-bucket neighbourhoods. The neighbourhood is visited as 9 rows of 3
//   buckets that are contiguous in hash order. The warp streams the union of its lanes' candidate
//   ranges through shared memory in batches of 32 (four planes x, y, z, |c|^2 in a frame common to the
//   group), every lane tests the staged candidates two at a time with packed FP32 operations into a
//   32-bit hit mask, and appends one entry per batch with any hit to a column-major list in global
//   memory (entry = hit mask, batch base slot | row offset). Light on registers, so the candidate
//   stream runs at full occupancy; no per-neighbour bookkeeping.
// k_pair: one lane per particle walks its entries in order and the set bits of each from the highest
//   (the next neighbour's record requested while the current pair is evaluated, no branch around the
//   pair): pair fluxes, per-particle sums, then the wall images (mirror planes, searched around the
//   mirrored point; only particles near a wall find any), then the integration. A particle with more
//   neighbours than the list holds finishes the rest by re-scanning its buckets in the same order, so
//   results never depend on the list capacity.
//
// Pair formulation (reading of the Gamma-SPH-ALE interface state; the paper cites it from another
// work): transport velocity v0 = v; acoustic Riemann problem on the pair normal n (L = lower sorted
// slot, n from L to R); interface velocity v_E = mean v + (u* - mean u) n, density and energy means,
// traction t* n plus the averaged tangential traction; Wendland C2 gradient |dW/dr| n.
//
// MUSCL reconstruction (reconstruction = 1, reading of the second-order SPH-ALE variant): a gradient
//   pass (k_pair<PM_GRAD>) sums the SPH gradients of v and sigma = -p I + S over the same lists and
//   images into a gradient record per particle; the flux pass (k_pair<PM_MUSCL>) reconstructs v and
//   sigma of both ends at the pair midpoint, each component limited by minmod against the centred
//   difference, for the Riemann problem, with the particle velocities as transport velocities. Both
//   ends form the same reconstructed pair from the raw difference (odd in it), so the fluxes stay
//   bitwise antisymmetric. The stress rate takes L from the gradient record.
//
// Variable smoothing lengths (VARH, variable_h = 1): the list test and every pair term take the pair's
//   own support and kernel, r^2 < (h_i + h_j)^2 and |dW/dr| of h_ij = (h_i + h_j) / 2, from the sorted
//   lengths (FP64 and their FP32 roundings); the FP32 list test decides outside a relative band of
//   1e-3 around (h_i + h_j)^2, the FP64 positions and lengths inside it.
//
// Split path: pair math in FP32 from FP32 records (positions relative to each particle's bucket corner,
// so differences keep ~2^-24 * 2h; the stress diagonal stored as sigma = -p I + S), FP32 sums with
// Kahan compensation for the conserved quantities (volume, mass, momentum, energy) and plain FP32 sums
// for the velocity gradient; the FP64 state advances by increments of v, E and S formed in FP32 and
// added once, w, m and x in FP64. The support predicate stays exact: the FP32 r^2 decides only outside
// a band of relative width 3e-5 around (2h)^2, inside which the FP64 positions decide with the same
// rounding as FP64 code.
#include <type_traits>

#include "gsph_internal.cuh"

namespace gsph {

constexpr int NL_THREADS = 256;            // neighbour-list kernel
constexpr int PK_THREADS = 128;            // pair kernel
constexpr uint32_t IT_JMASK = (1u << 26) - 1;   // list entry .y: batch base slot (26 bits) | row offset (4 bits)

// interaction inputs of one particle; txx, tyy, tzz are the diagonal of the full stress sigma = -p I + S
template <class R> struct PIn { R vx, vy, vz, rho, Z, E, txx, tyy, tzz, sxy, sxz, syz, w; };

// split record: (vx, vy, vz, rho), (sigma_zz, Z, E, sigma_xx), (sigma_yy, S_xy, S_xz, S_yz)
__device__ __forceinline__ PIn<float> unpack(const RecF &r, float w) {
    PIn<float> q;
    q.vx = r.a.x; q.vy = r.a.y; q.vz = r.a.z; q.rho = r.a.w;
    q.tzz = r.b.x; q.Z = r.b.y; q.E = r.b.z; q.txx = r.b.w;
    q.tyy = r.c.x; q.sxy = r.c.y; q.sxz = r.c.z; q.syz = r.c.w;
    q.w = w;
    return q;
}
// FP64 record: (vx, vy, vz, rho), (p, Z, E, S_xx), (S_yy, S_zz, S_xy, S_xz), (S_yz, -, -, -)
__device__ __forceinline__ PIn<double> unpack(const RecD &r, double w) {
    PIn<double> q;
    q.vx = r.a.x; q.vy = r.a.y; q.vz = r.a.z; q.rho = r.a.w;
    q.Z = r.b.y; q.E = r.b.z;
    q.txx = r.b.w - r.b.x; q.tyy = r.c.x - r.b.x; q.tzz = r.c.y - r.b.x;
    q.sxy = r.c.z; q.sxz = r.c.w; q.syz = r.d.x;
    q.w = w;
    return q;
}

__device__ __forceinline__ PIn<float> load_rec(const RecF *__restrict__ rec, float w, int64_t j) {
    RecF r;
    r.a = __ldg(&rec[j].a);
    r.b = __ldg(&rec[j].b);
    r.c = __ldg(&rec[j].c);
    return unpack(r, w);
}
__device__ __forceinline__ PIn<double> load_rec(const RecD *__restrict__ rec, double w, int64_t j) {
    RecD r;
    r.a = rec[j].a; r.b = rec[j].b; r.c = rec[j].c; r.d = rec[j].d;
    return unpack(r, w);
}

// Mirror image of a state in the plane normal to `ax`.
template <class R> __device__ __forceinline__ void mirror(PIn<R> &q, int ax) {
    if (ax == 0) { q.vx = -q.vx; q.sxy = -q.sxy; q.sxz = -q.sxz; }
    else if (ax == 1) { q.vy = -q.vy; q.sxy = -q.sxy; q.syz = -q.syz; }
    else { q.vz = -q.vz; q.sxz = -q.sxz; q.syz = -q.syz; }
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rcp_r(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// flux factors: the pair's mass, momentum and energy fluxes are w2a Xm, w2a Xv and (w2a / 2) Xe
template <class R> struct PairRes { R Xm, Xv[3], Xe, a, n[3], du_vol, w2a; };

// Pair fluxes on the canonical pair: e = x_j - x_i as seen from this end (the canonical difference
// x_R - x_L, L the lower sorted slot, is sgn e), `me` the particle being updated and `oth` its
// neighbour, sgn = +1 when me is L, -1 when me is R. Every per-particle
// projection is taken on the same canonical normal at both ends of the pair, every symmetric
// combination uses commutative operations (the two Riemann sums of products are rounded product by
// product, never fused), and the two antisymmetric differences are oriented by the exact factor sgn,
// so the two ends produce bitwise-opposite fluxes.
// CLAMP: the pair may lie beyond the support (second Heun stage over the step-start lists), where the
// kernel gradient is 0.
// RECON: me and oth are the reconstructed interface states and me0, oth0 the particles' own, whose
// velocities are the transport velocities (mass flux and volume rate); otherwise me0, oth0 are unused.
template <class R, bool CLAMP = false, bool RECON = false>
__device__ __forceinline__ void pair_terms(R e0, R e1, R e2, const PIn<R> &me, const PIn<R> &oth, R sgn, R inv_2h,
                                           R kdwh, PairRes<R> &o, const PIn<R> &me0, const PIn<R> &oth0) {
    const R half = R(0.5);
    const R r2 = e0 * e0 + e1 * e1 + e2 * e2;
    const R inv_r = rsqrt_r(r2);
    const R r = r2 * inv_r;
    const R sir = sgn * inv_r;   // the canonical normal n = sgn e / r
    const R n0 = e0 * sir, n1 = e1 * sir, n2 = e2 * sir;
    // |dW/dr| = kdw q (1 - q/2)^3 with q = r / h, as (kdw / h) r (1 - r / 2h)^3
    R sq = R(1) - inv_2h * r;
    if (CLAMP) sq = sq > R(0) ? sq : R(0);
    const R a = kdwh * r * sq * sq * sq;
    // normal velocity, traction sigma n and normal traction of each particle
    const R um = me.vx * n0 + me.vy * n1 + me.vz * n2;
    const R uo = oth.vx * n0 + oth.vy * n1 + oth.vz * n2;
    const R sm0 = me.txx * n0 + me.sxy * n1 + me.sxz * n2;
    const R sm1 = me.sxy * n0 + me.tyy * n1 + me.syz * n2;
    const R sm2 = me.sxz * n0 + me.syz * n1 + me.tzz * n2;
    const R so0 = oth.txx * n0 + oth.sxy * n1 + oth.sxz * n2;
    const R so1 = oth.sxy * n0 + oth.tyy * n1 + oth.syz * n2;
    const R so2 = oth.sxz * n0 + oth.syz * n1 + oth.tzz * n2;
    const R tmn = sm0 * n0 + sm1 * n1 + sm2 * n2;
    const R ton = so0 * n0 + so1 * n1 + so2 * n2;
    // acoustic Riemann problem, left = L, right = R:
    //   u* = (ZL uL + ZR uR + (tR - tL)) / (ZL + ZR),  t* = (ZR tL + ZL tR + ZL ZR (uR - uL)) / (ZL + ZR)
    const R izs = rcp_r(me.Z + oth.Z);
    const R dRL_t = sgn * (ton - tmn);   // tR - tL
    const R dRL_u = sgn * (uo - um);     // uR - uL
    // u* - (uL + uR)/2 = ((ZR - ZL)(uR - uL)/2 + (tR - tL)) / (ZL + ZR): the product of the two
    // differences is the same at both ends, and the correction is exactly 0 between equal states
    const R dus = (half * (oth.Z - me.Z) * (uo - um) + dRL_t) * izs;
    const R ts = (add_rn(mul_rn(oth.Z, tmn), mul_rn(me.Z, ton)) + (me.Z * oth.Z) * dRL_u) * izs;
    // transport velocities of the particles (the interface states' own unless reconstructed)
    R um0 = um, uo0 = uo;
    if (RECON) {
        um0 = me0.vx * n0 + me0.vy * n1 + me0.vz * n2;
        uo0 = oth0.vx * n0 + oth0.vy * n1 + oth0.vz * n2;
    }
    // (v_E - v0_LR) . n, the mass flux's velocity
    const R du = RECON ? dus + half * ((um + uo) - (um0 + uo0)) : dus;
    // interface velocity and traction at twice their value (binary scalings, exact): V = 2 v_E =
    // (v_i + v_j) + 2 du n, T = 2 sigma_E n = 2 t* n + (sigma_i n + sigma_j n) - (t_i + t_j) n
    const R du2 = dus + dus, ts2 = ts + ts, tm2 = tmn + ton;
    const R V0 = (me.vx + oth.vx) + du2 * n0;
    const R V1 = (me.vy + oth.vy) + du2 * n1;
    const R V2 = (me.vz + oth.vz) + du2 * n2;
    const R T0 = ts2 * n0 + ((sm0 + so0) - tm2 * n0);
    const R T1 = ts2 * n1 + ((sm1 + so1) - tm2 * n1);
    const R T2 = ts2 * n2 + ((sm2 + so2) - tm2 * n2);
    // with w2a = w_i w_j a and the mass flux mf = rho_E du (mf2 = 2 mf):
    //   2 w_i w_j a (mf v_E - sigma_E n) = w2a (mf V - T),
    //   2 w_i w_j a (mf E_E - sigma_E n . v_E) = (w2a / 2) (mf2 (E_i + E_j) - T . V)
    const R w2a = me.w * oth.w * a;
    const R mf2 = (me.rho + oth.rho) * du;
    const R mf = half * mf2;
    o.Xm = mf2;
    o.Xv[0] = mf * V0 - T0;
    o.Xv[1] = mf * V1 - T1;
    o.Xv[2] = mf * V2 - T2;
    o.Xe = mf2 * (me.E + oth.E) - (T0 * V0 + T1 * V1 + T2 * V2);
    o.a = a;
    o.n[0] = n0; o.n[1] = n1; o.n[2] = n2;
    o.du_vol = RECON ? sgn * (uo0 - um0) : dRL_u;
    o.w2a = w2a;
}

// ---- MUSCL pieces. Gradient record order: the 9 fields vx vy vz, sigma xx yy zz xy xz yz, each as
// d/dx, d/dy, d/dz (27 values, padded to 28).
constexpr int kNGrad = 27;
template <class R> __device__ __forceinline__ R pin_field(const PIn<R> &q, int f) {
    return f == 0 ? q.vx : f == 1 ? q.vy : f == 2 ? q.vz : f == 3 ? q.txx : f == 4 ? q.tyy : f == 5 ? q.tzz
         : f == 6 ? q.sxy : f == 7 ? q.sxz : q.syz;
}
template <class R> __device__ __forceinline__ void set_field(PIn<R> &q, int f, R v) {
    if (f == 0) q.vx = v; else if (f == 1) q.vy = v; else if (f == 2) q.vz = v;
    else if (f == 3) q.txx = v; else if (f == 4) q.tyy = v; else if (f == 5) q.tzz = v;
    else if (f == 6) q.sxy = v; else if (f == 7) q.sxz = v; else q.syz = v;
}
// minmod, odd in its arguments: minmod(-a, -b) = -minmod(a, b)
template <class R> __device__ __forceinline__ R minmod(R a, R b) {
    const R aa = a < R(0) ? -a : a, ab = b < R(0) ? -b : b;
    return a * b > R(0) ? (aa < ab ? a : b) : R(0);
}
// gradient of the mirror image in wall axis ax: each index along the axis (the field's and the
// derivative's) flips the sign
template <class R> __device__ __forceinline__ void mirror_grad(R *G, int ax) {
#pragma unroll
    for (int f = 0; f < 9; ++f) {
        const int i0 = f < 3 ? f : (f < 6 ? f - 3 : (f == 6 ? 0 : (f == 7 ? 0 : 1)));
        const int i1 = f < 3 ? -1 : (f < 6 ? f - 3 : (f == 6 ? 1 : 2));
        const int own = (i0 == ax) + (i1 == ax);
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if ((own + (b == ax)) & 1) G[3 * f + b] = -G[3 * f + b];
    }
}
// interface states of the pair from the raw difference e = x_oth - x_me (this end's)
template <class R>
__device__ __forceinline__ void reconstruct(const PIn<R> &me, const R *Gm, const PIn<R> &oth, const R *Go, R e0, R e1,
                                            R e2, PIn<R> &mes, PIn<R> &oths) {
    mes = me;
    oths = oth;
#pragma unroll
    for (int f = 0; f < 9; ++f) {
        const R vm = pin_field(me, f), vo = pin_field(oth, f), d = vo - vm;
        const R sm = Gm[3 * f] * e0 + Gm[3 * f + 1] * e1 + Gm[3 * f + 2] * e2;
        const R so = Go[3 * f] * e0 + Go[3 * f + 1] * e1 + Go[3 * f + 2] * e2;
        set_field(mes, f, vm + R(0.5) * minmod(sm, d));
        set_field(oths, f, vo - R(0.5) * minmod(so, d));
    }
}

// Per-particle sums. FP32: compensated for the conserved quantities (fields 0-5: volume, mass,
// momentum, energy) in blocks - the terms of a block of 8 pairs are summed plainly into p, and fold()
// adds the block sum to s with Kahan compensation c -, plain for the velocity gradient (fields 6-14,
// which only feed the stress rate). FP64: plain.
template <class R> struct Acc;
template <> struct Acc<float> {
    float s[kNRate], c[6], p[6];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) s[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) { c[k] = 0.f; p[k] = 0.f; }
    }
    __device__ __forceinline__ void add(int k, float x) {
        if (k < 6) p[k] += x;
        else s[k] += x;
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float y = p[k] - c[k];
            const float t = s[k] + y;
            c[k] = (t - s[k]) - y;
            s[k] = t;
            p[k] = 0.f;
        }
    }
    // parked sums of the two-pass order (after fold): field f of halo index h at b[f * n + h]
    __device__ __forceinline__ void store(float *b, int64_t n, int64_t h) const {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) b[k * n + h] = s[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) b[(kNRate + k) * n + h] = c[k];
    }
    __device__ __forceinline__ void load(const float *b, int64_t n, int64_t h) {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) s[k] = b[k * n + h];
#pragma unroll
        for (int k = 0; k < 6; ++k) { c[k] = b[(kNRate + k) * n + h]; p[k] = 0.f; }
    }
    // the compensated sum s - c rounded once to FP32 keeps the compensation's benefit (one rounding
    // of the final value instead of one per term) and widens with a single conversion
    __device__ __forceinline__ double get(int k) const { return (double)(k < 6 ? s[k] - c[k] : s[k]); }
    __device__ __forceinline__ float getr(int k) const { return k < 6 ? s[k] - c[k] : s[k]; }
};
template <> struct Acc<double> {
    double s[kNRate];
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ void store(double *b, int64_t n, int64_t h) const {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) b[k * n + h] = s[k];
    }
    __device__ __forceinline__ void load(const double *b, int64_t n, int64_t h) {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) s[k] = b[k * n + h];
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) s[k] = 0.0;
    }
    __device__ __forceinline__ void add(int k, double x) { s[k] += x; }
    __device__ __forceinline__ double get(int k) const { return s[k]; }
    __device__ __forceinline__ double getr(int k) const { return s[k]; }
};

// Adds one pair to the sums of particle i. sg = -1 when i is the left state (n points from i to j),
// +1 when i is the right state; oth = the other particle's state.
template <class R, bool WITH_L = true>
__device__ __forceinline__ void accumulate(Acc<R> &acc, const PairRes<R> &o, R sg, const PIn<R> &me,
                                           const PIn<R> &oth) {
    // sg (w2a X) = (sg w2a) X exactly: the fluxes' scale and orientation in one factor
    const R sgw = sg * o.w2a;
    acc.add(0, o.w2a * o.du_vol);
    acc.add(1, sgw * o.Xm);
    acc.add(2, sgw * o.Xv[0]);
    acc.add(3, sgw * o.Xv[1]);
    acc.add(4, sgw * o.Xv[2]);
    acc.add(5, (R(0.5) * sgw) * o.Xe);
    if (!WITH_L) return;
    // L_i += w_j (v_j - v_i) (x) a n_ij, n_ij = -sg n
    R an = -sg * o.a * oth.w;
    R g0 = an * o.n[0], g1 = an * o.n[1], g2 = an * o.n[2];
    R dv0 = oth.vx - me.vx, dv1 = oth.vy - me.vy, dv2 = oth.vz - me.vz;
    acc.add(6, dv0 * g0); acc.add(7, dv0 * g1); acc.add(8, dv0 * g2);
    acc.add(9, dv1 * g0); acc.add(10, dv1 * g1); acc.add(11, dv1 * g2);
    acc.add(12, dv2 * g0); acc.add(13, dv2 * g1); acc.add(14, dv2 * g2);
}

template <bool SPLIT>
struct Types {
    using R = typename std::conditional<SPLIT, float, double>::type;
    using Pos = typename std::conditional<SPLIT, float4, D4>::type;
    using Rec = typename std::conditional<SPLIT, RecF, RecD>::type;
    using G4 = typename std::conditional<SPLIT, float4, D4>::type;   // 7 per particle: the gradient record
};

// Row window of one search centre: the particles of buckets (bx-1 .. bx+1, Yc, Zc), which are
// contiguous in hash order. rs = 0xffffffff, re = 0 when empty.
__device__ __forceinline__ void row_window(const DevParams &P, const uint2 *__restrict__ cellr, int bx, int Yc, int Zc,
                                           uint32_t &rs, uint32_t &re) {
    rs = 0xffffffffu;
    re = 0u;
    if (Yc < 0 || Yc >= P.dims[1] || Zc < 0 || Zc >= P.dims[2] || bx < -1 || bx > P.dims[0]) return;
    const uint32_t rb = (uint32_t)P.dims[0] * ((uint32_t)Yc + (uint32_t)P.dims[1] * (uint32_t)Zc);
    uint2 cm = make_uint2(0, 0), c0 = make_uint2(0, 0), cp = make_uint2(0, 0);
    if (bx - 1 >= 0 && bx - 1 < P.dims[0]) cm = __ldg(&cellr[rb + bx - 1]);
    if (bx >= 0 && bx < P.dims[0]) c0 = __ldg(&cellr[rb + bx]);
    if (bx + 1 >= 0 && bx + 1 < P.dims[0]) cp = __ldg(&cellr[rb + bx + 1]);
    const bool em = cm.y > cm.x, e0 = c0.y > c0.x, ep = cp.y > cp.x;
    if (em || e0 || ep) {
        rs = em ? cm.x : (e0 ? c0.x : cp.x);
        re = ep ? cp.y : (e0 ? c0.y : cm.y);
    }
}

// Exact support predicate from the FP64 positions (real neighbour, or image in wall `wax` at `wpos`).
__device__ __forceinline__ bool support_exact(const DevParams &P, const double *__restrict__ xs,
                                              const double *__restrict__ ys, const double *__restrict__ zs,
                                              uint32_t j, double X, double Y, double Z, int wax, double wpos,
                                              double R2) {
    double qx = xs[j], qy = ys[j], qz = zs[j];
    const double two_w = __dmul_rn(2.0, wpos);
    if (wax == 0) qx = __dsub_rn(two_w, qx);
    if (wax == 1) qy = __dsub_rn(two_w, qy);
    if (wax == 2) qz = __dsub_rn(two_w, qz);
    return dist2_rn(__dsub_rn(qx, X), __dsub_rn(qy, Y), __dsub_rn(qz, Z)) < R2;
}
// support of a pair: (2h)^2, or (h_i + h_j)^2 with per-particle lengths, each operation rounded
__device__ __forceinline__ double pair_R2(bool varh, const DevParams &P, double hi, double hj) {
    if (!varh) return P.R2;
    const double sij = __dadd_rn(hi, hj);
    return __dmul_rn(sij, sij);
}

// ---------------------------------------------------------------------------------------------
// Neighbour list (real neighbours). list[k * n + i], k < kmax: (mask, base | (dcy + 1) << 26 | (dcz + 1) << 28),
// the neighbours being slots base + t for the set bits t of mask, in ascending (row, slot) order;
// cnt[i] = min(entries found, 255) | (neighbours in the stored entries) << 8. Entries found beyond kmax
// are not stored: the pair kernel finds those neighbours by re-scanning. Both precisions build their
// lists here, from the FP32 positions relative to each particle's bucket corner (the split record's, or
// a copy the FP64 path's reorder writes): the decision is the exact FP64 predicate either way.
// ---------------------------------------------------------------------------------------------
template <bool VARH>
__global__ void __launch_bounds__(NL_THREADS, 4) k_nbr_list(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                                                         const uint2 *__restrict__ cellr,
                                                         const float4 *__restrict__ pos,
                                                         const float *__restrict__ cxs, const double *__restrict__ xs,
                                                         const double *__restrict__ ys, const double *__restrict__ zs,
                                                         int kmax, uint2 *__restrict__ list,
                                                         uint32_t *__restrict__ cnt_out, const double *__restrict__ hs,
                                                         const float *__restrict__ hsf,
                                                         unsigned long long *__restrict__ cost_clear) {
    pdl_wait();      // a programmatic dependent launch (its predecessor's writes are visible from here)
    pdl_release();
    // the step's per-label pair counters, which the pair kernel fills, cleared here rather than by a
    // separate clearing before the pair kernel
    if (cost_clear && blockIdx.x == 0 && threadIdx.x < kMaxLabel) cost_clear[threadIdx.x] = 0ull;
    // staged candidate (c, |c|^2) with c = (x in the group frame, y, z in the row frame), as four planes
    // (x, y, z, |c|^2) of NL_THREADS floats, so that one 16-byte load gives a coordinate of four candidates
    // and the tests run on packed pairs (variable h: a fifth plane of FP32 lengths)
    __shared__ __align__(16) float splane[NL_THREADS * (VARH ? 5 : 4)];
    const int tid = threadIdx.x, lane = tid & 31, wbase = tid & ~31;
    const int64_t s = (int64_t)blockIdx.x * NL_THREADS + tid;
    const bool valid = s < n;
    const uint32_t key = valid ? skey[s] : P.ncell;
    const bool active = valid && key < P.ncell;
    int cx = 0, cy = 0, cz = 0;
    if (active) decode_cell(P, key, cx, cy, cz);
    float ox = 0.f, oy = 0.f, oz = 0.f;
    if (active) {
        const float4 p = pos[s];
        ox = p.x; oy = p.y; oz = p.z;
    }
    const float fcell = P.f_cell, hcell = 0.5f * P.f_cell;
    const uint32_t self = (uint32_t)s;
    // variable h: the own length (FP32 for the fast test, FP64 for the exact one); 0 when unused
    const float hif = VARH && active ? hsf[s] : 0.0f;
    const double hid = VARH && active ? hs[s] : 0.0;
    uint32_t cnt = 0, nlisted = 0;
    uint2 *out = list + (size_t)s;             // next free list entry of this particle (column-major)
    const size_t colstep = (size_t)n;
    bool need = active;
    while (true) {
        const unsigned todo = __ballot_sync(kFullMask, need);
        if (!todo) break;
        const int leader = __ffs(todo) - 1;
        const int gby = __shfl_sync(kFullMask, cy, leader), gbz = __shfl_sync(kFullMask, cz, leader);
        const int gbx = __shfl_sync(kFullMask, cx, leader);
        // a group shares the bucket row: its buckets are the leader's and the next two in x (the leader
        // has the lowest x bucket of its row among the remaining lanes), and the group frame has its x
        // origin 1.5 buckets above the leader's bucket corner, so |x| < 5h for own positions and window
        // candidates
        const bool ing = need && cy == gby && cz == gbz && (unsigned)(cx - gbx) <= 2u;
        const float oxg = fmaf((float)(cx - gbx) - 1.5f, fcell, ox);   // own x in the group frame
        const float gx15 = (float)gbx + 1.5f;   // exact: candidate x in the group frame is (cx_j - gx15) 2h + x
        for (int row = 0; row < 9; ++row) {
            const int dcy = row % 3 - 1, dcz = row / 3 - 1;
            const int Yc = gby + dcy, Zc = gbz + dcz;
            if (Yc < 0 || Yc >= P.dims[1] || Zc < 0 || Zc >= P.dims[2]) continue;
            uint32_t rs = 0xffffffffu, re = 0u;
            if (ing) row_window(P, cellr, cx, Yc, Zc, rs, re);
            const uint32_t lo = __reduce_min_sync(kFullMask, rs);
            const uint32_t hi = __reduce_max_sync(kFullMask, re);
            // own y, z in the row frame (origin at the centre of the row's buckets in y and z); the test
            // below evaluates |c - o|^2 - R2lo as |c|^2 + (|o|^2 - R2lo) - 2 c.o
            const float oyr = fmaf(-(float)dcy - 0.5f, fcell, oy), ozr = fmaf(-(float)dcz - 0.5f, fcell, oz);
            // variable h: |c - o|^2 - (1 - d)(h_i + h_j)^2 = (|c|^2 - (1 - d) h_j^2) + mh h_j + Kr with
            // Kr = |o|^2 - (1 - d) h_i^2 and mh = -2 (1 - d) h_i
            const float Kr = fmaf(oxg, oxg, fmaf(oyr, oyr, fmaf(ozr, ozr, VARH ? -P.f_vlo * hif * hif : -P.f_R2lo)));
            const float mh = -2.0f * P.f_vlo * hif;
            const float mx = -2.0f * oxg, my = -2.0f * oyr, mz = -2.0f * ozr;
            const uint32_t code_yz = (uint32_t)(dcy + 1) << 26 | (uint32_t)(dcz + 1) << 28;
            const int cxm1 = cx - 1;
            for (uint32_t b = lo; b < hi; b += 32) {
                const uint32_t jl = b + lane;
                {
                    // stage: slots past the range load the last slot of the range and get |c|^2 = +inf,
                    // which no test accepts (inf plus finite terms stays inf, above the band)
                    const bool inr = jl < hi;
                    const uint32_t jc = inr ? jl : hi - 1u;
                    const float4 q = pos[jc];
                    const float qx = fmaf(cxs[jc] - gx15, fcell, q.x);
                    const float qy = q.y - hcell, qz = q.z - hcell;
                    float qw = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                    if (VARH) {
                        const float hj = hsf[jc];
                        qw = fmaf(-P.f_vlo * hj, hj, qw);
                        splane[4 * NL_THREADS + tid] = inr ? hj : 0.0f;
                    }
                    splane[tid] = qx;
                    splane[NL_THREADS + tid] = qy;
                    splane[2 * NL_THREADS + tid] = qz;
                    splane[3 * NL_THREADS + tid] = inr ? qw : __int_as_float(0x7f800000);
                }
                __syncwarp();
                // never its own neighbour
                const uint32_t selfbit = (self - b < 32u) ? 1u << (self - b) : 0u;
                uint32_t hitm = 0u, bandm = 0u;
                {
                    // every lane tests (lanes outside the group discard their mask): straight-line packed
                    // tests build the hit mask; the sign of r^2 - R2lo is shifted into the mask, candidate t
                    // ending at bit 31 - t after the alignment shift, and one reversal restores bit t. r^2 - R2lo =
                    // fma(mx, x, fma(my, y, fma(mz, z, |c|^2 + Kr))) on packed pairs of candidates (each lane
                    // of a pair rounded as the scalar operation); the band below R2hi is found from the
                    // smallest unsigned value of r^2 - R2lo (variable h: the widest band of this particle's
                    // pairs, h_j <= h). A candidate outside the own 3-bucket window is more than 2h away, so
                    // its FP32 r^2 cannot fall below the band and the fast test needs no window check.
                    const float hw = hif + (float)P.h;
                    const uint32_t wbits = VARH ? __float_as_uint((P.f_vhi - P.f_vlo) * hw * hw)
                                                : __float_as_uint(P.f_R2hi - P.f_R2lo);
                    uint32_t umin = 0xffffffffu;
                    const float2 mx2 = make_float2(mx, mx), my2 = make_float2(my, my), mz2 = make_float2(mz, mz);
                    const float2 kr2 = make_float2(Kr, Kr), mh2 = make_float2(mh, mh);
                    // the last batch of a row tests only its staged slots, in groups of four (the slots past
                    // the range hold |c|^2 = +inf and would add no hit)
                    const uint32_t nt = min(hi - b, 32u), ntest = (nt + 3u) & ~3u;
#pragma unroll
                    for (int t = 0; t < 32; t += 4) {
                        if (t > 0 && (uint32_t)t >= ntest) break;
                        const float4 X4 = *(const float4 *)&splane[wbase + t];
                        const float4 Y4 = *(const float4 *)&splane[NL_THREADS + wbase + t];
                        const float4 Z4 = *(const float4 *)&splane[2 * NL_THREADS + wbase + t];
                        const float4 W4 = *(const float4 *)&splane[3 * NL_THREADS + wbase + t];
                        float4 H4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (VARH) H4 = *(const float4 *)&splane[4 * NL_THREADS + wbase + t];
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const float2 xx = h2 ? make_float2(X4.z, X4.w) : make_float2(X4.x, X4.y);
                            const float2 yy = h2 ? make_float2(Y4.z, Y4.w) : make_float2(Y4.x, Y4.y);
                            const float2 zz = h2 ? make_float2(Z4.z, Z4.w) : make_float2(Z4.x, Z4.y);
                            const float2 ww = h2 ? make_float2(W4.z, W4.w) : make_float2(W4.x, W4.y);
                            float2 d = __fadd2_rn(ww, kr2);
                            if (VARH) d = __ffma2_rn(mh2, h2 ? make_float2(H4.z, H4.w) : make_float2(H4.x, H4.y), d);
                            d = __ffma2_rn(mz2, zz, d);
                            d = __ffma2_rn(my2, yy, d);
                            d = __ffma2_rn(mx2, xx, d);
                            hitm = __funnelshift_l(__float_as_uint(d.x), hitm, 1);
                            hitm = __funnelshift_l(__float_as_uint(d.y), hitm, 1);
                            umin = min(umin, min(__float_as_uint(d.x), __float_as_uint(d.y)));
                        }
                    }
                    hitm = __brev(hitm << (32u - ntest)) & ~selfbit;
                    // a candidate is in the band when 0 <= d < R2hi - R2lo, i.e. its bits as an unsigned
                    // integer are below those of the band width (negative d has the sign bit set); the
                    // smallest such bits of the batch say whether any is, and the rare batch that has one
                    // rebuilds the band mask with the same scalar roundings, then decides each member with
                    // its own window and the exactly rounded FP64 predicate
                    if (ing && umin < wbits) {
#pragma unroll 4
                        for (int t = 0; t < 32; ++t) {
                            float d0 = splane[3 * NL_THREADS + wbase + t] + Kr;
                            if (VARH) d0 = fmaf(mh, splane[4 * NL_THREADS + wbase + t], d0);
                            const float d = fmaf(mx, splane[wbase + t], fmaf(my, splane[NL_THREADS + wbase + t],
                                            fmaf(mz, splane[2 * NL_THREADS + wbase + t], d0)));
                            if (__float_as_uint(d) < wbits) bandm |= 1u << t;
                        }
                        bandm &= ~(hitm | selfbit);
                        while (bandm) {
                            const int t = __ffs(bandm) - 1;
                            bandm &= bandm - 1;
                            const int cxj = (int)cxs[b + (uint32_t)t];
                            if ((uint32_t)(cxj - cxm1) <= 2u &&
                                support_exact(P, xs, ys, zs, b + (uint32_t)t, xs[s], ys[s], zs[s], -1, 0.0,
                                              pair_R2(VARH, P, hid, VARH ? hs[b + (uint32_t)t] : 0.0)))
                                hitm |= 1u << t;
                        }
                    }
                    if (!ing) hitm = 0u;
                }
                // one entry per batch with a hit
                const bool any = hitm != 0u;
                if (any && cnt < (uint32_t)kmax) *out = make_uint2(hitm, b | code_yz);
                nlisted += (any && cnt < (uint32_t)kmax) ? (uint32_t)__popc(hitm) : 0u;
                out += any ? colstep : 0;
                cnt += any ? 1u : 0u;
                __syncwarp();
            }
        }
        need = need && !ing;
    }
    if (valid) cnt_out[s] = min(cnt, 255u) | nlisted << 8;
}

// ---------------------------------------------------------------------------------------------
// Pair kernel: list walk, wall images, integration.
//
// Modes (Sec. II steps d-f):
//   PM_ALL      every pair of every particle in one pass, then the integration.
//   PM_LOCAL    the pairs of each particle with neighbours of its own label (and the wall images of
//               those). Particles without a neighbour of another label (not MGPU boundary particles)
//               are complete and integrate; boundary particles park their partial sums (by halo index).
//   PM_BOUNDARY one lane per MGPU boundary particle (the boundary list, label-major): the partial sums
//               back, the pairs with neighbours of other labels, whose records come from the halo
//               buffer (the broadcast boundary set), then the integration.
// ---------------------------------------------------------------------------------------------
//   PM_HEUN1    all pairs; the Euler prediction y* = E(y_n) goes to the output state (no time step).
//   PM_HEUN2    all pairs of the predicted state, whose records the refresh rebuilt, over the lists of the
//               step's start (the re-scan paths decide membership on the step-start FP64 positions);
//               y_{n+1} = (y_n + E(y*)) / 2 on the conserved variables, then the time step.
//   PM_GRAD     MUSCL gradient pass: the SPH gradients of v and sigma over all pairs into the gradient
//               record (no integration).
//   PM_MUSCL    all pairs with MUSCL-reconstructed Riemann states, then the integration.
enum { PM_ALL = 0, PM_LOCAL = 1, PM_BOUNDARY = 2, PM_HEUN1 = 3, PM_HEUN2 = 4, PM_GRAD = 5, PM_MUSCL = 6 };

template <bool SPLIT>
struct PairArgs {
    using Pos = typename Types<SPLIT>::Pos;
    using Rec = typename Types<SPLIT>::Rec;
    DevParams P;
    int64_t n;
    const uint32_t *skey;
    const uint2 *cellr;
    const Pos *pos;
    const Rec *rec;
    const float *cxs;
    const double *xs, *ys, *zs;
    int kmax;
    const uint2 *list;
    const uint32_t *cnt_in;
    const uint32_t *perm;
    State A, B;
    const uint8_t *lab_s, *mat_s;
    const uint32_t *id_s;
    const double *dt_ptr;
    DtArgs dtc;                  // time-step reduction (candidate filter of the new state's signal speeds)
    unsigned long long *pairs;
    unsigned long long *cost;    // pair interactions per label of this step (Sec. V cost function)
    int32_t *nreal_out, *nimage_out;
    double *rates_out;
    // two-pass order only
    const uint8_t *flag;         // MGPU boundary flag per slot
    const uint32_t *blist;       // boundary slots, label-major (halo index -> slot)
    const unsigned long long *btotal;   // boundary set size
    const uint32_t *hidx;        // slot -> halo index (boundary particles)
    const Pos *hpos;             // halo records by halo index
    const Rec *hrec;
    const float *hcx;
    void *part;                  // parked partial sums by halo index: field f at f * n + h
    int32_t *part_cnt;           // parked real and image neighbour counts: 2 * h, 2 * h + 1
    // MUSCL only: gradient records, 7 G4 per slot (written by PM_GRAD, read by PM_MUSCL)
    typename Types<SPLIT>::G4 *grad;
    // variable h only: sorted smoothing lengths, FP64 and FP32
    const double *hs;
    const float *hsf;
    // split path, linear EOS: the records of the integrated state by slot (the next reorder gathers them)
    RecF *rec_next;
};

template <bool SPLIT, bool DIAG, int MODE, bool VARH>
__device__ __forceinline__ void pair_body(const PairArgs<SPLIT> &a, int64_t s, bool valid, int64_t hk) {
    using R = typename Types<SPLIT>::R;
    using Pos = typename Types<SPLIT>::Pos;
    using Rec = typename Types<SPLIT>::Rec;
    using G4 = typename Types<SPLIT>::G4;
    constexpr bool GRAD = MODE == PM_GRAD, RECON = MODE == PM_MUSCL;
    const DevParams &P = a.P;
    const int64_t n = a.n;
    const Pos *__restrict__ pos = a.pos;
    const Rec *__restrict__ rec = a.rec;
    const float *__restrict__ cxs = a.cxs;
    const double *__restrict__ xs = a.xs;
    const double *__restrict__ ys = a.ys;
    const double *__restrict__ zs = a.zs;
    const uint2 *__restrict__ list = a.list;
    const int kmax = a.kmax;
    const int lane = threadIdx.x & 31;
    const uint32_t key = valid ? a.skey[s] : P.ncell;
    const bool active = valid && key < P.ncell;
    PIn<R> me;
    R mrx = 0, mry = 0, mrz = 0;   // own position: relative to the own bucket corner (split) or absolute
    if (active) {
        const Pos p = pos[s];
        mrx = p.x; mry = p.y; mrz = p.z;
        me = load_rec(rec, p.w, s);
    } else {
        me = PIn<R>{};
    }
    const R inv_2h = SPLIT ? (R)(0.5f * P.f_inv_h) : (R)(0.5 / P.h);
    const R kdwh = SPLIT ? (R)(P.f_kdw * P.f_inv_h) : (R)(P.kdw / P.h);
    // variable h: the own length; kernel factors of a pair with length hj: 1/(2 h_ij) = 1/(h_i + h_j)
    // and kdw/h of h_ij = k5 (1/(h_i + h_j))^5, the same bits at both ends (h_i + h_j commutes)
    const R hme = VARH && active ? (SPLIT ? (R)a.hsf[s] : (R)a.hs[s]) : R(0);
    const double hmed = VARH && active ? a.hs[s] : 0.0;
    auto kfac = [&](R hj, R &i2h, R &kw) {
        if (VARH) {
            const R inv = rcp_r(hme + hj);
            const R i2 = inv * inv;
            i2h = inv;
            kw = (SPLIT ? (R)P.f_k5 : (R)P.k5) * (i2 * i2) * inv;
        } else {
            i2h = inv_2h;
            kw = kdwh;
        }
    };
    auto hof = [&](uint32_t j) -> R { return VARH ? (SPLIT ? (R)a.hsf[j] : (R)a.hs[j]) : R(0); };
    const R fcell = SPLIT ? (R)P.f_cell : (R)P.cell;
    // label filter of the two-pass order: PM_LOCAL takes neighbours of the own label, PM_BOUNDARY the others
    constexpr bool ALLPAIRS = MODE == PM_ALL || MODE == PM_HEUN1 || MODE == PM_HEUN2 || GRAD || RECON;
    const uint32_t mylab = (!ALLPAIRS && valid) ? a.lab_s[s] : 0u;
    auto take = [&](uint32_t j) -> bool {
        if (ALLPAIRS) return true;
        const bool same = a.lab_s[j] == mylab;
        return MODE == PM_LOCAL ? same : !same;
    };
    Acc<R> acc;
    acc.zero();
    // MUSCL: gradient sums (PM_GRAD), or the own gradient record staged in shared memory (PM_MUSCL)
    R gs[kNGrad];
#pragma unroll
    for (int k = 0; k < kNGrad; ++k) gs[k] = R(0);
    G4 *gme = nullptr;
    if constexpr (RECON) {
        __shared__ G4 gsh[7 * PK_THREADS];
        gme = gsh + threadIdx.x;
#pragma unroll
        for (int q = 0; q < 7; ++q) gme[q * PK_THREADS] = valid ? a.grad[(size_t)s * 7 + q] : G4{};
    }
    auto load_grad = [&](const G4 *src, int stride, R *G) {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const G4 g = src[q * stride];
            G[4 * q] = g.x;
            if (4 * q + 1 < kNGrad) G[4 * q + 1] = g.y;
            if (4 * q + 2 < kNGrad) G[4 * q + 2] = g.z;
            if (4 * q + 3 < kNGrad) G[4 * q + 3] = g.w;
        }
    };
    // one pair's work from the raw difference e (this end's x_oth - x_me) and the neighbour's state:
    // gradient sums, or the (reconstructed) fluxes. jg: the neighbour's slot for its gradient record,
    // wax >= 0 for a wall image (mirrored state and gradient; me is the left state)
    auto pair_work = [&](R e0, R e1, R e2, const PIn<R> &oth, R sgn, R kw, R inv_2h, uint32_t jg, int wax) {
        if constexpr (GRAD) {
            const R r2 = e0 * e0 + e1 * e1 + e2 * e2;
            const R inv_r = rsqrt_r(r2);
            const R r = r2 * inv_r;
            R sq = R(1) - inv_2h * r;
            const R c = kw * r * sq * sq * sq * oth.w * inv_r;   // w_j |dW/dr| / r
            const R g0 = c * e0, g1 = c * e1, g2 = c * e2;       // w_j grad_i W_ij
#pragma unroll
            for (int f = 0; f < 9; ++f) {
                const R d = pin_field(oth, f) - pin_field(me, f);
                gs[3 * f] += d * g0;
                gs[3 * f + 1] += d * g1;
                gs[3 * f + 2] += d * g2;
            }
        } else if constexpr (RECON) {
            R Gm[kNGrad], Go[kNGrad];
            load_grad(gme, PK_THREADS, Gm);
            load_grad(a.grad + (size_t)jg * 7, 1, Go);
            if (wax >= 0) mirror_grad(Go, wax);
            PIn<R> mes, oths;
            reconstruct(me, Gm, oth, Go, e0, e1, e2, mes, oths);
            PairRes<R> o;
            pair_terms<R, false, true>(e0, e1, e2, mes, oths, sgn, inv_2h, kw, o, me, oth);
            accumulate<R, false>(acc, o, -sgn, me, oth);
        } else {
            PairRes<R> o;
            pair_terms<R, MODE == PM_HEUN2>(e0, e1, e2, me, oth, sgn, inv_2h, kw, o, me, oth);
            accumulate<R>(acc, o, -sgn, me, oth);
        }
    };
    int nr0 = 0, ni0 = 0;
    if (MODE == PM_BOUNDARY && valid) {   // the partial sums of the first pass
        const R *pr = (const R *)a.part;
        acc.load(pr, n, hk);
        nr0 = a.part_cnt[2 * hk];
        ni0 = a.part_cnt[2 * hk + 1];
    }
    const uint32_t cw = active ? a.cnt_in[s] : 0u;
    const uint32_t cnt = cw & 255u;                  // entries found
    const int ne = (int)min(cnt, (uint32_t)kmax);    // entries stored
    const uint32_t nlist = cw >> 8;                  // neighbours in the stored entries
    const R cxf = SPLIT ? (R)(active ? cxs[s] : 0.0f) : R(0);   // own bucket x

    // one real neighbour jj, in row (dcy, dcz) = code - 1 and bucket x cxj: canonical orientation (the
    // lower sorted slot is the left state); both ends of the pair evaluate x_R - x_L from the same
    // operands in the same order
    // act = false evaluates a harmless stand-in pair (a nonzero offset, kernel weight 0) that adds zeros,
    // so the listed-neighbour loop needs no branch around the pair
    auto real_pair = [&](uint32_t jj, uint32_t code, R cxj, const Pos &pj, const Rec &rj, bool act, R hj) {
        const PIn<R> oth = unpack(rj, (R)pj.w);
        // x_j - x_i from this end; the exact factor sgn orients it L -> R inside the pair terms, so both
        // ends obtain the same canonical normal bit for bit (a - b = -(b - a) in IEEE arithmetic)
        const R sgn = s < (int64_t)jj ? R(1) : R(-1);
        R d0, d1, d2;
        if (SPLIT) {
            const R ey = (R)(int)(code & 3u) * fcell - fcell, ez = (R)(int)(code >> 2) * fcell - fcell;
            d0 = ((R)pj.x - mrx) + (cxj - cxf) * fcell;
            d1 = ((R)pj.y - mry) + ey;
            d2 = ((R)pj.z - mrz) + ez;
        } else {
            d0 = (R)pj.x - mrx; d1 = (R)pj.y - mry; d2 = (R)pj.z - mrz;
        }
        if (!act) d0 = fcell;
        R i2h, kw;
        kfac(hj, i2h, kw);
        pair_work(d0, d1, d2, oth, sgn, act ? kw : R(0), i2h, jj, -1);
    };

    // ---- listed real neighbours, all lanes in lockstep: the set bits of the current entry give the
    // slots; the entry after it and the next neighbour's record are in flight while the current pair
    // is evaluated
    int nsel = 0;   // listed neighbours taken by this pass
    {
        const uint2 *lp = list + (size_t)s;
        const size_t colstep = (size_t)n;
        uint32_t m = 0u, y = 0u;
        uint2 nx = make_uint2(0u, 0u);
        if (ne > 0) { const uint2 e = lp[0]; m = e.x; y = e.y; }
        if (ne > 1) nx = lp[colstep];
        int ke = 2;
        // next listed neighbour when `more` (a neighbour is left), by selects rather than a branch: slot j,
        // row code c, the highest set bit of the mask first (the order within a batch only affects
        // rounding); refills the mask from the entry in flight when the current one is used up (the
        // refill's load predicated). Without `more`, j and c keep a valid slot. The record loads that
        // follow are unconditional (a lane past its last neighbour reloads its last valid slot), which
        // keeps the loop body free of branches
        auto next = [&](bool more, uint32_t &j, uint32_t &c) {
            const int t = 31 - __clz(m | 1u);
            const uint32_t mn = m ^ (1u << t);
            const uint32_t jn = (y & IT_JMASK) + (uint32_t)t;
            const uint32_t cn = y >> 26;
            j = more ? jn : j;
            c = more ? cn : c;
            const bool rf = more && mn == 0u;
            m = more ? (rf ? nx.x : mn) : m;
            y = rf ? nx.y : y;
            if (rf && ke < ne) nx = lp[(size_t)ke * colstep];
            ke += rf ? 1 : 0;
        };
        // record source: the particle arrays, or (second pass, other labels) the halo buffer
        auto fetch = [&](uint32_t j, bool t, Pos &pj, Rec &rj, float &xj, R &hj) {
            hj = hof(j);
            if (MODE == PM_BOUNDARY) {
                const uint32_t h = t ? a.hidx[j] : 0u;
                pj = a.hpos[h];
                rj = a.hrec[h];
                xj = SPLIT ? a.hcx[h] : 0.0f;
            } else {
                pj = pos[j];
                rj = rec[j];
                xj = SPLIT ? cxs[j] : 0.0f;
            }
        };
        const int mc = (int)__reduce_max_sync(kFullMask, nlist);
        uint32_t j1 = 0u, c1 = 0u;
        next(nlist > 0, j1, c1);
        bool t1 = take(j1);
        Pos p1;
        Rec r1;
        float x1;
        R h1;
        fetch(j1, t1, p1, r1, x1, h1);
        // unrolled twice (measured faster than 1, 3, 4 or 8); the MUSCL flux pass (168 registers) measured
        // faster with the loop rolled
#pragma unroll (MODE == PM_MUSCL ? 1 : 2)
        for (int k = 0; k < mc; ++k) {
            const uint32_t j = j1, c = c1;
            const Pos pj = p1;
            const Rec rj = r1;
            const float xj = x1;
            const R hj = h1;
            const bool tj = t1;
            next((uint32_t)k + 1 < nlist, j1, c1);   // else j1 stays a valid slot
            t1 = take(j1);
            fetch(j1, t1, p1, r1, x1, h1);
            const bool act = (uint32_t)k < nlist && tj;
            real_pair(j, c, (R)xj, pj, rj, act, hj);
            if (!ALLPAIRS) nsel += act ? 1 : 0;
            if ((k & 7) == 7) acc.fold();
        }
    }

    // ---- neighbours beyond the list capacity, and the wall images: re-scan the buckets around the
    // own position (overflow) or the mirrored position (images) in the list's candidate order. In the
    // two-pass order this rare path reads the particle arrays.
    const double X = valid ? xs[s] : 0.0, Y = valid ? ys[s] : 0.0, Z = valid ? zs[s] : 0.0;
    // own FP64 position of the fluxes: the step's start, or the predicted state in the second Heun stage
    // (the search keeps X, Y, Z)
    const double XF = (MODE == PM_HEUN2 && valid) ? a.B.f[FX][s] : X;
    const double YF = (MODE == PM_HEUN2 && valid) ? a.B.f[FY][s] : Y;
    const double ZF = (MODE == PM_HEUN2 && valid) ? a.B.f[FZ][s] : Z;
    int cx = 0, cy = 0, cz = 0;
    if (active) decode_cell(P, key, cx, cy, cz);
    int ni = 0;
    uint32_t nover = 0;
    for (int src = (__any_sync(kFullMask, (int)cnt > kmax) ? 0 : 1); src <= P.nwalls; ++src) {
        const int wax = src > 0 ? P.wall_axis[src - 1] : -1;
        const double wpos = src > 0 ? P.wall_pos[src - 1] : 0.0;
        // a particle farther than the support from the wall plane (with a 1e-6 margin over the FP64
        // roundings) has no image neighbour: |x_i - x_j'| >= |x_i - w| for j on the same side. Warps with
        // no particle near the wall skip the mirrored search.
        bool near = src == 0;
        if (src > 0) {
            const double dw = __dsub_rn(wax == 0 ? X : (wax == 1 ? Y : Z), wpos);
            near = fabs(dw) <= P.wall_reach;
            if (!__any_sync(kFullMask, active && near)) continue;
        }
        double CX = X, CY = Y, CZ = Z;
        int bx = cx, by = cy, bz = cz;
        R ox = mrx, oy = mry, oz = mrz;
        if (src > 0) {
            const double two_w = __dmul_rn(2.0, wpos);
            if (wax == 0) CX = __dsub_rn(two_w, X);
            if (wax == 1) CY = __dsub_rn(two_w, Y);
            if (wax == 2) CZ = __dsub_rn(two_w, Z);
            bx = bucket_coord_signed(CX, P.lo[0], P.cell);
            by = bucket_coord_signed(CY, P.lo[1], P.cell);
            bz = bucket_coord_signed(CZ, P.lo[2], P.cell);
            // the flux offsets use the mirrored flux position (the search one except in Heun stage 2)
            double FX_ = XF, FY_ = YF, FZ_ = ZF;
            if (wax == 0) FX_ = __dsub_rn(two_w, XF);
            if (wax == 1) FY_ = __dsub_rn(two_w, YF);
            if (wax == 2) FZ_ = __dsub_rn(two_w, ZF);
            if (SPLIT) {
                // (the corner as the reorder's tables hold it; bx may lie outside the grid here)
                ox = (R)(FX_ - __fma_rn((double)bx, P.cell, P.lo[0]));
                oy = (R)(FY_ - __fma_rn((double)by, P.cell, P.lo[1]));
                oz = (R)(FZ_ - __fma_rn((double)bz, P.cell, P.lo[2]));
            } else {
                ox = (R)FX_; oy = (R)FY_; oz = (R)FZ_;
            }
        }
        const bool mine = active && (src > 0 ? near : (int)cnt > kmax);
        if (!__any_sync(kFullMask, mine)) continue;
        uint32_t seen = 0;
        for (int row = 0; row < 9 && mine; ++row) {
            const int dcy = row % 3 - 1, dcz = row / 3 - 1;
            uint32_t rs, re;
            row_window(P, a.cellr, bx, by + dcy, bz + dcz, rs, re);
            for (uint32_t j = rs; j < re; ++j) {
                if (src == 0 && (int64_t)j == s) continue;
                const Pos pj = pos[j];
                const int dcx = (int)cxs[j] - bx;
                bool hit;
                const double R2j = pair_R2(VARH, P, hmed, VARH ? a.hs[j] : 0.0);
                if (MODE == PM_HEUN2) {   // membership from the step's start: the FP64 positions
                    hit = support_exact(P, xs, ys, zs, j, X, Y, Z, wax, wpos, R2j);
                } else if (SPLIT) {
                    const float exf = ((float)pj.x - (float)ox) + (float)dcx * (float)fcell;
                    const float eyf = ((float)pj.y - (float)oy) + (float)dcy * (float)fcell;
                    const float ezf = ((float)pj.z - (float)oz) + (float)dcz * (float)fcell;
                    const float r2 = exf * exf + eyf * eyf + ezf * ezf;
                    float lo = P.f_R2lo, hi = P.f_R2hi;
                    if (VARH) {
                        const float sf = (float)hme + a.hsf[j];
                        lo = P.f_vlo * sf * sf;
                        hi = P.f_vhi * sf * sf;
                    }
                    hit = r2 < lo;
                    if (!hit && r2 < hi) hit = support_exact(P, xs, ys, zs, j, X, Y, Z, wax, wpos, R2j);
                } else {
                    hit = support_exact(P, xs, ys, zs, j, X, Y, Z, wax, wpos, R2j);
                }
                if (!hit) continue;
                if (src == 0) {
                    // real neighbour past the list capacity
                    if (seen++ < nlist) continue;
                    if (!take(j)) continue;
                    real_pair(j, (uint32_t)(dcy + 1) | (uint32_t)(dcz + 1) << 2, (R)cxs[j], pj, rec[j], true, hof(j));
                    ++nover;
                } else {
                    if (!take(j)) continue;
                    PIn<R> oth = load_rec(rec, (R)pj.w, j);
                    R d0, d1, d2;
                    if (SPLIT) {
                        d0 = ((R)pj.x - ox) + (R)dcx * fcell;
                        d1 = ((R)pj.y - oy) + (R)dcy * fcell;
                        d2 = ((R)pj.z - oz) + (R)dcz * fcell;
                        if (wax == 0) d0 = -d0;
                        if (wax == 1) d1 = -d1;
                        if (wax == 2) d2 = -d2;
                    } else {
                        double qx = (double)pj.x, qy = (double)pj.y, qz = (double)pj.z;
                        const double two_w = 2.0 * wpos;
                        if (wax == 0) qx = two_w - qx;
                        if (wax == 1) qy = two_w - qy;
                        if (wax == 2) qz = two_w - qz;
                        d0 = (R)(qx - XF); d1 = (R)(qy - YF); d2 = (R)(qz - ZF);
                    }
                    mirror<R>(oth, wax);
                    R i2h, kw;
                    kfac(hof(j), i2h, kw);
                    pair_work(d0, d1, d2, oth, R(1), kw, i2h, j, wax);
                    ++ni;
                }
            }
        }
    }
    if constexpr (GRAD) {
        if (valid) {
            G4 *out = a.grad + (size_t)s * 7;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                G4 g;
                g.x = gs[4 * q];
                g.y = 4 * q + 1 < kNGrad ? gs[4 * q + 1] : R(0);
                g.z = 4 * q + 2 < kNGrad ? gs[4 * q + 2] : R(0);
                g.w = 4 * q + 3 < kNGrad ? gs[4 * q + 3] : R(0);
                out[q] = g;
            }
        }
        return;
    }
    acc.fold();
    const int ntaken = ALLPAIRS ? (int)nlist : nsel;   // listed neighbours summed by this pass
    const unsigned pc = __reduce_add_sync(kFullMask, (unsigned)(ntaken + (int)nover + ni));
    const int nr = nr0 + ntaken + (int)nover;
    ni += ni0;

    // ---- first pass of the two-pass order: a boundary particle parks its sums for the second pass
    bool integrate = valid;
    if (MODE == PM_LOCAL && valid && a.flag[s]) {
        const uint32_t h = a.hidx[s];
        acc.store((R *)a.part, n, h);
        a.part_cnt[2 * (size_t)h] = nr;
        a.part_cnt[2 * (size_t)h + 1] = ni;
        integrate = false;
    }

    // ---- integration (Sec. II step g): forward Euler on the conserved variables, Jaumann-rate
    // stress with radial return, positions with the velocity of the step's start.
    // (the new state's inputs of the next time step)
    double tm_ = 0.0, tw = 1.0, tvx = 0.0, tvy = 0.0, tvz = 0.0, tE = 0.0;
    int tmat = 0;
    if (integrate) {
        const State &A = a.A;
        const State &B = a.B;
        const uint32_t o = a.perm[s];
        const int mt = a.mat_s[s] < P.nmat ? a.mat_s[s] : 0;
        const double dt = *a.dt_ptr;
        // the state the Euler stage starts from: y_n (A through the permutation), or y* (B in slot order)
        const State &Y0 = MODE == PM_HEUN2 ? B : A;
        const uint32_t o0 = MODE == PM_HEUN2 ? (uint32_t)s : o;
        const double w = Y0.f[FW][o0], m = Y0.f[FM][o0], E = Y0.f[FE][o0];
        const double vx = Y0.f[FVX][o0], vy = Y0.f[FVY][o0], vz = Y0.f[FVZ][o0];
        double S[6] = {Y0.f[FSXX][o0], Y0.f[FSYY][o0], Y0.f[FSZZ][o0], Y0.f[FSXY][o0], Y0.f[FSXZ][o0], Y0.f[FSYZ][o0]};
        double r6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) r6[k] = acc.get(k);
        // split path (Euler stage): the increments of v, E and S in FP32 from the FP32 rates, each added once
        // to the FP64 state: v_{n+1} = v + dt (F - v dm) / m_{n+1}, E_{n+1} = E + dt (dE - E dm) / m_{n+1},
        // the same update as (m v + dt F) / m_{n+1}; w, m and x advance in FP64
        constexpr bool FAST = SPLIT && MODE != PM_HEUN2;
        const double wn = w + dt * r6[0];
        const double mn = m + dt * r6[1];
        double nvx, nvy, nvz, En, Sn[6];
        double mvx = 0.0, mvy = 0.0, mvz = 0.0, mE = 0.0;
        R Lm[3][3];
        if constexpr (RECON) {   // the velocity gradient of the gradient record (the same sum)
            R Gm[kNGrad];
            load_grad(gme, PK_THREADS, Gm);
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) Lm[u][v] = Gm[3 * u + v];
        } else {
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) Lm[u][v] = acc.getr(6 + 3 * u + v);
        }
        // the stress of the step's start as the record holds it (the FP32 rounding on the split path)
        // (split: the record's sigma plus the pressure its trace gives; FP64: the state's S)
        R Sr[3][3];
        if (SPLIT) {
            const R pr = -(me.txx + me.tyy + me.tzz) * (R(1) / R(3));
            Sr[0][0] = me.txx + pr; Sr[1][1] = me.tyy + pr; Sr[2][2] = me.tzz + pr;
            Sr[0][1] = Sr[1][0] = me.sxy;
            Sr[0][2] = Sr[2][0] = me.sxz;
            Sr[1][2] = Sr[2][1] = me.syz;
        } else {
            Sr[0][0] = (R)S[0]; Sr[1][1] = (R)S[1]; Sr[2][2] = (R)S[2];
            Sr[0][1] = Sr[1][0] = (R)S[3];
            Sr[0][2] = Sr[2][0] = (R)S[4];
            Sr[1][2] = Sr[2][1] = (R)S[5];
        }
        const R trD = Lm[0][0] + Lm[1][1] + Lm[2][2];
        const R G2 = SPLIT ? (R)(2.0f * P.f_G[mt]) : (R)(2.0 * P.G[mt]);
        const int iu[6] = {0, 1, 2, 0, 0, 1}, iv[6] = {0, 1, 2, 1, 2, 2};
        R srate[6];   // stress rate 2G (D - tr D / 3) + Om S - S Om
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int u = iu[q], v = iv[q];
            R D = R(0.5) * (Lm[u][v] + Lm[v][u]);
            if (u == v) D -= trD / R(3);
            R rot = R(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const R Ouk = R(0.5) * (Lm[u][k] - Lm[k][u]);
                const R Okv = R(0.5) * (Lm[k][v] - Lm[v][k]);
                rot += Ouk * Sr[k][v] - Sr[u][k] * Okv;
            }
            srate[q] = G2 * D + rot;
        }
        const R Yr = SPLIT ? (R)(float)P.Y[mt] : (R)P.Y[mt];
        if (FAST) {
            const float dtf = (float)dt, imf = 1.0f / (float)mn, mf = (float)(me.rho * me.w), dm = (float)acc.getr(1);
            float F[3] = {(float)acc.getr(2), (float)acc.getr(3), (float)acc.getr(4)}, dE = (float)acc.getr(5);
            if (P.has_gravity) {
                const float g0 = (float)P.g[0], g1 = (float)P.g[1], g2 = (float)P.g[2];
                F[0] += mf * g0; F[1] += mf * g1; F[2] += mf * g2;
                dE += mf * (g0 * me.vx + g1 * me.vy + g2 * me.vz);
            }
            nvx = vx + (double)(dtf * (F[0] - me.vx * dm) * imf);
            nvy = vy + (double)(dtf * (F[1] - me.vy * dm) * imf);
            nvz = vz + (double)(dtf * (F[2] - me.vz * dm) * imf);
            En = E + (double)(dtf * (dE - me.E * dm) * imf);
            // stress increment; its trace removed in FP32 (the state's own trace is zero to rounding)
            float dS[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) dS[q] = dtf * (float)srate[q];
            const float tr3 = (dS[0] + dS[1] + dS[2]) * (1.0f / 3.0f);
            dS[0] -= tr3; dS[1] -= tr3; dS[2] -= tr3;
            const float a0 = (float)Sr[0][0] + dS[0], a1 = (float)Sr[1][1] + dS[1], a2 = (float)Sr[2][2] + dS[2];
            const float a3 = (float)Sr[0][1] + dS[3], a4 = (float)Sr[0][2] + dS[4], a5 = (float)Sr[1][2] + dS[5];
#pragma unroll
            for (int q = 0; q < 6; ++q) Sn[q] = S[q] + (double)dS[q];
            const float ss = a0 * a0 + a1 * a1 + a2 * a2 + 2.0f * (a3 * a3 + a4 * a4 + a5 * a5);
            const float seq = sqrtf(1.5f * ss);
            if (seq > (float)Yr) {
                const double f = (double)((float)Yr / seq);
#pragma unroll
                for (int q = 0; q < 6; ++q) Sn[q] *= f;
            }
        } else {
            if (P.has_gravity) {   // body force m g and its power m g.v (skipped when g = 0: the same values)
                const double gv = P.g[0] * vx + P.g[1] * vy + P.g[2] * vz;
                r6[2] += m * P.g[0];
                r6[3] += m * P.g[1];
                r6[4] += m * P.g[2];
                r6[5] += m * gv;
            }
            mvx = m * vx + dt * r6[2];
            mvy = m * vy + dt * r6[3];
            mvz = m * vz + dt * r6[4];
            mE = m * E + dt * r6[5];
#pragma unroll
            for (int q = 0; q < 6; ++q) Sn[q] = S[q] + dt * (double)srate[q];
            const double trS = (Sn[0] + Sn[1] + Sn[2]) / 3.0;
            Sn[0] -= trS; Sn[1] -= trS; Sn[2] -= trS;
            const R a0 = (R)Sn[0], a1 = (R)Sn[1], a2 = (R)Sn[2], a3 = (R)Sn[3], a4 = (R)Sn[4], a5 = (R)Sn[5];
            const R ss = a0 * a0 + a1 * a1 + a2 * a2 + R(2) * (a3 * a3 + a4 * a4 + a5 * a5);
            const R seq = sqrt(R(1.5) * ss);
            if (seq > Yr) {
                const double f = (double)(Yr / seq);
#pragma unroll
                for (int q = 0; q < 6; ++q) Sn[q] *= f;
            }
            double inv_mn;
            if (SPLIT) {   // FP32 estimate refined by two Newton steps (relative error at the FP64 rounding level)
                const double r0 = (double)__fdividef(1.0f, (float)mn);
                const double r1 = fma(r0, fma(-mn, r0, 1.0), r0);
                inv_mn = fma(r1, fma(-mn, r1, 1.0), r1);
            } else {
                inv_mn = 1.0 / mn;
            }
            nvx = mvx * inv_mn; nvy = mvy * inv_mn; nvz = mvz * inv_mn;
            En = mE * inv_mn;
        }

        double xn = XF + dt * vx, yn = YF + dt * vy, zn = ZF + dt * vz;
        double wo = wn, mo = mn;
        if (MODE == PM_HEUN2) {
            // y_{n+1} = (y_n + E(y*)) / 2 on the conserved variables w, m, m v, m E, x, S
            const double w0 = A.f[FW][o], m0 = A.f[FM][o];
            const double mh = 0.5 * (m0 + mn);
            const double imh = 1.0 / mh;
            nvx = 0.5 * (m0 * A.f[FVX][o] + mvx) * imh;
            nvy = 0.5 * (m0 * A.f[FVY][o] + mvy) * imh;
            nvz = 0.5 * (m0 * A.f[FVZ][o] + mvz) * imh;
            En = 0.5 * (m0 * A.f[FE][o] + mE) * imh;
            xn = 0.5 * (X + xn);
            yn = 0.5 * (Y + yn);
            zn = 0.5 * (Z + zn);
            wo = 0.5 * (w0 + wn);
            mo = mh;
            Sn[0] = 0.5 * (A.f[FSXX][o] + Sn[0]);
            Sn[1] = 0.5 * (A.f[FSYY][o] + Sn[1]);
            Sn[2] = 0.5 * (A.f[FSZZ][o] + Sn[2]);
            Sn[3] = 0.5 * (A.f[FSXY][o] + Sn[3]);
            Sn[4] = 0.5 * (A.f[FSXZ][o] + Sn[4]);
            Sn[5] = 0.5 * (A.f[FSYZ][o] + Sn[5]);
        }
        B.f[FX][s] = xn;
        B.f[FY][s] = yn;
        B.f[FZ][s] = zn;
        B.f[FVX][s] = nvx;
        B.f[FVY][s] = nvy;
        B.f[FVZ][s] = nvz;
        B.f[FW][s] = wo;
        B.f[FM][s] = mo;
        B.f[FE][s] = En;
        B.f[FSXX][s] = Sn[0];
        B.f[FSYY][s] = Sn[1];
        B.f[FSZZ][s] = Sn[2];
        B.f[FSXY][s] = Sn[3];
        B.f[FSXZ][s] = Sn[4];
        B.f[FSYZ][s] = Sn[5];
        B.mat[s] = a.mat_s[s];
        B.label[s] = a.lab_s[s];
        B.id[s] = a.id_s[s];
        if (SPLIT && MODE != PM_HEUN1 && a.rec_next)   // the end state's record, as the reorder forms it
            a.rec_next[s] = record_split_linear(P, mt, wo, mo, nvx, nvy, nvz, En, Sn[0], Sn[1], Sn[3], Sn[4], Sn[5]);
        if (VARH) B.h[s] = A.h[o];
        if (DIAG && MODE != PM_HEUN2) {   // the step's counts and rates: those of its start
            a.nreal_out[s] = nr;
            a.nimage_out[s] = ni;
#pragma unroll
            for (int k = 0; k < kNRate; ++k)
                a.rates_out[(size_t)s * kNRate + k] = (RECON && k >= 6) ? (double)Lm[(k - 6) / 3][(k - 6) % 3] : acc.get(k);
        }
        tm_ = mo; tw = wo; tvx = nvx; tvy = nvy; tvz = nvz; tE = En; tmat = mt;
    }
    // next step's time step: the exact FP64 maximum of the signal speeds over the candidates this filter
    // lists (the Heun prediction's state is not a step's end)
    if (MODE != PM_HEUN1)
        dt_candidate(P, a.dtc, integrate, tmat, tm_, tw, tvx, tvy, tvz, tE,
                     (VARH && integrate) ? a.hs[s] : 1.0);
    if (lane == 0) atomicAdd(a.pairs, (unsigned long long)pc);
    // cost per label: this pass's pairs of the particle, summed over the lanes of each label
    {
        const uint32_t lab = valid ? (uint32_t)a.lab_s[s] : 0xffffffffu;
        const unsigned mine = MODE == PM_HEUN2 ? 0u : (unsigned)(ntaken + (int)nover + (ni - ni0));
        const unsigned peers = __match_any_sync(kFullMask, lab);
        const unsigned sum = __reduce_add_sync(peers, valid ? mine : 0u);
        if (valid && (__ffs(peers) - 1) == lane && sum) atomicAdd(&a.cost[lab], (unsigned long long)sum);
    }
}

// split path: 4 blocks/SM (128 registers, no spills) for the flux passes, 5 for the lighter gradient
// pass, 3 for the MUSCL flux pass (168 registers)
template <bool SPLIT, bool DIAG, int MODE, bool VARH = false>
__global__ void __launch_bounds__(PK_THREADS, SPLIT ? (MODE == PM_MUSCL ? 3 : (MODE == PM_GRAD ? 5 : 4)) : 2) k_pair(const PairArgs<SPLIT> a) {
    pdl_wait();      // a programmatic dependent launch (its predecessor's writes are visible from here)
    pdl_release();
    if (MODE == PM_BOUNDARY) {
        // one lane per boundary particle, warp-uniform strides over the boundary list
        const int64_t total = (int64_t)*a.btotal;
        const int64_t stride = (int64_t)gridDim.x * PK_THREADS;
        for (int64_t kb = (int64_t)blockIdx.x * PK_THREADS + (threadIdx.x & ~31); kb < total; kb += stride) {
            const int64_t k = kb + (threadIdx.x & 31);
            const bool valid = k < total;
            const int64_t s = valid ? (int64_t)a.blist[k] : 0;
            pair_body<SPLIT, DIAG, MODE, VARH>(a, s, valid, k);
        }
    } else {
        const int64_t s = (int64_t)blockIdx.x * PK_THREADS + threadIdx.x;
        pair_body<SPLIT, DIAG, MODE, VARH>(a, s, s < a.n, 0);
    }
}

// Gather of the MGPU boundary set's records into the halo buffer (the broadcast of Sec. II step d on
// one device): halo index h holds the particle at boundary-list position h.
template <bool SPLIT>
__global__ void k_halo_gather(const PairArgs<SPLIT> a, typename Types<SPLIT>::Pos *hpos,
                              typename Types<SPLIT>::Rec *hrec, float *hcx) {
    const int64_t total = (int64_t)*a.btotal;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < total; h += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = a.blist[h];
        hpos[h] = a.pos[s];
        hrec[h] = a.rec[s];
        hcx[h] = a.cxs[s];
    }
}

template <bool SPLIT>
static PairArgs<SPLIT> pair_args(const DevParams &P, int64_t n, const uint32_t *skey, const uint2 *cellr,
                                 const void *pos, const void *rec, const float *cxs, const double *xs,
                                 const double *ys, const double *zs, int kmax, const uint2 *list,
                                 const uint32_t *cnt, const uint32_t *perm, const State &A, const State &B,
                                 const uint8_t *lab_s, const uint8_t *mat_s, const uint32_t *id_s,
                                 const double *dt, const DtArgs &dtc, unsigned long long *pairs,
                                 unsigned long long *cost, int32_t *nreal, int32_t *nimage, double *rates,
                                 const OverlapBufs *ov, void *grad, const double *hs, const float *hsf,
                                 RecF *rec_next) {
    using Pos = typename Types<SPLIT>::Pos;
    using Rec = typename Types<SPLIT>::Rec;
    PairArgs<SPLIT> a;
    a.P = P; a.n = n; a.skey = skey; a.cellr = cellr; a.pos = (const Pos *)pos; a.rec = (const Rec *)rec;
    a.cxs = cxs; a.xs = xs; a.ys = ys; a.zs = zs; a.kmax = kmax; a.list = list; a.cnt_in = cnt; a.perm = perm;
    a.A = A; a.B = B; a.lab_s = lab_s; a.mat_s = mat_s; a.id_s = id_s; a.dt_ptr = dt; a.dtc = dtc;
    a.pairs = pairs; a.cost = cost; a.nreal_out = nreal; a.nimage_out = nimage; a.rates_out = rates;
    a.flag = ov ? ov->flag : nullptr;
    a.blist = ov ? ov->blist : nullptr;
    a.btotal = ov ? ov->btotal : nullptr;
    a.hidx = ov ? ov->hidx : nullptr;
    a.hpos = ov ? (const Pos *)ov->hpos : nullptr;
    a.hrec = ov ? (const Rec *)ov->hrec : nullptr;
    a.hcx = ov ? ov->hcx : nullptr;
    a.part = ov ? ov->part : nullptr;
    a.part_cnt = ov ? ov->part_cnt : nullptr;
    a.grad = (typename Types<SPLIT>::G4 *)grad;
    a.hs = hs;
    a.hsf = hsf;
    a.rec_next = SPLIT ? rec_next : nullptr;
    return a;
}

// The neighbour lists (before launch_interact): they read the sorted FP32 bucket-relative positions
// (pos_rel: the split record's, or the FP64 path's copy) and the bucket ranges only, so they can be built
// while the labels are still changing.
cudaError_t launch_nbr_list(const DevParams &P, int64_t n, const uint32_t *skey, const uint2 *cellr,
                            const float4 *pos_rel, const float *cxs, const double *xs, const double *ys,
                            const double *zs, int kmax, uint2 *list, uint32_t *cnt, const double *hs,
                            const float *hsf, unsigned long long *cost_clear, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned gl = (unsigned)((n + NL_THREADS - 1) / NL_THREADS);
    if (P.variable_h != 0)
        return pdl_launch(k_nbr_list<true>, dim3(gl), dim3(NL_THREADS), s, P, n, skey, cellr, pos_rel, cxs, xs, ys, zs,
                          kmax, list, cnt, hs, hsf, cost_clear);
    return pdl_launch(k_nbr_list<false>, dim3(gl), dim3(NL_THREADS), s, P, n, skey, cellr, pos_rel, cxs, xs, ys, zs,
                      kmax, list, cnt, hs, hsf, cost_clear);
}

cudaError_t launch_interact(bool split, bool diag, const DevParams &P, int64_t n, const uint32_t *skey,
                            const uint2 *cellr, const void *pos, const void *rec, const float *cxs,
                            const double *xs, const double *ys, const double *zs, int kmax, uint2 *list,
                            uint32_t *cnt, const uint32_t *perm, const State &A, const State &B, cudaEvent_t mid,
                            const uint8_t *lab_s, const uint8_t *mat_s, const uint32_t *id_s, const double *dt,
                            const DtArgs &dtc, unsigned long long *pairs, unsigned long long *cost,
                            int32_t *nreal, int32_t *nimage, double *rates, const OverlapBufs *ov,
                            int stage, void *grad, const double *hs, const float *hsf, void *rec_next,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const bool varh = P.variable_h != 0;
    const unsigned gp = (unsigned)((n + PK_THREADS - 1) / PK_THREADS);
#define GSPH_PAIR_ARGS pair_args<SP>(P, n, skey, cellr, pos, rec, cxs, xs, ys, zs, kmax, list, cnt, perm, A, B, \
                                     lab_s, mat_s, id_s, dt, dtc, pairs, cost, nreal, nimage, rates, ov, grad, hs, hsf, \
                                     (RecF *)rec_next)
#define GSPH_PAIRS(MODE_)                                                                   \
    do {                                                                                    \
        const auto pa = GSPH_PAIR_ARGS;                                                      \
        const unsigned g_ = MODE_ == PM_BOUNDARY ? ov->boundary_grid : gp;                  \
        if (varh) {                                                                         \
            if (diag) pdl_launch(k_pair<SP, true, MODE_, true>, dim3(g_), dim3(PK_THREADS), s, pa);  \
            else pdl_launch(k_pair<SP, false, MODE_, true>, dim3(g_), dim3(PK_THREADS), s, pa);      \
        } else {                                                                            \
            if (diag) pdl_launch(k_pair<SP, true, MODE_>, dim3(g_), dim3(PK_THREADS), s, pa);         \
            else pdl_launch(k_pair<SP, false, MODE_>, dim3(g_), dim3(PK_THREADS), s, pa);             \
        }                                                                                   \
    } while (0)
#define GSPH_INTERACT                                                                       \
    do {                                                                                    \
        if (mid) cudaEventRecord(mid, s);                                                   \
        if (stage == 1) {                                                                   \
            GSPH_PAIRS(PM_HEUN1);                                                           \
        } else if (stage == 2) {                                                            \
            GSPH_PAIRS(PM_HEUN2);                                                           \
        } else if (grad) {                                                                  \
            /* MUSCL: the gradient pass, then the reconstructed fluxes */                  \
            if (varh) k_pair<SP, false, PM_GRAD, true><<<gp, PK_THREADS, 0, s>>>(GSPH_PAIR_ARGS); \
            else k_pair<SP, false, PM_GRAD><<<gp, PK_THREADS, 0, s>>>(GSPH_PAIR_ARGS);      \
            GSPH_PAIRS(PM_MUSCL);                                                           \
        } else if (!ov) {                                                                   \
            GSPH_PAIRS(PM_ALL);                                                             \
        } else {                                                                            \
            /* step d on the second stream while the local pairs run (steps e, then f) */  \
            cudaEventRecord(ov->ev_fork, s);                                                \
            cudaStreamWaitEvent(ov->aux, ov->ev_fork, 0);                                   \
            if (ov->ev_halo0) cudaEventRecord(ov->ev_halo0, ov->aux);                       \
            k_halo_gather<SP><<<ov->gather_grid, 256, 0, ov->aux>>>(                        \
                GSPH_PAIR_ARGS, (typename Types<SP>::Pos *)ov->hpos,                        \
                (typename Types<SP>::Rec *)ov->hrec, ov->hcx);                              \
            if (ov->ev_halo1) cudaEventRecord(ov->ev_halo1, ov->aux);                       \
            cudaEventRecord(ov->ev_join, ov->aux);                                          \
            GSPH_PAIRS(PM_LOCAL);                                                           \
            if (ov->ev_local) cudaEventRecord(ov->ev_local, s);                             \
            cudaStreamWaitEvent(s, ov->ev_join, 0);                                         \
            GSPH_PAIRS(PM_BOUNDARY);                                                        \
        }                                                                                   \
    } while (0)
    if (split) {
        constexpr bool SP = true;
        GSPH_INTERACT;
    } else {
        constexpr bool SP = false;
        GSPH_INTERACT;
    }
#undef GSPH_INTERACT
#undef GSPH_PAIRS
#undef GSPH_PAIR_ARGS
    return cudaGetLastError();
}

}  // namespace gsph
