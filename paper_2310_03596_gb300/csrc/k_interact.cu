// k_interact.cu - the interaction loop (Sec. II step f) fused with the integration (step g).
//
// One lane per sorted particle i. The 27 buckets around i are visited as 9 rows of 3 buckets that
// are contiguous in hash order. Phase 1 tests candidates and appends the in-support ones to a per-lane
// list in shared memory (column-major, conflict-free); phase 2 evaluates the pair fluxes of the listed
// neighbours in lockstep, so the heavy pair math runs with every lane busy instead of at the ~17% hit
// rate of the raw candidate stream. Wall images (mirror planes) are searched around the mirrored point
// with the same two phases.
//
// Pair formulation (reading of the Gamma-SPH-ALE interface state; the paper cites it from another
// work): transport velocity v0 = v; acoustic Riemann problem on the pair normal n (L = lower sorted
// slot, n from L to R); interface velocity v_E = mean v + (u* - mean u) n, density and energy means,
// traction t* n plus the averaged tangential traction; Wendland C2 gradient |dW/dr| n.
//
// Split path: pair math in FP32 from FP32 records (positions relative to each particle's bucket corner,
// so differences keep ~2^-24 * 2h), FP32 Kahan-compensated per-particle sums, FP64 integration. The
// support predicate stays exact: the FP32 r^2 decides only outside a band of relative width 1.2e-5
// around (2h)^2, inside which the FP64 positions decide with the same rounding as FP64 code.
#include <type_traits>

#include "gsph_internal.cuh"

namespace gsph {

constexpr int IT_THREADS = 128;
constexpr int IT_CAP = 48;                 // list entries per lane before a flush
constexpr uint32_t IT_JMASK = (1u << 27) - 1;

template <class R> struct PIn { R vx, vy, vz, rho, p, Z, E, sxx, syy, szz, sxy, sxz, syz, w; };

__device__ __forceinline__ PIn<float> load_rec(const RecF *__restrict__ rec, float w, int64_t j) {
    RecF r;
    r.a = __ldg(&rec[j].a);
    r.b = __ldg(&rec[j].b);
    r.c = __ldg(&rec[j].c);
    PIn<float> q;
    q.vx = r.a.x; q.vy = r.a.y; q.vz = r.a.z; q.rho = r.a.w;
    q.p = r.b.x; q.Z = r.b.y; q.E = r.b.z; q.sxx = r.b.w;
    q.syy = r.c.x; q.szz = -(r.b.w + r.c.x); q.sxy = r.c.y; q.sxz = r.c.z; q.syz = r.c.w;
    q.w = w;
    return q;
}
__device__ __forceinline__ PIn<double> load_rec(const RecD *__restrict__ rec, double w, int64_t j) {
    PIn<double> q;
    const D4 a = rec[j].a, b = rec[j].b, c = rec[j].c, d = rec[j].d;
    q.vx = a.x; q.vy = a.y; q.vz = a.z; q.rho = a.w;
    q.p = b.x; q.Z = b.y; q.E = b.z; q.sxx = b.w;
    q.syy = c.x; q.szz = c.y; q.sxy = c.z; q.sxz = c.w; q.syz = d.x;
    q.w = w;
    return q;
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

template <class R> struct PairRes { R Fm, Fmv[3], Fe, a, n[3], uL, uR; };

// Pair fluxes with L = left state, R = right state, d = x_R - x_L.
template <class R>
__device__ __forceinline__ void pair_terms(R d0, R d1, R d2, const PIn<R> &L, const PIn<R> &Rr, R inv_h, R kdw,
                                           PairRes<R> &o) {
    const R half = R(0.5);
    R r2 = d0 * d0 + d1 * d1 + d2 * d2;
    R inv_r = rsqrt_r(r2);
    R r = r2 * inv_r;
    R n0 = d0 * inv_r, n1 = d1 * inv_r, n2 = d2 * inv_r;
    R q = r * inv_h;
    R sq = R(1) - half * q;
    R a = kdw * q * sq * sq * sq;
    R uL = L.vx * n0 + L.vy * n1 + L.vz * n2;
    R uR = Rr.vx * n0 + Rr.vy * n1 + Rr.vz * n2;
    R sL0 = L.sxx * n0 + L.sxy * n1 + L.sxz * n2 - L.p * n0;
    R sL1 = L.sxy * n0 + L.syy * n1 + L.syz * n2 - L.p * n1;
    R sL2 = L.sxz * n0 + L.syz * n1 + L.szz * n2 - L.p * n2;
    R sR0 = Rr.sxx * n0 + Rr.sxy * n1 + Rr.sxz * n2 - Rr.p * n0;
    R sR1 = Rr.sxy * n0 + Rr.syy * n1 + Rr.syz * n2 - Rr.p * n1;
    R sR2 = Rr.sxz * n0 + Rr.syz * n1 + Rr.szz * n2 - Rr.p * n2;
    R tL = sL0 * n0 + sL1 * n1 + sL2 * n2;
    R tR = sR0 * n0 + sR1 * n1 + sR2 * n2;
    R izs = rcp_r(L.Z + Rr.Z);
    R us = (L.Z * uL + Rr.Z * uR + (tR - tL)) * izs;
    R ts = (Rr.Z * tL + L.Z * tR + L.Z * Rr.Z * (uR - uL)) * izs;
    R du = us - half * (uL + uR);
    R rhoE = half * (L.rho + Rr.rho);
    R EE = half * (L.E + Rr.E);
    R tm = half * (tL + tR);
    R vE0 = half * (L.vx + Rr.vx) + du * n0;
    R vE1 = half * (L.vy + Rr.vy) + du * n1;
    R vE2 = half * (L.vz + Rr.vz) + du * n2;
    R TE0 = ts * n0 + (half * (sL0 + sR0) - tm * n0);
    R TE1 = ts * n1 + (half * (sL1 + sR1) - tm * n1);
    R TE2 = ts * n2 + (half * (sL2 + sR2) - tm * n2);
    R wwa = R(2) * L.w * Rr.w * a;
    R mf = rhoE * du;
    o.Fm = wwa * mf;
    o.Fmv[0] = wwa * (mf * vE0 - TE0);
    o.Fmv[1] = wwa * (mf * vE1 - TE1);
    o.Fmv[2] = wwa * (mf * vE2 - TE2);
    o.Fe = wwa * (mf * EE - (TE0 * vE0 + TE1 * vE1 + TE2 * vE2));
    o.a = a;
    o.n[0] = n0; o.n[1] = n1; o.n[2] = n2;
    o.uL = uL;
    o.uR = uR;
}

// Per-particle sums: Kahan-compensated in FP32, plain in FP64.
template <class R> struct Acc;
template <> struct Acc<float> {
    float s[kNRate], c[kNRate];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) { s[k] = 0.f; c[k] = 0.f; }
    }
    __device__ __forceinline__ void add(int k, float x) {
        float y = x - c[k];
        float t = s[k] + y;
        c[k] = (t - s[k]) - y;
        s[k] = t;
    }
    __device__ __forceinline__ double get(int k) const { return (double)s[k] - (double)c[k]; }
};
template <> struct Acc<double> {
    double s[kNRate];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < kNRate; ++k) s[k] = 0.0;
    }
    __device__ __forceinline__ void add(int k, double x) { s[k] += x; }
    __device__ __forceinline__ double get(int k) const { return s[k]; }
};

// Adds one pair to the sums of particle i. sg = -1 when i is the left state (n points from i to j),
// +1 when i is the right state; oth = the other particle's state.
template <class R>
__device__ __forceinline__ void accumulate(Acc<R> &acc, const PairRes<R> &o, R sg, const PIn<R> &me,
                                           const PIn<R> &oth) {
    acc.add(0, me.w * oth.w * o.a * (o.uR - o.uL));
    acc.add(1, sg * o.Fm);
    acc.add(2, sg * o.Fmv[0]);
    acc.add(3, sg * o.Fmv[1]);
    acc.add(4, sg * o.Fmv[2]);
    acc.add(5, sg * o.Fe);
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
};

// Search centre of one source (0 = real neighbours, 1.. = images in wall k-1).
struct Centre {
    int bx, by, bz;
    float ox, oy, oz;      // split path: i (or its mirror) relative to the centre bucket corner
    double X, Y, Z;        // FP64 search point (i or its mirror)
};

template <bool SPLIT, bool DIAG>
__global__ void __launch_bounds__(IT_THREADS, SPLIT ? 4 : 2)
k_interact(DevParams P, int64_t n, const uint32_t *__restrict__ skey, const uint2 *__restrict__ cellr,
           const typename Types<SPLIT>::Pos *__restrict__ pos, const typename Types<SPLIT>::Rec *__restrict__ rec,
           const double *__restrict__ xs, const double *__restrict__ ys, const double *__restrict__ zs,
           const uint32_t *__restrict__ perm, State A, State B, const uint8_t *__restrict__ lab_s,
           const uint8_t *__restrict__ mat_s, const uint32_t *__restrict__ id_s, const double *__restrict__ dt_ptr,
           unsigned long long *__restrict__ sig, int32_t *__restrict__ nreal_out, int32_t *__restrict__ nimage_out,
           double *__restrict__ rates_out) {
    using R = typename Types<SPLIT>::R;
    __shared__ uint32_t list[IT_CAP * IT_THREADS];
    const int tid = threadIdx.x;
    const int64_t s = (int64_t)blockIdx.x * IT_THREADS + tid;
    const bool valid = s < n;
    const uint32_t key = valid ? skey[s] : P.ncell;
    const bool active = valid && key < P.ncell;
    int cx = 0, cy = 0, cz = 0;
    if (active) decode_cell(P, key, cx, cy, cz);
    const double X = valid ? xs[s] : 0.0, Y = valid ? ys[s] : 0.0, Z = valid ? zs[s] : 0.0;
    PIn<R> me;
    R mrx = 0, mry = 0, mrz = 0;   // own position: relative (split) or absolute (FP64)
    if (active) {
        auto p = pos[s];
        mrx = p.x; mry = p.y; mrz = p.z;
        me = load_rec(rec, p.w, s);
    } else {
        me = PIn<R>{};
    }
    const R inv_h = SPLIT ? (R)P.f_inv_h : (R)(1.0 / P.h);
    const R kdw = SPLIT ? (R)P.f_kdw : (R)P.kdw;
    const float fcell = P.f_cell;
    Acc<R> acc;
    acc.zero();
    int nr = 0, ni = 0;

    for (int src = 0; src <= P.nwalls; ++src) {
        const int wax = src > 0 ? P.wall_axis[src - 1] : -1;
        const double wpos = src > 0 ? P.wall_pos[src - 1] : 0.0;
        Centre C;
        C.X = X; C.Y = Y; C.Z = Z;
        if (src == 0) {
            C.bx = cx; C.by = cy; C.bz = cz;
            C.ox = (float)mrx; C.oy = (float)mry; C.oz = (float)mrz;
        } else {
            double two_w = __dmul_rn(2.0, wpos);
            if (wax == 0) C.X = __dsub_rn(two_w, X);
            if (wax == 1) C.Y = __dsub_rn(two_w, Y);
            if (wax == 2) C.Z = __dsub_rn(two_w, Z);
            C.bx = bucket_coord_signed(C.X, P.lo[0], P.cell);
            C.by = bucket_coord_signed(C.Y, P.lo[1], P.cell);
            C.bz = bucket_coord_signed(C.Z, P.lo[2], P.cell);
            C.ox = (float)(C.X - (P.lo[0] + (double)C.bx * P.cell));
            C.oy = (float)(C.Y - (P.lo[1] + (double)C.by * P.cell));
            C.oz = (float)(C.Z - (P.lo[2] + (double)C.bz * P.cell));
        }
        bool done = !active;
        int row = -1;
        uint32_t j = 0, jend = 0, s1 = 0, s2 = 0;
        int dcy = 0, dcz = 0;
        int cnt = 0;
        while (__any_sync(kFullMask, !done)) {
            // ---- phase 1: fill the lane lists
            while (true) {
                const bool want = !done && cnt < IT_CAP;
                if (!__any_sync(kFullMask, want)) break;
                if (!want) continue;
                if (j < jend) {
                    const uint32_t jj = j++;
                    if (src == 0 && (int64_t)jj == s) continue;
                    const int dcx = jj < s1 ? -1 : (jj < s2 ? 0 : 1);
                    bool hit;
                    auto pj = pos[jj];
                    if (SPLIT) {
                        float ex = ((float)pj.x - C.ox) + (float)dcx * fcell;
                        float ey = ((float)pj.y - C.oy) + (float)dcy * fcell;
                        float ez = ((float)pj.z - C.oz) + (float)dcz * fcell;
                        float r2 = ex * ex + ey * ey + ez * ez;
                        hit = r2 < P.f_R2lo;
                        if (!hit && r2 < P.f_R2hi) {
                            // inside the rounding band: decide with exactly rounded FP64
                            double qx = xs[jj], qy = ys[jj], qz = zs[jj];
                            double two_w = __dmul_rn(2.0, wpos);
                            if (wax == 0) qx = __dsub_rn(two_w, qx);
                            if (wax == 1) qy = __dsub_rn(two_w, qy);
                            if (wax == 2) qz = __dsub_rn(two_w, qz);
                            hit = dist2_rn(__dsub_rn(qx, X), __dsub_rn(qy, Y), __dsub_rn(qz, Z)) < P.R2;
                        }
                    } else {
                        double qx = (double)pj.x, qy = (double)pj.y, qz = (double)pj.z;
                        double two_w = __dmul_rn(2.0, wpos);
                        if (wax == 0) qx = __dsub_rn(two_w, qx);
                        if (wax == 1) qy = __dsub_rn(two_w, qy);
                        if (wax == 2) qz = __dsub_rn(two_w, qz);
                        hit = dist2_rn(__dsub_rn(qx, X), __dsub_rn(qy, Y), __dsub_rn(qz, Z)) < P.R2;
                    }
                    if (hit) {
                        const uint32_t code = (uint32_t)((dcx + 1) + 3 * (dcy + 1) + 9 * (dcz + 1));
                        list[cnt * IT_THREADS + tid] = jj | (code << 27);
                        ++cnt;
                    }
                } else {
                    ++row;
                    if (row >= 9) {
                        done = true;
                        continue;
                    }
                    dcy = row % 3 - 1;
                    dcz = row / 3 - 1;
                    const int Yc = C.by + dcy, Zc = C.bz + dcz;
                    j = jend = s1 = s2 = 0;
                    if (Yc >= 0 && Yc < P.dims[1] && Zc >= 0 && Zc < P.dims[2] && C.bx >= -1 && C.bx <= P.dims[0]) {
                        const uint32_t rb = (uint32_t)P.dims[0] * ((uint32_t)Yc + (uint32_t)P.dims[1] * (uint32_t)Zc);
                        uint2 cm = make_uint2(0, 0), c0 = make_uint2(0, 0), cp = make_uint2(0, 0);
                        if (C.bx - 1 >= 0 && C.bx - 1 < P.dims[0]) cm = __ldg(&cellr[rb + C.bx - 1]);
                        if (C.bx >= 0 && C.bx < P.dims[0]) c0 = __ldg(&cellr[rb + C.bx]);
                        if (C.bx + 1 >= 0 && C.bx + 1 < P.dims[0]) cp = __ldg(&cellr[rb + C.bx + 1]);
                        const bool em = cm.y > cm.x, e0 = c0.y > c0.x, ep = cp.y > cp.x;
                        if (em || e0 || ep) {
                            uint32_t lo = em ? cm.x : (e0 ? c0.x : cp.x);
                            uint32_t hi = ep ? cp.y : (e0 ? c0.y : cm.y);
                            s1 = em ? cm.y : lo;
                            s2 = ep ? cp.x : hi;
                            j = lo;
                            jend = hi;
                        }
                    }
                }
            }
            // ---- phase 2: pair fluxes of the listed neighbours
            const int mc = __reduce_max_sync(kFullMask, cnt);
            for (int k = 0; k < mc; ++k) {
                if (k >= cnt) continue;
                const uint32_t e = list[k * IT_THREADS + tid];
                const uint32_t jj = e & IT_JMASK;
                const uint32_t code = e >> 27;
                const int ex = (int)(code % 3u) - 1, ey = (int)((code / 3u) % 3u) - 1, ez = (int)(code / 9u) - 1;
                auto pj = pos[jj];
                PIn<R> oth = load_rec(rec, (R)pj.w, jj);
                PairRes<R> o;
                if (src == 0) {
                    const bool iL = s < (int64_t)jj;
                    R d0, d1, d2;
                    if (SPLIT) {
                        // canonical difference x_R - x_L = (r_R - r_L) + (c_R - c_L) 2h: both ends of
                        // the pair evaluate the same operands in the same order
                        if (iL) {
                            d0 = ((R)pj.x - mrx) + (R)ex * (R)fcell;
                            d1 = ((R)pj.y - mry) + (R)ey * (R)fcell;
                            d2 = ((R)pj.z - mrz) + (R)ez * (R)fcell;
                        } else {
                            d0 = (mrx - (R)pj.x) + (R)(-ex) * (R)fcell;
                            d1 = (mry - (R)pj.y) + (R)(-ey) * (R)fcell;
                            d2 = (mrz - (R)pj.z) + (R)(-ez) * (R)fcell;
                        }
                    } else {
                        if (iL) { d0 = (R)pj.x - mrx; d1 = (R)pj.y - mry; d2 = (R)pj.z - mrz; }
                        else { d0 = mrx - (R)pj.x; d1 = mry - (R)pj.y; d2 = mrz - (R)pj.z; }
                    }
                    if (iL) pair_terms<R>(d0, d1, d2, me, oth, inv_h, kdw, o);
                    else pair_terms<R>(d0, d1, d2, oth, me, inv_h, kdw, o);
                    accumulate<R>(acc, o, iL ? R(-1) : R(1), me, oth);
                    ++nr;
                } else {
                    R d0, d1, d2;
                    if (SPLIT) {
                        d0 = ((R)pj.x - (R)C.ox) + (R)ex * (R)fcell;
                        d1 = ((R)pj.y - (R)C.oy) + (R)ey * (R)fcell;
                        d2 = ((R)pj.z - (R)C.oz) + (R)ez * (R)fcell;
                        if (wax == 0) d0 = -d0;
                        if (wax == 1) d1 = -d1;
                        if (wax == 2) d2 = -d2;
                    } else {
                        double qx = (double)pj.x, qy = (double)pj.y, qz = (double)pj.z;
                        double two_w = 2.0 * wpos;
                        if (wax == 0) qx = two_w - qx;
                        if (wax == 1) qy = two_w - qy;
                        if (wax == 2) qz = two_w - qz;
                        d0 = (R)(qx - X); d1 = (R)(qy - Y); d2 = (R)(qz - Z);
                    }
                    mirror<R>(oth, wax);
                    pair_terms<R>(d0, d1, d2, me, oth, inv_h, kdw, o);
                    accumulate<R>(acc, o, R(-1), me, oth);
                    ++ni;
                }
            }
            cnt = 0;
        }
    }

    // ---- integration (Sec. II step g): forward Euler on the conserved variables, Jaumann-rate
    // stress with radial return, positions with the velocity of the step's start.
    double sp = 0.0;
    if (valid) {
    double r[kNRate];
#pragma unroll
    for (int k = 0; k < kNRate; ++k) r[k] = acc.get(k);
    const uint32_t o = perm[s];
    const int mt = mat_s[s] < P.nmat ? mat_s[s] : 0;
    const double dt = *dt_ptr;
    const double w = A.f[FW][o], m = A.f[FM][o], E = A.f[FE][o];
    const double vx = A.f[FVX][o], vy = A.f[FVY][o], vz = A.f[FVZ][o];
    double S[3][3];
    S[0][0] = A.f[FSXX][o]; S[1][1] = A.f[FSYY][o]; S[2][2] = A.f[FSZZ][o];
    S[0][1] = S[1][0] = A.f[FSXY][o];
    S[0][2] = S[2][0] = A.f[FSXZ][o];
    S[1][2] = S[2][1] = A.f[FSYZ][o];
    const double wn = w + dt * r[0];
    const double mn = m + dt * r[1];
    const double mvx = m * vx + dt * (r[2] + m * P.g[0]);
    const double mvy = m * vy + dt * (r[3] + m * P.g[1]);
    const double mvz = m * vz + dt * (r[4] + m * P.g[2]);
    const double gv = P.g[0] * vx + P.g[1] * vy + P.g[2] * vz;
    const double mE = m * E + dt * (r[5] + m * gv);
    double Lm[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) Lm[u][v] = r[6 + 3 * u + v];
    const double trD = Lm[0][0] + Lm[1][1] + Lm[2][2];
    const double G2 = 2.0 * P.G[mt];
    double Sn[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = u; v < 3; ++v) {
            double D = 0.5 * (Lm[u][v] + Lm[v][u]);
            if (u == v) D -= trD / 3.0;
            double rot = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double Ouk = 0.5 * (Lm[u][k] - Lm[k][u]);
                double Okv = 0.5 * (Lm[k][v] - Lm[v][k]);
                rot += Ouk * S[k][v] - S[u][k] * Okv;
            }
            Sn[u][v] = S[u][v] + dt * (G2 * D + rot);
        }
    const double trS = (Sn[0][0] + Sn[1][1] + Sn[2][2]) / 3.0;
    Sn[0][0] -= trS; Sn[1][1] -= trS; Sn[2][2] -= trS;
    const double ss = Sn[0][0] * Sn[0][0] + Sn[1][1] * Sn[1][1] + Sn[2][2] * Sn[2][2] +
                      2.0 * (Sn[0][1] * Sn[0][1] + Sn[0][2] * Sn[0][2] + Sn[1][2] * Sn[1][2]);
    const double seq = sqrt(1.5 * ss);
    if (seq > P.Y[mt]) {
        const double f = P.Y[mt] / seq;
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = u; v < 3; ++v) Sn[u][v] *= f;
    }
    const double inv_mn = 1.0 / mn;
    const double nvx = mvx * inv_mn, nvy = mvy * inv_mn, nvz = mvz * inv_mn;
    B.f[FX][s] = X + dt * vx;
    B.f[FY][s] = Y + dt * vy;
    B.f[FZ][s] = Z + dt * vz;
    B.f[FVX][s] = nvx;
    B.f[FVY][s] = nvy;
    B.f[FVZ][s] = nvz;
    B.f[FW][s] = wn;
    B.f[FM][s] = mn;
    B.f[FE][s] = mE * inv_mn;
    B.f[FSXX][s] = Sn[0][0];
    B.f[FSYY][s] = Sn[1][1];
    B.f[FSZZ][s] = Sn[2][2];
    B.f[FSXY][s] = Sn[0][1];
    B.f[FSXZ][s] = Sn[0][2];
    B.f[FSYZ][s] = Sn[1][2];
    B.mat[s] = mat_s[s];
    B.label[s] = lab_s[s];
    B.id[s] = id_s[s];
    if (DIAG) {
        nreal_out[s] = nr;
        nimage_out[s] = ni;
#pragma unroll
        for (int k = 0; k < kNRate; ++k) rates_out[(size_t)s * kNRate + k] = r[k];
    }
    // next step's CFL signal speed, exactly rounded
    sp = signal_speed(P, mt, mn, wn, nvx, nvy, nvz);
    }
    unsigned long long b = __double_as_longlong(sp);
    for (int o2 = 16; o2; o2 >>= 1) {
        unsigned long long c2 = __shfl_xor_sync(kFullMask, b, o2);
        b = c2 > b ? c2 : b;
    }
    if ((tid & 31) == 0) atomicMax(sig, b);
}

cudaError_t launch_interact(bool split, bool diag, const DevParams &P, int64_t n, const uint32_t *skey,
                            const uint2 *cellr, const void *pos, const void *rec, const double *xs, const double *ys,
                            const double *zs, const uint32_t *perm, const State &A, const State &B,
                            const uint8_t *lab_s, const uint8_t *mat_s, const uint32_t *id_s, const double *dt,
                            unsigned long long *sig, int32_t *nreal, int32_t *nimage, double *rates, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    unsigned g = (unsigned)((n + IT_THREADS - 1) / IT_THREADS);
#define GSPH_IT_ARGS P, n, skey, cellr, (const typename Types<SP>::Pos *)pos, (const typename Types<SP>::Rec *)rec, \
                     xs, ys, zs, perm, A, B, lab_s, mat_s, id_s, dt, sig, nreal, nimage, rates
    if (split) {
        constexpr bool SP = true;
        if (diag) k_interact<SP, true><<<g, IT_THREADS, 0, s>>>(GSPH_IT_ARGS);
        else k_interact<SP, false><<<g, IT_THREADS, 0, s>>>(GSPH_IT_ARGS);
    } else {
        constexpr bool SP = false;
        if (diag) k_interact<SP, true><<<g, IT_THREADS, 0, s>>>(GSPH_IT_ARGS);
        else k_interact<SP, false><<<g, IT_THREADS, 0, s>>>(GSPH_IT_ARGS);
    }
#undef GSPH_IT_ARGS
    return cudaGetLastError();
}

}  // namespace gsph
