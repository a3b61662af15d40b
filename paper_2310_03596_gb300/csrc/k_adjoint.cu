// k_adjoint.cu - hand-written adjoint (reverse mode) of one step: the interaction loop (Sec. II step
// f) and the integration (step g), in FP64, with the step's neighbour set and time step held fixed.
//
// Given lam_next = dJ/dy_{n+1} (15 fields per particle in the sorted order of step n, which is the slot
// order of y_{n+1}), one adjoint step returns lam_prev = dJ/dy_n (in the slot order of y_n) and the
// step's contributions to dJ/dY and dJ/dG of material 0:
//   k_adj_integrate  per particle: the transpose of the integration map y_{n+1} = Phi(y_n, r_n) with
//                    respect to the state (direct part of lam_prev) and to the rates (mu = dJ/dr_n),
//                    and the yield-stress and shear-modulus terms of the stress update;
//   k_adj_pair       per particle k: for every pair (k, i) the reverse sweep of the pair function,
//                    fed by the rate adjoints of both ends (k's own term and i's term both depend on
//                    k's state), keeping the part that lands on k's inputs; wall images in both
//                    orientations (k with j's image, j with k's image); then the chain through
//                    rho = m/w, p = K (rho/rho0 - 1), Z = sqrt((K + 4G/3) rho) to the state.
// Each pair is swept at both of its ends (gather form: no atomics, deterministic sums).
#include "gsph_internal.cuh"

namespace gsph {

namespace {

struct Prim64 {
    double v[3], rho, p, Z, E, w;
    double S[6];  // xx yy zz xy xz yz
};

__device__ __forceinline__ int sidx(int a, int b) {
    // symmetric-matrix element (a, b) -> stored component
    if (a == b) return a;
    const int s = a + b;  // 1: xy, 2: xz, 3: yz
    return s == 1 ? 3 : (s == 2 ? 4 : 5);
}

__device__ __forceinline__ Prim64 prim_of(const RecD &r, double w) {
    Prim64 q;
    q.v[0] = r.a.x; q.v[1] = r.a.y; q.v[2] = r.a.z; q.rho = r.a.w;
    q.p = r.b.x; q.Z = r.b.y; q.E = r.b.z; q.S[0] = r.b.w;
    q.S[1] = r.c.x; q.S[2] = r.c.y; q.S[3] = r.c.z; q.S[4] = r.c.w; q.S[5] = r.d.x;
    q.w = w;
    return q;
}

__device__ __forceinline__ void mirror64(Prim64 &q, int ax) {
    q.v[ax] = -q.v[ax];
    if (ax == 0) { q.S[3] = -q.S[3]; q.S[4] = -q.S[4]; }
    if (ax == 1) { q.S[3] = -q.S[3]; q.S[5] = -q.S[5]; }
    if (ax == 2) { q.S[4] = -q.S[4]; q.S[5] = -q.S[5]; }
}

// Bars of one side's primitive inputs.
struct PBar {
    double v[3], rho, p, Z, E, w, S[6];
    __device__ __forceinline__ void zero() {
        for (int c = 0; c < 3; ++c) v[c] = 0.0;
        rho = p = Z = E = w = 0.0;
        for (int c = 0; c < 6; ++c) S[c] = 0.0;
    }
};

// Output bars of one pair evaluation.
struct OutBar {
    double Fm, Fmv[3], Fe, V;   // V: the volume-rate pair value w_L w_R a (u_R - u_L)
    double a, n[3];             // extra bars on |dW/dr| and on n (from the velocity-gradient terms)
};

// Forward values of the pair needed by the velocity-gradient terms.
struct PairFwd {
    double a, n[3];
};

// Forward pair function (same formulas as the forward kernels, FP64) followed by its reverse sweep.
// d = x_R - x_L. Returns the bars of L's and R's primitive inputs and of d.
__device__ void pair_reverse(const double d[3], const Prim64 &L, const Prim64 &R, double ih, double kdw,
                             const OutBar &ob, PBar &bL, PBar &bR, double dbar[3]) {
    // ---- forward
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double r = sqrt(r2);
    const double ir = 1.0 / r;
    double n[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    const double q = r * ih;
    const double sq = 1.0 - 0.5 * q;
    const double a = kdw * q * sq * sq * sq;
    const double uL = L.v[0] * n[0] + L.v[1] * n[1] + L.v[2] * n[2];
    const double uR = R.v[0] * n[0] + R.v[1] * n[1] + R.v[2] * n[2];
    double sL[3], sR[3];
    for (int c = 0; c < 3; ++c) {
        sL[c] = L.S[sidx(c, 0)] * n[0] + L.S[sidx(c, 1)] * n[1] + L.S[sidx(c, 2)] * n[2] - L.p * n[c];
        sR[c] = R.S[sidx(c, 0)] * n[0] + R.S[sidx(c, 1)] * n[1] + R.S[sidx(c, 2)] * n[2] - R.p * n[c];
    }
    const double tL = sL[0] * n[0] + sL[1] * n[1] + sL[2] * n[2];
    const double tR = sR[0] * n[0] + sR[1] * n[1] + sR[2] * n[2];
    const double zs = L.Z + R.Z;
    const double izs = 1.0 / zs;
    const double A1 = L.Z * uL + R.Z * uR + (tR - tL);
    const double us = A1 * izs;
    const double dur = uR - uL;
    const double A2 = R.Z * tL + L.Z * tR + L.Z * R.Z * dur;
    const double ts = A2 * izs;
    const double du = us - 0.5 * (uL + uR);
    const double rhoE = 0.5 * (L.rho + R.rho);
    const double EE = 0.5 * (L.E + R.E);
    const double tm = 0.5 * (tL + tR);
    double vE[3], TE[3], P[3];
    for (int c = 0; c < 3; ++c) {
        vE[c] = 0.5 * (L.v[c] + R.v[c]) + du * n[c];
        TE[c] = ts * n[c] + (0.5 * (sL[c] + sR[c]) - tm * n[c]);
    }
    const double ww = 2.0 * L.w * R.w;
    const double wwa = ww * a;
    const double mf = rhoE * du;
    for (int c = 0; c < 3; ++c) P[c] = mf * vE[c] - TE[c];
    const double tv = TE[0] * vE[0] + TE[1] * vE[1] + TE[2] * vE[2];
    const double Q = mf * EE - tv;

    // ---- reverse
    double abar = ob.a, nbar[3] = {ob.n[0], ob.n[1], ob.n[2]};
    double uLb = 0.0, uRb = 0.0, tLb = 0.0, tRb = 0.0;
    double sLb[3] = {0, 0, 0}, sRb[3] = {0, 0, 0};
    // V = wL wR a (uR - uL)
    bL.w += ob.V * R.w * a * dur;
    bR.w += ob.V * L.w * a * dur;
    abar += ob.V * L.w * R.w * dur;
    uRb += ob.V * L.w * R.w * a;
    uLb -= ob.V * L.w * R.w * a;
    // fluxes
    double wwab = ob.Fe * Q + ob.Fm * mf;
    double Pb[3];
    for (int c = 0; c < 3; ++c) {
        wwab += ob.Fmv[c] * P[c];
        Pb[c] = ob.Fmv[c] * wwa;
    }
    const double Qb = ob.Fe * wwa;
    double mfb = ob.Fm * wwa + Qb * EE;
    for (int c = 0; c < 3; ++c) mfb += Pb[c] * vE[c];
    const double EEb = Qb * mf;
    const double tvb = -Qb;
    double TEb[3], vEb[3];
    for (int c = 0; c < 3; ++c) {
        TEb[c] = tvb * vE[c] - Pb[c];
        vEb[c] = tvb * TE[c] + Pb[c] * mf;
    }
    const double rhoEb = mfb * du;
    double dub = mfb * rhoE;
    const double wwb = wwab * a;
    abar += wwab * ww;
    bL.w += 2.0 * wwb * R.w;
    bR.w += 2.0 * wwb * L.w;
    // TE_c = ts n_c + 0.5 (sL_c + sR_c) - tm n_c
    double tsb = 0.0, tmb = 0.0;
    for (int c = 0; c < 3; ++c) {
        tsb += TEb[c] * n[c];
        tmb -= TEb[c] * n[c];
        nbar[c] += TEb[c] * (ts - tm);
        sLb[c] += 0.5 * TEb[c];
        sRb[c] += 0.5 * TEb[c];
    }
    // vE_c = 0.5 (vL_c + vR_c) + du n_c
    for (int c = 0; c < 3; ++c) {
        bL.v[c] += 0.5 * vEb[c];
        bR.v[c] += 0.5 * vEb[c];
        dub += vEb[c] * n[c];
        nbar[c] += vEb[c] * du;
    }
    tLb += 0.5 * tmb;
    tRb += 0.5 * tmb;
    bL.E += 0.5 * EEb;
    bR.E += 0.5 * EEb;
    bL.rho += 0.5 * rhoEb;
    bR.rho += 0.5 * rhoEb;
    // du = us - 0.5 (uL + uR)
    const double usb = dub;
    uLb -= 0.5 * dub;
    uRb -= 0.5 * dub;
    // us = A1 izs, ts = A2 izs
    const double A1b = usb * izs, A2b = tsb * izs;
    const double izsb = usb * A1 + tsb * A2;
    const double zsb = -izsb * izs * izs;
    bL.Z += zsb;
    bR.Z += zsb;
    // A2 = ZR tL + ZL tR + ZL ZR (uR - uL)
    bR.Z += A2b * (tL + L.Z * dur);
    bL.Z += A2b * (tR + R.Z * dur);
    tLb += A2b * R.Z;
    tRb += A2b * L.Z;
    uRb += A2b * L.Z * R.Z;
    uLb -= A2b * L.Z * R.Z;
    // A1 = ZL uL + ZR uR + tR - tL
    bL.Z += A1b * uL;
    bR.Z += A1b * uR;
    uLb += A1b * L.Z;
    uRb += A1b * R.Z;
    tRb += A1b;
    tLb -= A1b;
    // tL = sL . n, tR = sR . n
    for (int c = 0; c < 3; ++c) {
        sLb[c] += tLb * n[c];
        sRb[c] += tRb * n[c];
        nbar[c] += tLb * sL[c] + tRb * sR[c];
    }
    // sL_c = sum_b SL_cb n_b - pL n_c (and R)
    for (int c = 0; c < 3; ++c) {
        for (int b = 0; b < 3; ++b) {
            bL.S[sidx(c, b)] += sLb[c] * n[b];
            bR.S[sidx(c, b)] += sRb[c] * n[b];
            nbar[b] += sLb[c] * L.S[sidx(c, b)] + sRb[c] * R.S[sidx(c, b)];
        }
        bL.p -= sLb[c] * n[c];
        bR.p -= sRb[c] * n[c];
        nbar[c] -= sLb[c] * L.p + sRb[c] * R.p;
    }
    // uL = vL . n, uR = vR . n
    for (int c = 0; c < 3; ++c) {
        bL.v[c] += uLb * n[c];
        bR.v[c] += uRb * n[c];
        nbar[c] += uLb * L.v[c] + uRb * R.v[c];
    }
    // a = kdw q sq^3, sq = 1 - q / 2, q = r / h
    double qb = abar * kdw * sq * sq * sq;
    const double sqb = abar * kdw * q * 3.0 * sq * sq;
    qb -= 0.5 * sqb;
    double rb = qb * ih;
    // n = d / r
    double irb = 0.0;
    for (int c = 0; c < 3; ++c) {
        dbar[c] = nbar[c] * ir;
        irb += nbar[c] * d[c];
    }
    rb -= irb * ir * ir;
    // r = sqrt(r2)
    const double r2b = rb / (2.0 * r);
    for (int c = 0; c < 3; ++c) dbar[c] += 2.0 * r2b * d[c];
}

__device__ __forceinline__ void pair_fwd_an(const double d[3], double ih, double kdw, PairFwd &f) {
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double q = r * ih;
    const double sq = 1.0 - 0.5 * q;
    f.a = kdw * q * sq * sq * sq;
    for (int c = 0; c < 3; ++c) f.n[c] = d[c] / r;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Adjoint of the integration (per sorted particle s; old slot o = perm[s]).
// lam_next, lam_dir, mu: field-major arrays [15][n] in sorted order. part: per-block (dJ/dY, dJ/dG).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_integrate(DevParams P, int64_t n, const uint32_t *__restrict__ perm,
                                                       State A, const uint8_t *__restrict__ mat_s,
                                                       const double *__restrict__ rates, double dt,
                                                       const double *__restrict__ lam_next,
                                                       double *__restrict__ lam_dir, double *__restrict__ mu,
                                                       double *__restrict__ part) {
    __shared__ double red[2][128];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double Ybar = 0.0, Gbar = 0.0;
    if (s < n) {
        const uint32_t o = perm[s];
        const int mt = mat_s[s] < P.nmat ? mat_s[s] : 0;
        const double G = P.G[mt], Yv = P.Y[mt];
        const double w = A.f[FW][o], m = A.f[FM][o], E = A.f[FE][o];
        const double v[3] = {A.f[FVX][o], A.f[FVY][o], A.f[FVZ][o]};
        double S[6];
        for (int q = 0; q < 6; ++q) S[q] = A.f[FSXX + q][o];
        double r[kNRate];
        for (int k = 0; k < kNRate; ++k) r[k] = rates[(size_t)s * kNRate + k];
        double lb[15];
        for (int f = 0; f < 15; ++f) lb[f] = lam_next[(size_t)f * n + s];
        // ---- forward recompute
        const double mn = m + dt * r[1];
        double mv[3];
        for (int c = 0; c < 3; ++c) mv[c] = m * v[c] + dt * (r[2 + c] + m * P.g[c]);
        const double gv = P.g[0] * v[0] + P.g[1] * v[1] + P.g[2] * v[2];
        const double mE = m * E + dt * (r[5] + m * gv);
        double Lm[3][3];
        for (int u = 0; u < 3; ++u)
            for (int vv = 0; vv < 3; ++vv) Lm[u][vv] = r[6 + 3 * u + vv];
        const double trD = Lm[0][0] + Lm[1][1] + Lm[2][2];
        double Om[3][3], Dq[6], T[6];
        for (int u = 0; u < 3; ++u)
            for (int vv = 0; vv < 3; ++vv) Om[u][vv] = 0.5 * (Lm[u][vv] - Lm[vv][u]);
        const int iu[6] = {0, 1, 2, 0, 0, 1}, iv[6] = {0, 1, 2, 1, 2, 2};
        for (int q = 0; q < 6; ++q) {
            const int u = iu[q], vv = iv[q];
            double D = 0.5 * (Lm[u][vv] + Lm[vv][u]);
            if (u == vv) D -= trD / 3.0;
            Dq[q] = D;
            double rot = 0.0;
            for (int k = 0; k < 3; ++k) rot += Om[u][k] * S[sidx(k, vv)] - S[sidx(u, k)] * Om[k][vv];
            T[q] = S[q] + dt * (2.0 * G * D + rot);
        }
        const double trS = (T[0] + T[1] + T[2]) / 3.0;
        double Tp[6];
        for (int q = 0; q < 6; ++q) Tp[q] = q < 3 ? T[q] - trS : T[q];
        const double ss = Tp[0] * Tp[0] + Tp[1] * Tp[1] + Tp[2] * Tp[2] +
                          2.0 * (Tp[3] * Tp[3] + Tp[4] * Tp[4] + Tp[5] * Tp[5]);
        const double seq = sqrt(1.5 * ss);
        const bool yield = seq > Yv;
        const double inv = 1.0 / mn;
        // ---- reverse
        double xb[3], vb[3], wb, mb, Eb, Sb[6], rb[kNRate];
        for (int k = 0; k < kNRate; ++k) rb[k] = 0.0;
        for (int c = 0; c < 3; ++c) {
            xb[c] = lb[FX + c];
            vb[c] = dt * lb[FX + c];
        }
        double invb = lb[FE] * mE;
        double mvb[3];
        for (int c = 0; c < 3; ++c) {
            mvb[c] = lb[FVX + c] * inv;
            invb += lb[FVX + c] * mv[c];
        }
        const double mEb = lb[FE] * inv;
        double mnb = lb[FM] - invb * inv * inv;
        wb = lb[FW];
        rb[0] = dt * lb[FW];
        mb = mnb;
        rb[1] = dt * mnb;
        for (int c = 0; c < 3; ++c) {
            mb += mvb[c] * (v[c] + dt * P.g[c]);
            vb[c] += mvb[c] * m;
            rb[2 + c] = dt * mvb[c];
        }
        mb += mEb * (E + dt * gv);
        Eb = mEb * m;
        rb[5] = dt * mEb;
        for (int c = 0; c < 3; ++c) vb[c] += mEb * dt * m * P.g[c];
        // stress: radial return, trace removal, trial update
        double Tpb[6];
        if (yield) {
            const double f = Yv / seq;
            double Asum = 0.0;
            for (int q = 0; q < 6; ++q) {
                Tpb[q] = lb[FSXX + q] * f;
                Asum += lb[FSXX + q] * Tp[q];
            }
            Ybar += Asum / seq;
            const double seqb = -Asum * Yv / (seq * seq);
            const double ssb = 0.75 * seqb / seq;
            for (int q = 0; q < 6; ++q) Tpb[q] += ssb * (q < 3 ? 2.0 : 4.0) * Tp[q];
        } else {
            for (int q = 0; q < 6; ++q) Tpb[q] = lb[FSXX + q];
        }
        double Tb[6];
        const double mean_b = (Tpb[0] + Tpb[1] + Tpb[2]) / 3.0;
        for (int q = 0; q < 6; ++q) Tb[q] = q < 3 ? Tpb[q] - mean_b : Tpb[q];
        for (int q = 0; q < 6; ++q) Sb[q] = Tb[q];
        double Lb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double Omb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double trDb = 0.0;
        for (int q = 0; q < 6; ++q) {
            const int u = iu[q], vv = iv[q];
            Gbar += Tb[q] * dt * 2.0 * Dq[q];
            const double Db = Tb[q] * dt * 2.0 * G;
            const double rotb = Tb[q] * dt;
            Lb[u][vv] += 0.5 * Db;
            Lb[vv][u] += 0.5 * Db;
            if (u == vv) trDb -= Db / 3.0;
            for (int k = 0; k < 3; ++k) {
                Omb[u][k] += rotb * S[sidx(k, vv)];
                Sb[sidx(k, vv)] += rotb * Om[u][k];
                Sb[sidx(u, k)] -= rotb * Om[k][vv];
                Omb[k][vv] -= rotb * S[sidx(u, k)];
            }
        }
        for (int k = 0; k < 3; ++k) Lb[k][k] += trDb;
        for (int u = 0; u < 3; ++u)
            for (int vv = 0; vv < 3; ++vv) {
                Lb[u][vv] += 0.5 * Omb[u][vv];
                Lb[vv][u] -= 0.5 * Omb[u][vv];
            }
        for (int u = 0; u < 3; ++u)
            for (int vv = 0; vv < 3; ++vv) rb[6 + 3 * u + vv] = Lb[u][vv];
        // outputs
        for (int c = 0; c < 3; ++c) {
            lam_dir[(size_t)(FX + c) * n + s] = xb[c];
            lam_dir[(size_t)(FVX + c) * n + s] = vb[c];
        }
        lam_dir[(size_t)FW * n + s] = wb;
        lam_dir[(size_t)FM * n + s] = mb;
        lam_dir[(size_t)FE * n + s] = Eb;
        for (int q = 0; q < 6; ++q) lam_dir[(size_t)(FSXX + q) * n + s] = Sb[q];
        for (int k = 0; k < kNRate; ++k) mu[(size_t)k * n + s] = rb[k];
        if (mt != 0) { Ybar = 0.0; Gbar = 0.0; }
    }
    red[0][threadIdx.x] = Ybar;
    red[1][threadIdx.x] = Gbar;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[0][threadIdx.x] += red[0][threadIdx.x + st];
            red[1][threadIdx.x] += red[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[(size_t)blockIdx.x * 2] = red[0][0];
        part[(size_t)blockIdx.x * 2 + 1] = red[1][0];
    }
}

// ---------------------------------------------------------------------------------------------
// Adjoint of the interaction loop (per sorted particle k), plus the chain to the state and the
// scatter of lam_prev to the slot order of y_n. part: per-block dJ/dG (through Z).
// ---------------------------------------------------------------------------------------------
constexpr uint32_t ADJ_JMASK = (1u << 26) - 1;

// x = c ? a : b, y = c ? b : a, field by field
__device__ __forceinline__ void sel_prim(bool c, const Prim64 &a, const Prim64 &b, Prim64 &x, Prim64 &y) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { x.v[k] = c ? a.v[k] : b.v[k]; y.v[k] = c ? b.v[k] : a.v[k]; }
    x.rho = c ? a.rho : b.rho; y.rho = c ? b.rho : a.rho;
    x.p = c ? a.p : b.p; y.p = c ? b.p : a.p;
    x.Z = c ? a.Z : b.Z; y.Z = c ? b.Z : a.Z;
    x.E = c ? a.E : b.E; y.E = c ? b.E : a.E;
    x.w = c ? a.w : b.w; y.w = c ? b.w : a.w;
#pragma unroll
    for (int k = 0; k < 6; ++k) { x.S[k] = c ? a.S[k] : b.S[k]; y.S[k] = c ? b.S[k] : a.S[k]; }
}
// acc += c ? a : b, field by field
__device__ __forceinline__ void sel_add_bar(PBar &acc, bool c, const PBar &a, const PBar &b) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.v[k] += c ? a.v[k] : b.v[k];
    acc.rho += c ? a.rho : b.rho;
    acc.p += c ? a.p : b.p;
    acc.Z += c ? a.Z : b.Z;
    acc.E += c ? a.E : b.E;
    acc.w += c ? a.w : b.w;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.S[k] += c ? a.S[k] : b.S[k];
}

__device__ __forceinline__ void load_mu(const double *__restrict__ mu, int64_t n, int64_t i, double out[kNRate]) {
    for (int k = 0; k < kNRate; ++k) out[k] = mu[(size_t)k * n + i];
}

__device__ __forceinline__ void add_bar(PBar &acc, const PBar &b) {
    for (int c = 0; c < 3; ++c) acc.v[c] += b.v[c];
    acc.rho += b.rho; acc.p += b.p; acc.Z += b.Z; acc.E += b.E; acc.w += b.w;
    for (int q = 0; q < 6; ++q) acc.S[q] += b.S[q];
}

// Bars on a mirrored copy (mirror plane normal to ax) mapped back onto the original state.
__device__ __forceinline__ void add_bar_mirrored(PBar &acc, const PBar &b, int ax) {
    PBar t = b;
    t.v[ax] = -t.v[ax];
    if (ax == 0) { t.S[3] = -t.S[3]; t.S[4] = -t.S[4]; }
    if (ax == 1) { t.S[3] = -t.S[3]; t.S[5] = -t.S[5]; }
    if (ax == 2) { t.S[4] = -t.S[4]; t.S[5] = -t.S[5]; }
    add_bar(acc, t);
}

// Velocity-gradient part of one pair for the particle whose rates are `mur` (3 x 3 block mur[6..14]):
// L += w_o (v_o - v_self) (x) a n_dir. Adds the bars on v_self (vs), v_o (vo), w_o, a and n_dir.
__device__ __forceinline__ void lgrad_bars(const double mur[kNRate], double w_o, const double vself[3],
                                           const double vo[3], double a, const double ndir[3], double vsb[3],
                                           double vob[3], double &wob, double &ab, double ndb[3]) {
    double dv[3], G[3];
    for (int c = 0; c < 3; ++c) {
        dv[c] = vo[c] - vself[c];
        G[c] = a * ndir[c];
    }
    double dvb[3] = {0, 0, 0}, Gb[3] = {0, 0, 0};
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) {
            const double M = mur[6 + 3 * u + v];
            dvb[u] += w_o * M * G[v];
            Gb[v] += w_o * M * dv[u];
            wob += M * dv[u] * G[v];
        }
    for (int c = 0; c < 3; ++c) {
        vob[c] += dvb[c];
        vsb[c] -= dvb[c];
        ab += Gb[c] * ndir[c];
        ndb[c] += a * Gb[c];
    }
}

__global__ void __launch_bounds__(128) k_adj_pair(DevParams P, int64_t n, const uint32_t *__restrict__ skey,
                                                  const uint2 *__restrict__ cellr, const D4 *__restrict__ pos,
                                                  const RecD *__restrict__ rec, const double *__restrict__ xs,
                                                  const double *__restrict__ ys, const double *__restrict__ zs,
                                                  int kmax, const uint2 *__restrict__ list,
                                                  const uint32_t *__restrict__ cnt_in,
                                                  const uint32_t *__restrict__ perm,
                                                  const uint8_t *__restrict__ mat_s, const double *__restrict__ mu,
                                                  const double *__restrict__ lam_dir, double *__restrict__ lam_prev,
                                                  double *__restrict__ part) {
    __shared__ double red[128];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double Gbar = 0.0;
    if (s < n) {
        const uint32_t key = skey[s];
        const bool active = key < P.ncell;
        const int mt = mat_s[s] < P.nmat ? mat_s[s] : 0;
        const double ih = 1.0 / P.h, kdw = P.kdw;
        const D4 pk = pos[s];
        const Prim64 me = prim_of(rec[s], pk.w);
        double muk[kNRate];
        load_mu(mu, n, s, muk);
        PBar bk;
        bk.zero();
        double xb[3] = {0, 0, 0};
        if (active) {
            // one real pair (k, i): k's own rate term and i's rate term both depend on k's inputs
            auto real_pair = [&](uint32_t i) {
                const D4 pi = pos[i];
                const Prim64 oth = prim_of(rec[i], pi.w);
                double mui[kNRate];
                load_mu(mu, n, i, mui);
                const bool kL = s < (int64_t)i;
                const double sg = kL ? -1.0 : 1.0;   // sign of the flux in k's rates
                const double d[3] = {kL ? pi.x - pk.x : pk.x - pi.x, kL ? pi.y - pk.y : pk.y - pi.y,
                                     kL ? pi.z - pk.z : pk.z - pi.z};
                OutBar ob;
                ob.Fm = sg * (muk[1] - mui[1]);
                for (int c = 0; c < 3; ++c) ob.Fmv[c] = sg * (muk[2 + c] - mui[2 + c]);
                ob.Fe = sg * (muk[5] - mui[5]);
                ob.V = muk[0] + mui[0];
                PairFwd f;
                pair_fwd_an(d, ih, kdw, f);
                const double sn = kL ? 1.0 : -1.0;   // n_ki = sn n
                double nki[3] = {sn * f.n[0], sn * f.n[1], sn * f.n[2]};
                double nkb[3] = {0, 0, 0}, ob_a = 0.0, wib = 0.0, vib[3] = {0, 0, 0};
                // L_k += w_i (v_i - v_k) (x) a n_ki
                lgrad_bars(muk, oth.w, me.v, oth.v, f.a, nki, bk.v, vib, wib, ob_a, nkb);
                // L_i += w_k (v_k - v_i) (x) a n_ik, n_ik = -n_ki
                double nik[3] = {-nki[0], -nki[1], -nki[2]}, nib[3] = {0, 0, 0}, vkb2[3] = {0, 0, 0};
                lgrad_bars(mui, me.w, oth.v, me.v, f.a, nik, vib, vkb2, bk.w, ob_a, nib);
                for (int c = 0; c < 3; ++c) bk.v[c] += vkb2[c];
                ob.a = ob_a;
                for (int c = 0; c < 3; ++c) ob.n[c] = sn * (nkb[c] - nib[c]);
                PBar bL, bR;
                bL.zero();
                bR.zero();
                double db[3];
                // one sweep with the operands in the pair's orientation (selects, so that the lanes of a
                // warp whose pairs have either orientation run it together)
                Prim64 Lq, Rq;
                sel_prim(kL, me, oth, Lq, Rq);
                pair_reverse(d, Lq, Rq, ih, kdw, ob, bL, bR, db);
                sel_add_bar(bk, kL, bL, bR);
                for (int c = 0; c < 3; ++c) xb[c] += kL ? -db[c] : db[c];
            };
            // listed neighbours: the set bits of each entry's mask, slots base + t in ascending order
            // one flat loop over the listed neighbours (the lanes of a warp iterate together; only the
            // entry refill branches), lowest set bit first
            const uint32_t cw = cnt_in[s];
            const uint32_t cnt = cw & 255u;          // entries found (low byte)
            const uint32_t nlist = cw >> 8;          // neighbours in the stored entries
            {
                uint32_t m = 0u, yb = 0u;
                size_t ke = 0;
                for (uint32_t it = 0; it < nlist; ++it) {
                    while (m == 0u) {   // stored entries all have a hit
                        const uint2 e = list[ke * (size_t)n + s];
                        m = e.x;
                        yb = e.y & ADJ_JMASK;
                        ++ke;
                    }
                    const uint32_t t = (uint32_t)(__ffs(m) - 1);
                    m &= m - 1u;
                    real_pair(yb + t);
                }
            }
            // beyond the list capacity, and the wall images: re-scan around the own / mirrored point
            int cx, cy, cz;
            decode_cell(P, key, cx, cy, cz);
            const double X = xs[s], Y = ys[s], Z = zs[s];
            for (int src = (int)cnt > kmax ? 0 : 1; src <= P.nwalls; ++src) {
                const int wax = src > 0 ? P.wall_axis[src - 1] : -1;
                const double wpos = src > 0 ? P.wall_pos[src - 1] : 0.0;
                const double two_w = __dmul_rn(2.0, wpos);
                double C[3] = {X, Y, Z};
                int bx = cx, by = cy, bz = cz;
                if (src > 0) {
                    C[wax] = __dsub_rn(two_w, C[wax]);
                    bx = bucket_coord_signed(C[0], P.lo[0], P.cell);
                    by = bucket_coord_signed(C[1], P.lo[1], P.cell);
                    bz = bucket_coord_signed(C[2], P.lo[2], P.cell);
                }
                uint32_t seen = 0;
                for (int row = 0; row < 9; ++row) {
                    const int Yc = by + row % 3 - 1, Zc = bz + row / 3 - 1;
                    if (Yc < 0 || Yc >= P.dims[1] || Zc < 0 || Zc >= P.dims[2]) continue;
                    const uint32_t rb = (uint32_t)P.dims[0] * ((uint32_t)Yc + (uint32_t)P.dims[1] * (uint32_t)Zc);
                    uint32_t rs = 0xffffffffu, re = 0u;
                    for (int dxc = -1; dxc <= 1; ++dxc) {
                        const int Xc = bx + dxc;
                        if (Xc < 0 || Xc >= P.dims[0]) continue;
                        const uint2 cr = cellr[rb + Xc];
                        if (cr.y > cr.x) {
                            rs = min(rs, cr.x);
                            re = max(re, cr.y);
                        }
                    }
                    for (uint32_t j = rs; j < re; ++j) {
                        if (src == 0 && (int64_t)j == s) continue;
                        double qx = xs[j], qy = ys[j], qz = zs[j];
                        if (wax == 0) qx = __dsub_rn(two_w, qx);
                        if (wax == 1) qy = __dsub_rn(two_w, qy);
                        if (wax == 2) qz = __dsub_rn(two_w, qz);
                        if (!(dist2_rn(__dsub_rn(qx, X), __dsub_rn(qy, Y), __dsub_rn(qz, Z)) < P.R2)) continue;
                        if (src == 0) {
                            if (seen++ < nlist) continue;   // already in the list
                            real_pair(j);
                            continue;
                        }
                        const D4 pj = pos[j];
                        const Prim64 oj = prim_of(rec[j], pj.w);
                        double muj[kNRate];
                        load_mu(mu, n, j, muj);
                        // (k, j'): k is the left state, the image of j the right state; k's rates only
                        {
                            Prim64 jm = oj;
                            mirror64(jm, wax);
                            double xj[3] = {pj.x, pj.y, pj.z};
                            xj[wax] = two_w - xj[wax];
                            const double d[3] = {xj[0] - pk.x, xj[1] - pk.y, xj[2] - pk.z};
                            OutBar ob;
                            ob.Fm = -muk[1];
                            for (int c = 0; c < 3; ++c) ob.Fmv[c] = -muk[2 + c];
                            ob.Fe = -muk[5];
                            ob.V = muk[0];
                            PairFwd f;
                            pair_fwd_an(d, ih, kdw, f);
                            double nb[3] = {0, 0, 0}, ab = 0.0, wjb = 0.0, vjb[3] = {0, 0, 0};
                            lgrad_bars(muk, jm.w, me.v, jm.v, f.a, f.n, bk.v, vjb, wjb, ab, nb);
                            ob.a = ab;
                            for (int c = 0; c < 3; ++c) ob.n[c] = nb[c];
                            PBar bL, bR;
                            bL.zero();
                            bR.zero();
                            double db[3];
                            pair_reverse(d, me, jm, ih, kdw, ob, bL, bR, db);
                            add_bar(bk, bL);
                            for (int c = 0; c < 3; ++c) xb[c] -= db[c];
                        }
                        // (j, k'): j is the left state, the image of k the right state; j's rates only
                        {
                            Prim64 km = me;
                            mirror64(km, wax);
                            double xk[3] = {pk.x, pk.y, pk.z};
                            xk[wax] = two_w - xk[wax];
                            const double d[3] = {xk[0] - pj.x, xk[1] - pj.y, xk[2] - pj.z};
                            OutBar ob;
                            ob.Fm = -muj[1];
                            for (int c = 0; c < 3; ++c) ob.Fmv[c] = -muj[2 + c];
                            ob.Fe = -muj[5];
                            ob.V = muj[0];
                            PairFwd f;
                            pair_fwd_an(d, ih, kdw, f);
                            double nb[3] = {0, 0, 0}, ab = 0.0, vjb[3] = {0, 0, 0};
                            PBar bm;   // bars on k's mirrored state
                            bm.zero();
                            lgrad_bars(muj, km.w, oj.v, km.v, f.a, f.n, vjb, bm.v, bm.w, ab, nb);
                            ob.a = ab;
                            for (int c = 0; c < 3; ++c) ob.n[c] = nb[c];
                            PBar bL, bR;
                            bL.zero();
                            bR.zero();
                            double db[3];
                            pair_reverse(d, oj, km, ih, kdw, ob, bL, bR, db);
                            add_bar(bm, bR);
                            add_bar_mirrored(bk, bm, wax);
                            // x_k' = x_k except x_k'[wax] = 2 w - x_k[wax]
                            for (int c = 0; c < 3; ++c) xb[c] += c == wax ? -db[c] : db[c];
                        }
                    }
                }
            }
        }
        // chain: rho = m / w, p = K (rho / rho0 - 1), Z = sqrt((K + 4G/3) rho)
        const double K = P.K[mt], rho0 = P.rho0[mt];
        const double rho = me.rho, w = me.w;
        const double rhob = bk.rho + bk.p * K / rho0 + (me.Z > 0.0 ? bk.Z * me.Z / (2.0 * rho) : 0.0);
        const double mb = rhob / w;
        const double wb = bk.w - rhob * rho / w;
        if (mt == 0 && me.Z > 0.0) Gbar += bk.Z * (2.0 / 3.0) * rho / me.Z;
        double out[15];
        for (int c = 0; c < 3; ++c) {
            out[FX + c] = xb[c];
            out[FVX + c] = bk.v[c];
        }
        out[FW] = wb;
        out[FM] = mb;
        out[FE] = bk.E;
        for (int q = 0; q < 6; ++q) out[FSXX + q] = bk.S[q];
        const uint32_t o = perm[s];
        for (int f = 0; f < 15; ++f) lam_prev[(size_t)f * n + o] = out[f] + lam_dir[(size_t)f * n + s];
    }
    red[threadIdx.x] = Gbar;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Sums the per-block partials of both kernels in block order (deterministic) into out[0..1].
__global__ void k_adj_reduce(int nb, const double *__restrict__ p_int, const double *__restrict__ p_pair,
                             double *__restrict__ out) {
    if (threadIdx.x == 0) {
        double y = 0.0, g = 0.0;
        for (int b = 0; b < nb; ++b) {
            y += p_int[2 * b];
            g += p_int[2 * b + 1];
        }
        for (int b = 0; b < nb; ++b) g += p_pair[b];
        out[0] = y;
        out[1] = g;
    }
}

size_t adjoint_scratch_doubles(int64_t n) {
    const size_t nb = (size_t)((n + 127) / 128);
    return (size_t)n * 15 * 2 + nb * 3 + 2;   // lam_dir, mu, partials, result
}

// One adjoint step on the sorted view of step n (the forward pieces - sort, records, neighbour lists
// and FP64 rates - must already be computed for this step). scratch: adjoint_scratch_doubles(n).
cudaError_t launch_adjoint(const DevParams &P, int64_t n, const uint32_t *skey, const uint2 *cellr, const void *pos,
                           const void *rec, const double *xs, const double *ys, const double *zs, int kmax,
                           const uint2 *list, const uint32_t *cnt, const uint32_t *perm, const State &A,
                           const uint8_t *mat_s, const double *rates, double dt, const double *lam_next,
                           double *lam_prev, double *scratch, double *grad_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = (int)((n + 127) / 128);
    double *lam_dir = scratch;
    double *mu = scratch + (size_t)n * 15;
    double *p_int = mu + (size_t)n * 15;
    double *p_pair = p_int + (size_t)nb * 2;
    k_adj_integrate<<<nb, 128, 0, s>>>(P, n, perm, A, mat_s, rates, dt, lam_next, lam_dir, mu, p_int);
    k_adj_pair<<<nb, 128, 0, s>>>(P, n, skey, cellr, (const D4 *)pos, (const RecD *)rec, xs, ys, zs, kmax, list, cnt,
                                  perm, mat_s, mu, lam_dir, lam_prev, p_pair);
    k_adj_reduce<<<1, 32, 0, s>>>(nb, p_int, p_pair, grad_out);
    return cudaGetLastError();
}

}  // namespace gsph
