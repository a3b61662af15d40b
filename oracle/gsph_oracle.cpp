// gsph_oracle.cpp - plain, slow FP64 CPU oracle for the particle-decomposition Gamma-SPH-ALE hot path.
//
// TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's CPU-baseline leg load
// this library. It shares no code with the CUDA path. Compiled with -ffp-contract=off so that every
// product and sum is rounded separately (the integer decisions - hash, neighbour predicate, balancing
// hash - depend on that).
//
// Pins (tests/test_oracle_*.py): brute-force neighbour sets equal the bucket search; 80 interior
// neighbours on the jittered lattice; kernel closed form, unit integral and lattice sum; Riemann
// special cases; antisymmetry and conservation of mass, momentum and energy; uniform-state patch test;
// linear-velocity gradient; rigid-rotation stress rate; radial return; uniaxial wave speed; first law of
// the energy flux (pressure work); time step of the fastest particle; fixed-point Cg on exact grid points;
// hand-worked balancing hashes, single-type and two-type (biased Cg') swaps; label counts invariant under
// swaps; forward derivative against central differences. Every decision (hash, neighbour predicate,
// time step, Cg, balancing hash) is taken in FP64.
#include "gsph_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------------
// Scalar types: plain double, and a forward-mode dual number with 3 derivative components used
// only for the gradient check (derivatives w.r.t. yield stress, shear modulus, initial speed).
// ---------------------------------------------------------------------------------------------
struct Dual {
    double v;
    double d[3];
    Dual() : v(0), d{0, 0, 0} {}
    Dual(double x) : v(x), d{0, 0, 0} {}
};
inline Dual operator+(const Dual &a, const Dual &b) { Dual r(a.v + b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual &a, const Dual &b) { Dual r(a.v - b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual &a) { Dual r(-a.v); for (int k = 0; k < 3; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual &a, const Dual &b) { Dual r(a.v * b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual &a, const Dual &b) { Dual r(a.v / b.v); for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v); return r; }
inline Dual sqrt(const Dual &a) { double s = std::sqrt(a.v); Dual r(s); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] / (2.0 * s); return r; }
inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
inline double val(double x) { return x; }
inline double val(const Dual &x) { return x.v; }
using std::sqrt;

// Operation-counting scalar: each +, -, *, / and sqrt adds one to the counter (negation and
// comparisons add nothing). Run through the pair functions it gives the algorithmic FLOP count of one
// ordered pair interaction as written here.
thread_local int64_t g_flops = 0;
struct Count {
    double v;
    Count() : v(0) {}
    Count(double x) : v(x) {}
};
inline Count operator+(const Count &a, const Count &b) { ++g_flops; return Count(a.v + b.v); }
inline Count operator-(const Count &a, const Count &b) { ++g_flops; return Count(a.v - b.v); }
inline Count operator-(const Count &a) { return Count(-a.v); }
inline Count operator*(const Count &a, const Count &b) { ++g_flops; return Count(a.v * b.v); }
inline Count operator/(const Count &a, const Count &b) { ++g_flops; return Count(a.v / b.v); }
inline Count sqrt(const Count &a) { ++g_flops; return Count(std::sqrt(a.v)); }
inline bool operator>(const Count &a, const Count &b) { return a.v > b.v; }
inline double val(const Count &x) { return x.v; }

template <class T> struct Mat {
    T rho0, K, G, Y, c0, s, gamma0;
    int eos;
    double p_min;
};

// Equation of state (Sec. IV names a Mie-Gruneisen EOS with a cut-off pressure for spalling; it gives
// no formula, so this is a reading). Linear: p = K mu with mu = rho/rho0 - 1. Mie-Gruneisen with the
// Hugoniot of the linear shock relation Us = c0 + s up as reference curve and Gamma rho = gamma0 rho0:
//   p_H = rho0 c0^2 mu (1 + mu) / (1 - (s - 1) mu)^2 (mu > 0),  p_H = rho0 c0^2 mu (mu <= 0),
//   e_H = p_H mu / (2 rho0 (1 + mu))  (the Rankine-Hugoniot energy from the rest state),
//   p = p_H + gamma0 rho0 (e - e_H).
// The cut-off floors the pressure: p = max(p, p_min). The bulk sound speed is the isentropic
// derivative of the uncut pressure, c_b^2 = dp/drho|_e + (p / rho^2) dp/de|_rho, floored at 0.
template <class T> void eos_of(const Mat<T> &M, T rho, T e, T &p, T &cb2) {
    if (M.eos == 0) {
        p = M.K * (rho / M.rho0 - T(1.0));
        cb2 = M.K / rho;
    } else {
        T mu = rho / M.rho0 - T(1.0);
        T k0 = M.rho0 * M.c0 * M.c0;
        T pH, dpH;
        if (val(mu) > 0.0) {
            T D = T(1.0) - (M.s - T(1.0)) * mu;
            pH = k0 * mu * (T(1.0) + mu) / (D * D);
            dpH = k0 * ((T(1.0) + T(2.0) * mu) * D + T(2.0) * (M.s - T(1.0)) * mu * (T(1.0) + mu)) / (D * D * D);
        } else {
            pH = k0 * mu;
            dpH = k0;
        }
        T eH = pH * mu / (T(2.0) * M.rho0 * (T(1.0) + mu));
        T deH = (dpH * mu * (T(1.0) + mu) + pH) / (T(2.0) * M.rho0 * (T(1.0) + mu) * (T(1.0) + mu));
        p = pH + M.gamma0 * M.rho0 * (e - eH);
        // d/drho = (1 / rho0) d/dmu at fixed e; dp/de = gamma0 rho0
        cb2 = (dpH - M.gamma0 * M.rho0 * deH) / M.rho0 + p * M.gamma0 * M.rho0 / (rho * rho);
        if (val(cb2) < 0.0) cb2 = T(0.0);
    }
    if (val(p) < M.p_min) p = T(M.p_min);
}

// Per-particle primitive state seen by the interaction loop.
template <class T> struct Prim {
    T v[3], rho, p, Z, E, w;
    T S[6];  // xx yy zz xy xz yz
};

// (S n)_a for the symmetric tensor stored as xx yy zz xy xz yz.
template <class T> inline void sym_times(const T S[6], const T n[3], T out[3]) {
    out[0] = S[0] * n[0] + S[3] * n[1] + S[4] * n[2];
    out[1] = S[3] * n[0] + S[1] * n[1] + S[5] * n[2];
    out[2] = S[4] * n[0] + S[5] * n[1] + S[2] * n[2];
}

// ---------------------------------------------------------------------------------------------
// Kernel function: Wendland C2 in 3D with support 2h, W(q) = 21/(16 pi h^3) (1 - q/2)^4 (2q + 1),
// q = r/h. Its derivative is dW/dr = -5 * 21/(16 pi h^3) * q (1 - q/2)^3 / h, never positive.
// ---------------------------------------------------------------------------------------------
template <class T> inline T kernel_w(T r, double h) {
    double aw = 21.0 / (16.0 * PI * h * h * h);
    T q = r / h;
    if (!(val(q) < 2.0)) return T(0.0);
    T s = T(1.0) - q / 2.0;
    return aw * s * s * s * s * (T(2.0) * q + T(1.0));
}
template <class T> inline T kernel_dw_abs(T r, double h) {
    double aw = 21.0 / (16.0 * PI * h * h * h);
    T q = r / h;
    if (!(val(q) < 2.0)) return T(0.0);
    T s = T(1.0) - q / 2.0;
    return T(5.0 * aw) * q * s * s * s / h;
}

// ---------------------------------------------------------------------------------------------
// Acoustic Riemann problem on the pair normal n (left state L, right state R, n from L to R).
// The +c characteristic from the left keeps t - Z u and the -c characteristic from the right keeps
// t + Z u; the intermediate state (u*, t*) satisfies both.
// ---------------------------------------------------------------------------------------------
template <class T> inline void riemann(T uL, T uR, T tL, T tR, T ZL, T ZR, T &us, T &ts) {
    T zs = ZL + ZR;
    us = (ZL * uL + ZR * uR + (tR - tL)) / zs;
    ts = (ZR * tL + ZL * tR + ZL * ZR * (uR - uL)) / zs;
}

// Pair fluxes of the Gamma-SPH-ALE reading (Vila's conservative SPH-ALE with transport velocity
// v0 = v). dlr = x_R - x_L; the kernel gradient seen from L is |dW/dr| n, from R it is -|dW/dr| n.
// Outputs for L (R receives the negatives): Fm, Fmv, Fe are the amounts subtracted from the rates
// of L, i.e. d(m)_L/dt -= Fm, d(mv)_L/dt -= Fmv, d(mE)_L/dt -= Fe. Also returns a = |dW/dr|, n,
// and the normal velocities (for the volume rate).
// L and R are the states of the Riemann problem; L0 and R0 (null: L and R) are the particles' own
// states, whose velocities are the transport velocities v0 (they differ under MUSCL reconstruction):
// the mass flux carries (v_E - v0_LR) . n and the volume rate the particles' normal velocities.
template <class T> struct PairOut { T Fm, Fmv[3], Fe, a, n[3], uL, uR; };

template <class T>
inline void pair_flux(const T dlr[3], const Prim<T> &L, const Prim<T> &R, double h, PairOut<T> &o,
                      const Prim<T> *L0 = nullptr, const Prim<T> *R0 = nullptr) {
    if (!L0) L0 = &L;
    if (!R0) R0 = &R;
    T r2 = dlr[0] * dlr[0] + dlr[1] * dlr[1] + dlr[2] * dlr[2];
    T r = sqrt(r2);
    T n[3] = {dlr[0] / r, dlr[1] / r, dlr[2] / r};
    T a = kernel_dw_abs(r, h);
    T uL = L.v[0] * n[0] + L.v[1] * n[1] + L.v[2] * n[2];
    T uR = R.v[0] * n[0] + R.v[1] * n[1] + R.v[2] * n[2];
    // traction sigma n with sigma = -p I + S
    T sL[3], sR[3];
    sym_times(L.S, n, sL);
    sym_times(R.S, n, sR);
    for (int k = 0; k < 3; ++k) {
        sL[k] = sL[k] - L.p * n[k];
        sR[k] = sR[k] - R.p * n[k];
    }
    T tL = sL[0] * n[0] + sL[1] * n[1] + sL[2] * n[2];
    T tR = sR[0] * n[0] + sR[1] * n[1] + sR[2] * n[2];
    T us, ts;
    riemann(uL, uR, tL, tR, L.Z, R.Z, us, ts);
    T u0L = L0->v[0] * n[0] + L0->v[1] * n[1] + L0->v[2] * n[2];
    T u0R = R0->v[0] * n[0] + R0->v[1] * n[1] + R0->v[2] * n[2];
    T du = us - (u0L + u0R) / 2.0;               // (v_E - v0_LR) . n
    T dus = us - (uL + uR) / 2.0;                // the Riemann correction of the mean normal velocity
    T rhoE = (L.rho + R.rho) / 2.0;
    T EE = (L.E + R.E) / 2.0;
    T vE[3], TE[3];
    for (int k = 0; k < 3; ++k) {
        vE[k] = (L.v[k] + R.v[k]) / 2.0 + dus * n[k];
        // normal part from the Riemann solver, tangential part averaged
        TE[k] = ts * n[k] + ((sL[k] + sR[k]) - (tL + tR) * n[k]) / 2.0;
    }
    T ww = T(2.0) * L.w * R.w;
    T mflux = rhoE * du;
    o.Fm = ww * a * mflux;
    for (int k = 0; k < 3; ++k) o.Fmv[k] = ww * a * (mflux * vE[k] - TE[k]);
    T tv = TE[0] * vE[0] + TE[1] * vE[1] + TE[2] * vE[2];
    o.Fe = ww * a * (mflux * EE - tv);
    o.a = a;
    for (int k = 0; k < 3; ++k) o.n[k] = n[k];
    o.uL = u0L;
    o.uR = u0R;
}

// ---------------------------------------------------------------------------------------------
// State held by the templated core.
// ---------------------------------------------------------------------------------------------
template <class T> struct StateT {
    int64_t n = 0;
    std::vector<T> x, y, z, vx, vy, vz, w, m, E, S[6];
    std::vector<uint8_t> mat, label;
    std::vector<uint32_t> id;
    std::vector<double> hh;   // per-particle smoothing lengths (variable h), empty otherwise
    void resize(int64_t nn) {
        n = nn;
        for (auto *v : {&x, &y, &z, &vx, &vy, &vz, &w, &m, &E}) v->assign(nn, T(0.0));
        for (auto &s : S) s.assign(nn, T(0.0));
        mat.assign(nn, 0);
        label.assign(nn, 0);
        id.assign(nn, 0);
    }
};

StateT<double> load(const orc_state *S) {
    StateT<double> s;
    s.resize(S->n);
    for (int64_t i = 0; i < S->n; ++i) {
        s.x[i] = S->x[i]; s.y[i] = S->y[i]; s.z[i] = S->z[i];
        s.vx[i] = S->vx[i]; s.vy[i] = S->vy[i]; s.vz[i] = S->vz[i];
        s.w[i] = S->w[i]; s.m[i] = S->m[i]; s.E[i] = S->E[i];
        s.S[0][i] = S->sxx[i]; s.S[1][i] = S->syy[i]; s.S[2][i] = S->szz[i];
        s.S[3][i] = S->sxy[i]; s.S[4][i] = S->sxz[i]; s.S[5][i] = S->syz[i];
        s.mat[i] = S->mat[i]; s.label[i] = S->label[i]; s.id[i] = S->id[i];
    }
    if (S->h) s.hh.assign(S->h, S->h + S->n);
    return s;
}

template <class T> void store(const StateT<T> &s, orc_state *S) {
    for (int64_t i = 0; i < s.n; ++i) {
        S->x[i] = val(s.x[i]); S->y[i] = val(s.y[i]); S->z[i] = val(s.z[i]);
        S->vx[i] = val(s.vx[i]); S->vy[i] = val(s.vy[i]); S->vz[i] = val(s.vz[i]);
        S->w[i] = val(s.w[i]); S->m[i] = val(s.m[i]); S->E[i] = val(s.E[i]);
        S->sxx[i] = val(s.S[0][i]); S->syy[i] = val(s.S[1][i]); S->szz[i] = val(s.S[2][i]);
        S->sxy[i] = val(s.S[3][i]); S->sxz[i] = val(s.S[4][i]); S->syz[i] = val(s.S[5][i]);
        S->mat[i] = s.mat[i]; S->label[i] = s.label[i]; S->id[i] = s.id[i];
    }
    if (S->h && (int64_t)s.hh.size() == s.n) std::copy(s.hh.begin(), s.hh.end(), S->h);
}

inline int64_t ncells(const orc_params *P) {
    return (int64_t)P->dims[0] * P->dims[1] * P->dims[2];
}

// Bucket coordinate of one coordinate value: floor((x - lo) / 2h); -1 when below the grid, dims
// when at or beyond the top, so that callers can tell "outside" apart.
inline int64_t bucket_coord(double x, double lo, double cell, int32_t dim) {
    double t = (x - lo) / cell;
    if (!(t >= 0.0)) return -1;               // below the grid (or NaN)
    if (t >= (double)dim) return dim;
    return (int64_t)t;                        // truncation == floor for t >= 0
}

// Signed bucket coordinate, used for the mirrored search point, which may lie outside the grid.
inline int64_t bucket_coord_signed(double x, double lo, double cell) {
    return (int64_t)std::floor((x - lo) / cell);
}

uint32_t hash_of(const orc_params *P, double x, double y, double z) {
    double cell = 2.0 * P->h;
    int64_t c[3] = {bucket_coord(x, P->lo[0], cell, P->dims[0]),
                    bucket_coord(y, P->lo[1], cell, P->dims[1]),
                    bucket_coord(z, P->lo[2], cell, P->dims[2])};
    for (int a = 0; a < 3; ++a)
        if (c[a] < 0 || c[a] >= P->dims[a]) return (uint32_t)ncells(P);
    return (uint32_t)(c[0] + (int64_t)P->dims[0] * (c[1] + (int64_t)P->dims[1] * c[2]));
}

// Squared distance with each product and sum rounded separately.
inline double dist2(double dx, double dy, double dz) {
    double a = dx * dx;
    double b = dy * dy;
    double c = dz * dz;
    return (a + b) + c;
}

// Displacement from particle i to the image of particle j in wall k (mirror plane x_axis = pos).
inline void image_delta(const orc_wall &W, const double xi[3], const double xj[3], double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double xjp = xj[a];
        if (a == W.axis) xjp = 2.0 * W.pos - xj[a];
        d[a] = xjp - xi[a];
    }
}

// Bucket lists of the in-grid particles: particles of each bucket in slot order.
struct Buckets {
    std::vector<int64_t> head;   // CSR offsets per bucket
    std::vector<int64_t> items;
};

Buckets make_buckets(const orc_params *P, int64_t n, const uint32_t *key) {
    int64_t C = ncells(P);
    Buckets b;
    b.head.assign(C + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        if (key[i] < (uint64_t)C) b.head[key[i] + 1]++;
    for (int64_t c = 0; c < C; ++c) b.head[c + 1] += b.head[c];
    b.items.assign(b.head[C], 0);
    std::vector<int64_t> fill(b.head.begin(), b.head.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        if (key[i] < (uint64_t)C) b.items[fill[key[i]]++] = i;
    return b;
}

// Visits the in-grid particles of the 27 buckets around bucket coordinate (cx, cy, cz).
template <class F>
void for_27(const orc_params *P, const Buckets &b, int64_t cx, int64_t cy, int64_t cz, F &&f) {
    for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t X = cx + dx, Y = cy + dy, Z = cz + dz;
                if (X < 0 || Y < 0 || Z < 0 || X >= P->dims[0] || Y >= P->dims[1] || Z >= P->dims[2])
                    continue;
                int64_t c = X + (int64_t)P->dims[0] * (Y + (int64_t)P->dims[1] * Z);
                for (int64_t k = b.head[c]; k < b.head[c + 1]; ++k) f(b.items[k]);
            }
}

// Neighbour enumeration through the bucket search. Calls real(j) for each real neighbour and
// image(k, j) for each image of particle j in wall k within the support.
template <class FR, class FI>
void neighbours_of(const orc_params *P, const Buckets &b, int64_t n, const double *x, const double *y,
                   const double *z, const uint32_t *key, int64_t i, FR &&real, FI &&image,
                   const double *hv = nullptr) {
    int64_t C = ncells(P);
    if (key[i] >= (uint64_t)C) return;
    double cell = 2.0 * P->h;
    double R2u = cell * cell;
    // support of the pair: (2h)^2, or (h_i + h_j)^2 with per-particle smoothing lengths
    auto R2of = [&](int64_t j) {
        if (!hv) return R2u;
        double sij = hv[i] + hv[j];
        return sij * sij;
    };
    double xi[3] = {x[i], y[i], z[i]};
    int64_t ci[3];
    for (int a = 0; a < 3; ++a) ci[a] = bucket_coord(xi[a], P->lo[a], cell, P->dims[a]);
    for_27(P, b, ci[0], ci[1], ci[2], [&](int64_t j) {
        if (j == i) return;
        double r2 = dist2(x[j] - xi[0], y[j] - xi[1], z[j] - xi[2]);
        if (r2 < R2of(j)) real(j);
    });
    for (int k = 0; k < P->nwalls; ++k) {
        const orc_wall &W = P->wall[k];
        double m[3] = {xi[0], xi[1], xi[2]};
        m[W.axis] = 2.0 * W.pos - xi[W.axis];                       // mirrored search point
        int64_t cm[3];
        for (int a = 0; a < 3; ++a) cm[a] = bucket_coord_signed(m[a], P->lo[a], cell);
        for_27(P, b, cm[0], cm[1], cm[2], [&](int64_t j) {
            double xj[3] = {x[j], y[j], z[j]}, d[3];
            image_delta(W, xi, xj, d);
            if (dist2(d[0], d[1], d[2]) < R2of(j)) image(k, j);
        });
    }
    (void)n;
}

// Material constants and derived primitive state of particle i.
template <class T> Prim<T> prim_of(const StateT<T> &s, const Mat<T> *mats, int64_t i) {
    Prim<T> p;
    const Mat<T> &M = mats[s.mat[i]];
    p.v[0] = s.vx[i]; p.v[1] = s.vy[i]; p.v[2] = s.vz[i];
    p.w = s.w[i];
    p.rho = s.m[i] / s.w[i];
    T c;
    if (M.eos == 0) {   // linear EOS: c^2 = (K + 4G/3) / rho, the longitudinal modulus
        p.p = M.K * (p.rho / M.rho0 - T(1.0));
        c = sqrt((M.K + T(4.0) * M.G / 3.0) / p.rho);
        if (val(p.p) < M.p_min) p.p = T(M.p_min);
    } else {            // specific internal energy e = E - |v|^2 / 2
        T cb2;
        T e = s.E[i] - T(0.5) * (p.v[0] * p.v[0] + p.v[1] * p.v[1] + p.v[2] * p.v[2]);
        eos_of(M, p.rho, e, p.p, cb2);
        c = sqrt(cb2 + T(4.0) * M.G / (T(3.0) * p.rho));
    }
    p.Z = p.rho * c;
    p.E = s.E[i];
    for (int k = 0; k < 6; ++k) p.S[k] = s.S[k][i];
    return p;
}

// Mirror image of a primitive state in wall axis ax: the normal velocity component and the two
// shear components that carry one index along the axis change sign.
template <class T> Prim<T> mirror_prim(const Prim<T> &p, int ax) {
    Prim<T> q = p;
    q.v[ax] = -q.v[ax];
    // S components: 3 = xy, 4 = xz, 5 = yz
    if (ax == 0) { q.S[3] = -q.S[3]; q.S[4] = -q.S[4]; }
    if (ax == 1) { q.S[3] = -q.S[3]; q.S[5] = -q.S[5]; }
    if (ax == 2) { q.S[4] = -q.S[4]; q.S[5] = -q.S[5]; }
    return q;
}

// ---------------------------------------------------------------------------------------------
// MUSCL reconstruction (reading of the second-order SPH-ALE variant; the paper gives no scheme).
// Gradients of v and of the full stress sigma = -p I + S by the SPH gradient operator
//   G_i(phi) = sum_j w_j (phi_j - phi_i) grad_i W_ij,  grad_i W_ij = |dW/dr| (x_j - x_i) / r,
// over the same real and image neighbours as the fluxes. On a pair (L, R) with d = x_R - x_L each
// reconstructed component is limited by minmod against the centred difference:
//   phi_L* = phi_L + minmod(G_L(phi) . d, phi_R - phi_L) / 2,
//   phi_R* = phi_R - minmod(G_R(phi) . d, phi_R - phi_L) / 2,
// so the interface states stay between the two particle values, and a component at a local extremum
// (slope and difference of opposite signs) keeps its first-order value. Density, energy and impedance
// keep the particle values.
// ---------------------------------------------------------------------------------------------
constexpr int NGRAD = ORC_NGRAD;

// sigma = -p I + S as xx yy zz xy xz yz
template <class T> inline void sigma_of(const Prim<T> &p, T sg[6]) {
    for (int k = 0; k < 6; ++k) sg[k] = k < 3 ? p.S[k] - p.p : p.S[k];
}

template <class T> inline T minmod(T a, T b) {
    if (!(val(a) * val(b) > 0.0)) return T(0.0);
    return std::fabs(val(a)) < std::fabs(val(b)) ? a : b;
}

// Gradient of the mirror image of a particle in wall axis ax: d phi'/dx'_b picks up the sign of each
// index along the axis (the field's own indices and the derivative's).
template <class T> void mirror_grad(const T *G, int ax, T *Gm) {
    const int ci[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Gm[3 * a + b] = ((a == ax) != (b == ax)) ? -G[3 * a + b] : G[3 * a + b];
    for (int c = 0; c < 6; ++c)
        for (int b = 0; b < 3; ++b) {
            int flips = (ci[c][0] == ax) + (ci[c][1] == ax) + (b == ax);
            T g = G[9 + 3 * c + b];
            Gm[9 + 3 * c + b] = (flips & 1) ? -g : g;
        }
}

template <class T>
void grads_of(const orc_params *P, const StateT<T> &s, const Mat<T> *mats, const Buckets &b,
              const std::vector<double> &xv, const std::vector<double> &yv, const std::vector<double> &zv,
              const std::vector<uint32_t> &key, int64_t i, T *G) {
    for (int k = 0; k < NGRAD; ++k) G[k] = T(0.0);
    const double *hv = P->variable_h ? s.hh.data() : nullptr;
    Prim<T> pi = prim_of(s, mats, i);
    T si[6];
    sigma_of(pi, si);
    T xi[3] = {s.x[i], s.y[i], s.z[i]};
    auto add = [&](const Prim<T> &pj, const T d[3], int64_t j) {
        T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        T a = kernel_dw_abs(r, hv ? 0.5 * (hv[i] + hv[j]) : P->h);
        T gw[3] = {a * d[0] / r, a * d[1] / r, a * d[2] / r};
        T sj[6];
        sigma_of(pj, sj);
        for (int u = 0; u < 3; ++u)
            for (int c = 0; c < 3; ++c) G[3 * u + c] = G[3 * u + c] + pj.w * (pj.v[u] - pi.v[u]) * gw[c];
        for (int q = 0; q < 6; ++q)
            for (int c = 0; c < 3; ++c) G[9 + 3 * q + c] = G[9 + 3 * q + c] + pj.w * (sj[q] - si[q]) * gw[c];
    };
    neighbours_of(
        P, b, s.n, xv.data(), yv.data(), zv.data(), key.data(), i,
        [&](int64_t j) {
            T d[3] = {s.x[j] - xi[0], s.y[j] - xi[1], s.z[j] - xi[2]};
            add(prim_of(s, mats, j), d, j);
        },
        [&](int k, int64_t j) {
            const orc_wall &W = P->wall[k];
            T xj[3] = {s.x[j], s.y[j], s.z[j]};
            xj[W.axis] = T(2.0 * W.pos) - xj[W.axis];
            T d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
            add(mirror_prim(prim_of(s, mats, j), W.axis), d, j);
        },
        hv);
}

// Interface states of the pair (L, R), d = x_R - x_L: v and sigma reconstructed (the stress of the
// returned states is the full sigma with p = 0), the rest copied.
template <class T>
void reconstruct(const Prim<T> &L, const T *GL, const Prim<T> &R, const T *GR, const T d[3], Prim<T> &Ls,
                 Prim<T> &Rs) {
    Ls = L;
    Rs = R;
    auto dot = [&](const T *g) { return g[0] * d[0] + g[1] * d[1] + g[2] * d[2]; };
    for (int a = 0; a < 3; ++a) {
        T dphi = R.v[a] - L.v[a];
        Ls.v[a] = L.v[a] + minmod(dot(GL + 3 * a), dphi) / 2.0;
        Rs.v[a] = R.v[a] - minmod(dot(GR + 3 * a), dphi) / 2.0;
    }
    T sL[6], sR[6];
    sigma_of(L, sL);
    sigma_of(R, sR);
    for (int q = 0; q < 6; ++q) {
        T dphi = sR[q] - sL[q];
        Ls.S[q] = sL[q] + minmod(dot(GL + 9 + 3 * q), dphi) / 2.0;
        Rs.S[q] = sR[q] - minmod(dot(GR + 9 + 3 * q), dphi) / 2.0;
    }
    Ls.p = T(0.0);
    Rs.p = T(0.0);
}

// Adds one real pair to the rates r of particle i (Sec. II step f): volume rate from the transport
// velocities, the mass, momentum and energy fluxes with the orientation sign of i, and the velocity
// gradient L_i += w_j (v_j - v_i) (x) grad_i W_ij with grad_i W_ij = a n_{i->j}.
template <class T>
inline void accumulate_real(T *r, const Prim<T> &pi, const Prim<T> &pj, const PairOut<T> &o, bool i_left) {
    double sg = i_left ? -1.0 : 1.0;
    r[0] = r[0] + pi.w * pj.w * o.a * (o.uR - o.uL);
    r[1] = r[1] + sg * o.Fm;
    for (int k = 0; k < 3; ++k) r[2 + k] = r[2 + k] + sg * o.Fmv[k];
    r[5] = r[5] + sg * o.Fe;
    T nij[3];
    for (int k = 0; k < 3; ++k) nij[k] = i_left ? o.n[k] : -o.n[k];
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) r[6 + 3 * u + v] = r[6 + 3 * u + v] + pj.w * (pj.v[u] - pi.v[u]) * o.a * nij[v];
}

// Interaction loop (Sec. II step f): rates of particle i from all its real and image neighbours.
template <class T>
void rates_of(const orc_params *P, const StateT<T> &s, const Mat<T> *mats, const Buckets &b,
              const std::vector<double> &xv, const std::vector<double> &yv,
              const std::vector<double> &zv, const std::vector<uint32_t> &key, int64_t i, T *r,
              int32_t *nreal, int32_t *nimage, const T *grads = nullptr) {
    for (int k = 0; k < ORC_NRATE; ++k) r[k] = T(0.0);
    int32_t cr = 0, ci = 0;
    Prim<T> pi = prim_of(s, mats, i);
    T xi[3] = {s.x[i], s.y[i], s.z[i]};
    const double *hv = P->variable_h ? s.hh.data() : nullptr;
    auto hij = [&](int64_t j) { return hv ? 0.5 * (hv[i] + hv[j]) : P->h; };   // pair smoothing length
    auto add_L = [&](const T wj, const T vj[3], const T a, const T nij[3]) {
        // L_i += w_j (v_j - v_i) (x) grad_i W_ij, grad_i W_ij = a n_{i->j}
        for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v) r[6 + 3 * u + v] = r[6 + 3 * u + v] + wj * (vj[u] - pi.v[u]) * a * nij[v];
    };
    neighbours_of(
        P, b, s.n, xv.data(), yv.data(), zv.data(), key.data(), i,
        [&](int64_t j) {
            ++cr;
            Prim<T> pj = prim_of(s, mats, j);
            // canonical orientation: lower persistent id is the left state
            bool i_left = s.id[i] < s.id[j];
            int64_t l = i_left ? i : j, rr = i_left ? j : i;
            const Prim<T> &PL = i_left ? pi : pj;
            const Prim<T> &PR = i_left ? pj : pi;
            T d[3] = {s.x[rr] - s.x[l], s.y[rr] - s.y[l], s.z[rr] - s.z[l]};
            PairOut<T> o;
            if (grads) {
                Prim<T> Ls, Rs;
                reconstruct(PL, grads + NGRAD * l, PR, grads + NGRAD * rr, d, Ls, Rs);
                pair_flux(d, Ls, Rs, hij(j), o, &PL, &PR);
            } else {
                pair_flux(d, PL, PR, hij(j), o);
            }
            accumulate_real(r, pi, pj, o, i_left);
        },
        [&](int k, int64_t j) {
            ++ci;
            const orc_wall &W = P->wall[k];
            Prim<T> pj = mirror_prim(prim_of(s, mats, j), W.axis);
            T xj[3] = {s.x[j], s.y[j], s.z[j]};
            xj[W.axis] = T(2.0 * W.pos) - xj[W.axis];
            T d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
            PairOut<T> o;
            if (grads) {                                       // i is the left state
                T Gm[NGRAD];
                mirror_grad(grads + NGRAD * j, W.axis, Gm);
                Prim<T> Ls, Rs;
                reconstruct(pi, grads + NGRAD * i, pj, Gm, d, Ls, Rs);
                pair_flux(d, Ls, Rs, hij(j), o, &pi, &pj);
            } else {
                pair_flux(d, pi, pj, hij(j), o);
            }
            r[0] = r[0] + pi.w * pj.w * o.a * (o.uR - o.uL);
            r[1] = r[1] - o.Fm;
            for (int q = 0; q < 3; ++q) r[2 + q] = r[2 + q] - o.Fmv[q];
            r[5] = r[5] - o.Fe;
            add_L(pj.w, pj.v, o.a, o.n);
        },
        hv);
    if (nreal) nreal[i] = cr;
    if (nimage) nimage[i] = ci;
}

template <class T> void mats_of(const orc_params *P, Mat<T> *m) {
    for (int k = 0; k < P->nmat; ++k) {
        m[k].rho0 = T(P->mat[k].rho0);
        m[k].K = T(P->mat[k].K);
        m[k].G = T(P->mat[k].G);
        m[k].Y = T(P->mat[k].Y);
        m[k].c0 = T(P->mat[k].c0);
        m[k].s = T(P->mat[k].s);
        m[k].gamma0 = T(P->mat[k].gamma0);
        m[k].eos = P->mat[k].eos;
        m[k].p_min = P->mat[k].p_min;
    }
}

// Rates of every particle (or of a subset). The neighbour search (hash, buckets, support predicate)
// uses the positions of `search` (the state itself when null), the fluxes the state s: the second
// stage of the Heun step evaluates the predicted state over the neighbour set of the step's start.
template <class T>
void rates_all(const orc_params *P, const StateT<T> &s, const Mat<T> *mats, int64_t nsub,
               const int64_t *subset, T *rates, int32_t *nreal, int32_t *nimage,
               const StateT<T> *search = nullptr) {
    int64_t n = s.n;
    const StateT<T> &q = search ? *search : s;
    std::vector<double> xv(n), yv(n), zv(n);
    for (int64_t i = 0; i < n; ++i) { xv[i] = val(q.x[i]); yv[i] = val(q.y[i]); zv[i] = val(q.z[i]); }
    std::vector<uint32_t> key(n);
    orc_hash(P, n, xv.data(), yv.data(), zv.data(), key.data());
    Buckets b = make_buckets(P, n, key.data());
    // MUSCL: the gradients of every particle first (a pair needs both ends')
    std::vector<T> G;
    // (each particle's sums are its own: the loops over particles may run on several host threads,
    // orc_set_threads, without changing a bit)
    if (P->reconstruction == 1) {
        G.assign((size_t)n * NGRAD, T(0.0));
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) grads_of(P, s, mats, b, xv, yv, zv, key, i, G.data() + NGRAD * i);
    }
    const T *gp = G.empty() ? nullptr : G.data();
    if (subset) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t q = 0; q < nsub; ++q)
            rates_of(P, s, mats, b, xv, yv, zv, key, subset[q], rates + ORC_NRATE * subset[q], nreal, nimage, gp);
    } else {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i)
            rates_of(P, s, mats, b, xv, yv, zv, key, i, rates + ORC_NRATE * i, nreal, nimage, gp);
    }
}

// CFL signal speed c + |v| of one particle in FP64 (Sec. II step g; reading: the CFL condition on the
// largest signal speed). rho = m / w, |v|^2 with each product and sum rounded; linear EOS:
// c = sqrt(M / rho) with the longitudinal modulus M = K + 4G/3; Mie-Gruneisen: c = sqrt(c_b^2 + (4G/3) / rho)
// with c_b^2 from eos_of at e = E - |v|^2 / 2.
double signal_speed(const orc_params *P, const orc_state *S, int64_t i) {
    const orc_material &M = P->mat[S->mat[i]];
    double rho = S->m[i] / S->w[i];
    double v2 = dist2(S->vx[i], S->vy[i], S->vz[i]);
    double c;
    if (M.eos == 0) {
        double Mmod = M.K + 4.0 * M.G / 3.0;
        c = std::sqrt(Mmod / rho);
    } else {
        Mat<double> mm[ORC_MAX_MAT];
        mats_of(P, mm);
        double p, cb2;
        eos_of(mm[S->mat[i]], rho, S->E[i] - v2 / 2.0, p, cb2);
        double G43 = 4.0 * M.G / 3.0;
        c = std::sqrt(cb2 + G43 / rho);
    }
    return c + std::sqrt(v2);
}

// Forward Euler on the conserved variables and the Jaumann-rate stress update with radial return.
template <class T>
void integrate_one(const orc_params *P, StateT<T> &s, const Mat<T> *mats, int64_t i, const T *r, T dt) {
    const Mat<T> &M = mats[s.mat[i]];
    T v[3] = {s.vx[i], s.vy[i], s.vz[i]};
    T m = s.m[i];
    T g[3] = {T(P->g[0]), T(P->g[1]), T(P->g[2])};
    T wn = s.w[i] + dt * r[0];
    T mn = m + dt * r[1];
    T mv[3];
    for (int k = 0; k < 3; ++k) mv[k] = m * v[k] + dt * (r[2 + k] + m * g[k]);
    T gv = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
    T mE = m * s.E[i] + dt * (r[5] + m * gv);
    // stress: D = sym(L), Om = skew(L)
    T Lm[3][3];
    for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) Lm[u][w] = r[6 + 3 * u + w];
    T D[3][3], Om[3][3], Sm[3][3];
    for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) {
            D[u][w] = (Lm[u][w] + Lm[w][u]) / 2.0;
            Om[u][w] = (Lm[u][w] - Lm[w][u]) / 2.0;
        }
    const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) Sm[u][w] = s.S[idx[u][w]][i];
    T trD = D[0][0] + D[1][1] + D[2][2];
    T Sn[3][3];
    for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) {
            T dev = D[u][w];
            if (u == w) dev = dev - trD / 3.0;
            T rot = T(0.0);
            for (int k = 0; k < 3; ++k) rot = rot + (Om[u][k] * Sm[k][w] - Sm[u][k] * Om[k][w]);
            Sn[u][w] = Sm[u][w] + dt * (T(2.0) * M.G * dev + rot);
        }
    T trS = Sn[0][0] + Sn[1][1] + Sn[2][2];
    for (int u = 0; u < 3; ++u) Sn[u][u] = Sn[u][u] - trS / 3.0;
    T ss = Sn[0][0] * Sn[0][0] + Sn[1][1] * Sn[1][1] + Sn[2][2] * Sn[2][2] +
           T(2.0) * (Sn[0][1] * Sn[0][1] + Sn[0][2] * Sn[0][2] + Sn[1][2] * Sn[1][2]);
    T seq = sqrt(T(1.5) * ss);
    if (seq > M.Y) {
        T f = M.Y / seq;
        for (int u = 0; u < 3; ++u)
            for (int w = 0; w < 3; ++w) Sn[u][w] = Sn[u][w] * f;
    }
    s.x[i] = s.x[i] + dt * v[0];
    s.y[i] = s.y[i] + dt * v[1];
    s.z[i] = s.z[i] + dt * v[2];
    s.w[i] = wn;
    s.m[i] = mn;
    s.vx[i] = mv[0] / mn;
    s.vy[i] = mv[1] / mn;
    s.vz[i] = mv[2] / mn;
    s.E[i] = mE / mn;
    s.S[0][i] = Sn[0][0]; s.S[1][i] = Sn[1][1]; s.S[2][i] = Sn[2][2];
    s.S[3][i] = Sn[0][1]; s.S[4][i] = Sn[0][2]; s.S[5][i] = Sn[1][2];
}

// Fixed-point position for the centre of gravity (Sec. III.A; reading): per axis q = nearest integer
// (ties to even) to (x - lo) * s with s = 2^32 / L, L = dims * 2h the extent of the bucket grid, clamped
// to [0, 2^32 - 1] (NaN gives 0). The per-label sums of q are exact in int64 (at most 2^26 particles),
// and Cg = lo + (sum / count) * (L 2^-32).
struct Quant {
    double lo[3], s[3], step[3];
};
Quant quant_of(const orc_params *P) {
    Quant q;
    double cell = 2.0 * P->h;
    for (int a = 0; a < 3; ++a) {
        double ext = (double)P->dims[a] * cell;
        q.lo[a] = P->lo[a];
        q.s[a] = 4294967296.0 / ext;
        q.step[a] = ext * 0x1p-32;
    }
    return q;
}
inline int64_t quantise(const Quant &q, int a, double x) {
    double t = (x - q.lo[a]) * q.s[a];
    if (!(t > 0.0)) return 0;
    if (t >= 4294967295.0) return 4294967295LL;
    return (int64_t)std::nearbyint(t);
}

void cg_from_sums(const Quant &q, const int64_t sum[3], int64_t cnt, double cg[3]) {
    for (int a = 0; a < 3; ++a) {
        double mean = (double)sum[a] / (double)cnt;
        cg[a] = q.lo[a] + mean * q.step[a];
    }
}

}  // namespace

// =============================================================================================
// C entry points
// =============================================================================================
extern "C" {

int32_t orc_set_threads(int32_t nthreads) {
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : 1);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int64_t orc_flops_per_pair(void) {
    // one ordered pair of two particles in a generic state: the pair flux and its accumulation into the
    // 15 rates of one end (first-order Riemann states, uniform h)
    Prim<Count> L, R;
    const double vl[3] = {12.0, -3.0, 5.0}, vr[3] = {-7.0, 4.0, 1.0};
    const double sl[6] = {1e7, -2e7, 1e7, 3e6, -4e6, 5e6}, sr[6] = {-3e6, 1e6, 2e6, -1e6, 2e6, 7e6};
    for (int k = 0; k < 3; ++k) { L.v[k] = vl[k]; R.v[k] = vr[k]; }
    for (int k = 0; k < 6; ++k) { L.S[k] = sl[k]; R.S[k] = sr[k]; }
    L.rho = 2700.0; R.rho = 2710.0; L.p = 1e8; R.p = 2e8; L.Z = 1.7e7; R.Z = 1.71e7;
    L.E = 1e4; R.E = 2e4; L.w = 1e-9; R.w = 1.01e-9;
    Count d[3] = {3e-4, -2e-4, 5e-4};
    Count r[ORC_NRATE];
    PairOut<Count> o;
    g_flops = 0;
    pair_flux(d, L, R, 1.3e-3, o);
    accumulate_real(r, L, R, o, true);
    return g_flops;
}

void orc_eos(const orc_params *P, int32_t mat, double rho, double e, double *p, double *cb2) {
    Mat<double> m[ORC_MAX_MAT];
    mats_of(P, m);
    eos_of(m[mat], rho, e, *p, *cb2);
}

void orc_hash(const orc_params *P, int64_t n, const double *x, const double *y, const double *z,
              uint32_t *key) {
    for (int64_t i = 0; i < n; ++i) key[i] = hash_of(P, x[i], y[i], z[i]);
}

void orc_sort_order(int64_t n, const uint32_t *key, int64_t *perm) {
    std::vector<int64_t> p(n);
    std::iota(p.begin(), p.end(), 0);
    std::stable_sort(p.begin(), p.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    for (int64_t i = 0; i < n; ++i) perm[i] = p[i];
}

void orc_cell_ranges(int64_t n, const uint32_t *sorted_key, int64_t ncell, int64_t *start, int64_t *end) {
    for (int64_t c = 0; c < ncell; ++c) { start[c] = 0; end[c] = 0; }
    for (int64_t s = 0; s < n; ++s) {
        int64_t c = sorted_key[s];
        if (c >= ncell) continue;
        if (s == 0 || sorted_key[s - 1] != sorted_key[s]) start[c] = s;
        end[c] = s + 1;
    }
}

int64_t orc_neighbours_brute(const orc_params *P, int64_t n, const double *x, const double *y,
                             const double *z, int64_t cap, int32_t *count, int64_t *list, const double *h) {
    std::vector<uint32_t> key(n);
    orc_hash(P, n, x, y, z, key.data());
    uint32_t G = (uint32_t)ncells(P);
    double cell = 2.0 * P->h, R2u = cell * cell;
    int64_t mx = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        if (key[i] != G) {
            double xi[3] = {x[i], y[i], z[i]};
            auto R2of = [&](int64_t j) { double sij = h ? h[i] + h[j] : 0.0; return h ? sij * sij : R2u; };
            for (int64_t j = 0; j < n; ++j) {
                if (j == i || key[j] == G) continue;
                if (dist2(x[j] - xi[0], y[j] - xi[1], z[j] - xi[2]) < R2of(j)) {
                    if (c < cap) list[i * cap + c] = j;
                    ++c;
                }
            }
            for (int k = 0; k < P->nwalls; ++k)
                for (int64_t j = 0; j < n; ++j) {
                    if (key[j] == G) continue;
                    double xj[3] = {x[j], y[j], z[j]}, d[3];
                    image_delta(P->wall[k], xi, xj, d);
                    if (dist2(d[0], d[1], d[2]) < R2of(j)) {
                        if (c < cap) list[i * cap + c] = j + n * (1 + k);
                        ++c;
                    }
                }
        }
        count[i] = (int32_t)c;
        mx = std::max(mx, c);
    }
    return mx;
}

int64_t orc_neighbours_cells(const orc_params *P, int64_t n, const double *x, const double *y,
                             const double *z, int64_t cap, int32_t *count, int64_t *list, const double *h) {
    std::vector<uint32_t> key(n);
    orc_hash(P, n, x, y, z, key.data());
    Buckets b = make_buckets(P, n, key.data());
    int64_t mx = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        neighbours_of(
            P, b, n, x, y, z, key.data(), i,
            [&](int64_t j) { if (c < cap) list[i * cap + c] = j; ++c; },
            [&](int k, int64_t j) { if (c < cap) list[i * cap + c] = j + n * (1 + k); ++c; }, h);
        count[i] = (int32_t)c;
        mx = std::max(mx, c);
    }
    return mx;
}

void orc_rates(const orc_params *P, const orc_state *S, int64_t nsub, const int64_t *subset,
               double *rates, int32_t *nreal, int32_t *nimage) {
    StateT<double> s = load(S);
    Mat<double> mats[ORC_MAX_MAT];
    mats_of(P, mats);
    rates_all(P, s, mats, nsub, subset, rates, nreal, nimage);
}

double orc_signal_speed(const orc_params *P, const orc_state *S, int64_t i) { return signal_speed(P, S, i); }

double orc_dt(const orc_params *P, const orc_state *S) {
    double mx = 0.0;
    if (P->variable_h) {   // dt = cfl min_i h_i / s_i = cfl / max_i (s_i / h_i)
        for (int64_t i = 0; i < S->n; ++i) mx = std::max(mx, signal_speed(P, S, i) / S->h[i]);
        return P->cfl / mx;
    }
    for (int64_t i = 0; i < S->n; ++i) mx = std::max(mx, signal_speed(P, S, i));
    return (P->cfl * P->h) / mx;
}

void orc_integrate(const orc_params *P, orc_state *S, const double *rates, double dt) {
    StateT<double> s = load(S);
    Mat<double> mats[ORC_MAX_MAT];
    mats_of(P, mats);
    for (int64_t i = 0; i < s.n; ++i) integrate_one(P, s, mats, i, rates + ORC_NRATE * i, dt);
    store(s, S);
}

void orc_comm_hash(const orc_params *P, int64_t n, const uint32_t *key, const uint8_t *label,
                   uint8_t *flag, uint32_t *comm, int64_t *count) {
    uint32_t G = (uint32_t)ncells(P);
    Buckets b = make_buckets(P, n, key);
    for (int k = 0; k < P->K; ++k) count[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        flag[i] = 0;
        comm[i] = G;
        if (key[i] == G) continue;
        int64_t c = key[i];
        int64_t cx = c % P->dims[0], cy = (c / P->dims[0]) % P->dims[1], cz = c / ((int64_t)P->dims[0] * P->dims[1]);
        bool other = false;
        for_27(P, b, cx, cy, cz, [&](int64_t j) { if (label[j] != label[i]) other = true; });
        if (other) {
            flag[i] = 1;
            comm[i] = key[i];
            count[label[i]]++;
        }
    }
}

void orc_boundary_lists(int64_t n, const uint8_t *label, const uint32_t *comm, uint32_t garbage,
                        int32_t K, int64_t *offsets, int64_t *out) {
    int64_t pos = 0;
    for (int k = 0; k < K; ++k) {
        offsets[k] = pos;
        std::vector<int64_t> mine;
        for (int64_t i = 0; i < n; ++i)
            if (label[i] == k) mine.push_back(i);
        std::stable_sort(mine.begin(), mine.end(), [&](int64_t a, int64_t b) { return comm[a] < comm[b]; });
        for (int64_t i : mine)
            if (comm[i] != garbage) out[pos++] = i;
    }
    offsets[K] = pos;
}

int64_t orc_cg(const orc_params *P, int64_t n, const double *x, const double *y, const double *z,
               const uint8_t *label, const uint8_t *mat, int32_t lab, int32_t material, double cg[3]) {
    Quant q = quant_of(P);
    int64_t sum[3] = {0, 0, 0}, cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (label[i] != lab) continue;
        if (material >= 0 && mat[i] != material) continue;
        sum[0] += quantise(q, 0, x[i]);
        sum[1] += quantise(q, 1, y[i]);
        sum[2] += quantise(q, 2, z[i]);
        ++cnt;
    }
    if (cnt > 0) cg_from_sums(q, sum, cnt, cg);
    return cnt;
}

int32_t orc_balancing_hash(const double own[3], const double oth[3], const double p[3]) {
    // Sec. III.A in FP64: middle M of the Cg segment, d from the own Cg to the other, half-distance ell;
    // t = (p - M) . d / |d| is the signed distance of the projection past the middle.
    double M[3], d[3];
    for (int a = 0; a < 3; ++a) {
        M[a] = (own[a] + oth[a]) * 0.5;
        d[a] = oth[a] - own[a];
    }
    double dn = std::sqrt(dist2(d[0], d[1], d[2]));
    if (!(dn > 0.0)) return 0;                       // coincident Cgs: nothing to balance
    double ell = dn * 0.5;
    double e0 = p[0] - M[0], e1 = p[1] - M[1], e2 = p[2] - M[2];
    double a0 = e0 * d[0];
    double a1 = e1 * d[1];
    double a2 = e2 * d[2];
    double t = ((a0 + a1) + a2) / dn;
    if (!(t > 0.0)) return 0;                        // own side of the middle: not a swap candidate
    if (t >= ell) return ORC_HASH_MAX;               // at or beyond the other Cg
    double k = std::floor(1000.0 * t / ell);         // proportional to the distance past the middle
    if (k < 1.0) return 1;
    if (k >= (double)ORC_HASH_MAX) return ORC_HASH_MAX;
    return (int32_t)k;
}

int64_t orc_swap_pass(const orc_params *P, int64_t n, const double *x, const double *y,
                      const double *z, const uint8_t *mat, const uint32_t *id, uint8_t *label,
                      int64_t *swapped) {
    int K = P->K;
    bool multi = P->nmat > 1;
    int ntype = multi ? P->nmat : 1;
    double alpha = P->alpha;
    int64_t total = 0;
    for (int a = 0; a < K * K; ++a) swapped[a] = 0;
    for (int T = 0; T < ntype; ++T) {
        int mt = multi ? T : -1;
        for (int a = 0; a < K - 1; ++a)
            for (int b = a + 1; b < K; ++b) {
                double cga[3], cgb[3];
                int64_t na = orc_cg(P, n, x, y, z, label, mat, a, mt, cga);
                int64_t nb = orc_cg(P, n, x, y, z, label, mat, b, mt, cgb);
                if (na == 0 || nb == 0) continue;
                if (multi) {
                    // Sec. III.B: Cg' = alpha Cg_all + (1 - alpha) Cg_type, Cg_all of the same label
                    double alla[3], allb[3];
                    orc_cg(P, n, x, y, z, label, mat, a, -1, alla);
                    orc_cg(P, n, x, y, z, label, mat, b, -1, allb);
                    double beta = 1.0 - alpha;
                    for (int k = 0; k < 3; ++k) {
                        cga[k] = alpha * alla[k] + beta * cga[k];
                        cgb[k] = alpha * allb[k] + beta * cgb[k];
                    }
                }
                struct Cand { int32_t h; uint32_t id; int64_t slot; };
                std::vector<Cand> ca, cb;
                for (int64_t i = 0; i < n; ++i) {
                    if (mt >= 0 && mat[i] != mt) continue;
                    double p[3] = {x[i], y[i], z[i]};
                    if (label[i] == a) {
                        int32_t h = orc_balancing_hash(cga, cgb, p);
                        if (h > 0) ca.push_back({h, id[i], i});
                    } else if (label[i] == b) {
                        int32_t h = orc_balancing_hash(cgb, cga, p);
                        if (h > 0) cb.push_back({h, id[i], i});
                    }
                }
                int64_t m = std::min(ca.size(), cb.size());
                if (m == 0) continue;
                auto order = [](const Cand &u, const Cand &v) {
                    if (u.h != v.h) return u.h > v.h;   // largest balancing hash first
                    return u.id < v.id;                 // then lowest persistent id
                };
                std::sort(ca.begin(), ca.end(), order);
                std::sort(cb.begin(), cb.end(), order);
                for (int64_t k = 0; k < m; ++k) {
                    label[ca[k].slot] = (uint8_t)b;
                    label[cb[k].slot] = (uint8_t)a;
                }
                swapped[a * K + b] += m;
                total += 2 * m;
            }
    }
    return total;
}

void orc_step(const orc_params *P, orc_state *S, int32_t do_swap, uint32_t *key_out,
              uint32_t *comm_out, uint8_t *flag_out, int64_t *count_out, int32_t *nreal_out,
              int32_t *nimage_out, double *rates_out, double *dt_out) {
    int64_t n = S->n;
    double dt = (dt_out && *dt_out > 0.0) ? *dt_out : orc_dt(P, S);
    // a. hash, then the radix-sort step: a stable order by hash
    std::vector<uint32_t> key(n);
    orc_hash(P, n, S->x, S->y, S->z, key.data());
    std::vector<int64_t> perm(n);
    orc_sort_order(n, key.data(), perm.data());
    StateT<double> old = load(S), s;
    s.resize(n);
    std::vector<uint32_t> skey(n);
    for (int64_t t = 0; t < n; ++t) {
        int64_t o = perm[t];
        s.x[t] = old.x[o]; s.y[t] = old.y[o]; s.z[t] = old.z[o];
        s.vx[t] = old.vx[o]; s.vy[t] = old.vy[o]; s.vz[t] = old.vz[o];
        s.w[t] = old.w[o]; s.m[t] = old.m[o]; s.E[t] = old.E[o];
        for (int k = 0; k < 6; ++k) s.S[k][t] = old.S[k][o];
        s.mat[t] = old.mat[o]; s.label[t] = old.label[o]; s.id[t] = old.id[o];
        skey[t] = key[o];
    }
    if (!old.hh.empty()) {
        s.hh.resize(n);
        for (int64_t t = 0; t < n; ++t) s.hh[t] = old.hh[perm[t]];
    }
    std::vector<double> xv(s.x), yv(s.y), zv(s.z);
    if (do_swap) {
        std::vector<int64_t> sw(P->K * P->K);
        orc_swap_pass(P, n, xv.data(), yv.data(), zv.data(), s.mat.data(), s.id.data(), s.label.data(), sw.data());
    }
    // c. communication hash
    std::vector<uint8_t> flag(n);
    std::vector<uint32_t> comm(n);
    std::vector<int64_t> cnt(P->K);
    orc_comm_hash(P, n, skey.data(), s.label.data(), flag.data(), comm.data(), cnt.data());
    // f. interaction loop, g. integration
    Mat<double> mats[ORC_MAX_MAT];
    mats_of(P, mats);
    std::vector<double> rates((size_t)n * ORC_NRATE);
    std::vector<int32_t> nr(n), ni(n);
    rates_all(P, s, mats, 0, nullptr, rates.data(), nr.data(), ni.data());
    if (P->integrator == 1) {
        // two-stage Heun in its strong-stability-preserving form (reading of the second-order variant):
        // y* = E(y_n), y_{n+1} = (y_n + E(y*)) / 2 with E the forward Euler stage (radial return
        // included), both stages over the neighbour set of y_n; the average is taken on the conserved
        // variables (w, m, m v, m E, x, S), so the stress stays inside the convex yield set
        StateT<double> s1 = s;
        for (int64_t i = 0; i < n; ++i) integrate_one(P, s1, mats, i, rates.data() + ORC_NRATE * i, dt);
        std::vector<double> r2((size_t)n * ORC_NRATE);
        rates_all(P, s1, mats, 0, nullptr, r2.data(), nullptr, nullptr, &s);
        StateT<double> s2 = s1;
        for (int64_t i = 0; i < n; ++i) integrate_one(P, s2, mats, i, r2.data() + ORC_NRATE * i, dt);
        for (int64_t i = 0; i < n; ++i) {
            double m = 0.5 * (s.m[i] + s2.m[i]);
            double mv[3] = {0.5 * (s.m[i] * s.vx[i] + s2.m[i] * s2.vx[i]),
                            0.5 * (s.m[i] * s.vy[i] + s2.m[i] * s2.vy[i]),
                            0.5 * (s.m[i] * s.vz[i] + s2.m[i] * s2.vz[i])};
            double mE = 0.5 * (s.m[i] * s.E[i] + s2.m[i] * s2.E[i]);
            s.w[i] = 0.5 * (s.w[i] + s2.w[i]);
            s.x[i] = 0.5 * (s.x[i] + s2.x[i]);
            s.y[i] = 0.5 * (s.y[i] + s2.y[i]);
            s.z[i] = 0.5 * (s.z[i] + s2.z[i]);
            for (int k = 0; k < 6; ++k) s.S[k][i] = 0.5 * (s.S[k][i] + s2.S[k][i]);
            s.m[i] = m;
            s.vx[i] = mv[0] / m;
            s.vy[i] = mv[1] / m;
            s.vz[i] = mv[2] / m;
            s.E[i] = mE / m;
        }
    } else {
        for (int64_t i = 0; i < n; ++i) integrate_one(P, s, mats, i, rates.data() + ORC_NRATE * i, dt);
    }
    store(s, S);
    if (key_out) std::copy(skey.begin(), skey.end(), key_out);
    if (comm_out) std::copy(comm.begin(), comm.end(), comm_out);
    if (flag_out) std::copy(flag.begin(), flag.end(), flag_out);
    if (count_out) std::copy(cnt.begin(), cnt.end(), count_out);
    if (nreal_out) std::copy(nr.begin(), nr.end(), nreal_out);
    if (nimage_out) std::copy(ni.begin(), ni.end(), nimage_out);
    if (rates_out) std::copy(rates.begin(), rates.end(), rates_out);
    if (dt_out) *dt_out = dt;
}

void orc_gradients(const orc_params *P, const orc_state *S, double *grads) {
    StateT<double> s = load(S);
    int64_t n = s.n;
    Mat<double> mats[ORC_MAX_MAT];
    mats_of(P, mats);
    std::vector<uint32_t> key(n);
    orc_hash(P, n, s.x.data(), s.y.data(), s.z.data(), key.data());
    Buckets b = make_buckets(P, n, key.data());
    for (int64_t i = 0; i < n; ++i) grads_of(P, s, mats, b, s.x, s.y, s.z, key, i, grads + NGRAD * i);
}

double orc_kernel_w(double r, double h) { return kernel_w<double>(r, h); }
double orc_kernel_dw(double r, double h) { return kernel_dw_abs<double>(r, h); }

void orc_riemann(double uL, double uR, double tL, double tR, double ZL, double ZR, double out[2]) {
    riemann<double>(uL, uR, tL, tR, ZL, ZR, out[0], out[1]);
}

double orc_forward_gradient(const orc_params *P, orc_state *S, int32_t nsteps, const double *dts,
                            int64_t nobs, const uint32_t *obs_id, double grad[3]) {
    // Dual state: derivative 0 w.r.t. Y, 1 w.r.t. G (material 0), 2 w.r.t. the initial z speed v0,
    // seeded on every particle's initial z velocity (the initial state moves uniformly with v0,
    // and the specific total energy E = |v|^2 / 2 + e follows it).
    int64_t n = S->n;
    StateT<Dual> s;
    s.resize(n);
    StateT<double> d = load(S);
    for (int64_t i = 0; i < n; ++i) {
        s.x[i] = d.x[i]; s.y[i] = d.y[i]; s.z[i] = d.z[i];
        s.vx[i] = d.vx[i]; s.vy[i] = d.vy[i]; s.vz[i] = d.vz[i];
        s.vz[i].d[2] = 1.0;
        s.w[i] = d.w[i]; s.m[i] = d.m[i]; s.E[i] = d.E[i];
        s.E[i].d[2] = d.vz[i];                 // dE/dv0 = v_z for E = e + |v|^2/2
        for (int k = 0; k < 6; ++k) s.S[k][i] = d.S[k][i];
        s.mat[i] = d.mat[i]; s.label[i] = d.label[i]; s.id[i] = d.id[i];
    }
    s.hh = d.hh;
    Mat<Dual> mats[ORC_MAX_MAT];
    mats_of(P, mats);
    mats[0].Y.d[0] = 1.0;
    mats[0].G.d[1] = 1.0;
    std::vector<Dual> rates((size_t)n * ORC_NRATE);
    for (int st = 0; st < nsteps; ++st) {
        // the neighbour set and order come from the values; the sort is a permutation and does not
        // change the sums, so the oracle keeps slot order here
        rates_all(P, s, mats, 0, nullptr, rates.data(), nullptr, nullptr);
        for (int64_t i = 0; i < n; ++i) integrate_one(P, s, mats, i, rates.data() + ORC_NRATE * i, Dual(dts[st]));
    }
    Dual J(0.0);
    int64_t found = 0;
    for (int64_t q = 0; q < nobs; ++q)
        for (int64_t i = 0; i < n; ++i)
            if (s.id[i] == obs_id[q]) { J = J + s.vz[i]; ++found; break; }
    J = J / Dual((double)found);
    store(s, S);
    for (int k = 0; k < 3; ++k) grad[k] = J.d[k];
    return J.v;
}

}  // extern "C"
