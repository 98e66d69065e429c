// Injection sampling shared by the FP64 and MIXED particle kernels
// (reading of Sec. 3.1.3 / Sec. 5.2.2; the paper gives no sampler):
// uniform position on the face, flux-weighted normal speed by rejection,
// Gaussian tangential speeds plus drift, then a uniform fraction of one step.
#pragma once
#include "internal.h"

namespace pf {

constexpr int MAX_TRIES = 32;

struct InjArgs {
    const InjectDev* st;
    int nst;
    int* count;            // per stream, this step
    long long* idbase;     // per stream
    double* carry;         // per stream
    long long* next_id;    // per species
    const long long* step; // steps completed so far (device; advanced at the end of each step)
};

PF_D void box_muller(double u1, double u2, double& z0, double& z1) {
    double r = sqrt(-2.0 * log(u1));
    double t = (2.0 * 3.141592653589793) * u2;
    z0 = r * cos(t);
    z1 = r * sin(t);
}

// flux-weighted normal speed (units of vth): proposal N(mu, 1), mu the mode of
// v exp(-(v - s)^2 / 2), acceptance (v/mu) exp(1 - v/mu); bounded tries
PF_D bool flux_normal(unsigned long long m, unsigned long long seed, unsigned long long key1, double s, double& v) {
    double mu = 0.5 * (s + sqrt(s * s + 4.0));
    for (int t = 0; t < MAX_TRIES; ++t) {
        U64x4 r = philox4x64(m, 2 + t, 0, 0, seed, key1);
        double z, z1;
        box_muller(u01(r.v[0]), u01(r.v[1]), z, z1);
        double vv = mu + z;
        double ratio = vv / mu;
        if (vv > 0.0 && u01(r.v[2]) < ratio * exp(1.0 - ratio)) { v = vv; return true; }
    }
    return false;
}

struct InjSample {
    double p0[3], p[3], v[3];
    bool ok;
};

// particle mm of stream d in step `step`: start point p0 on the face, velocity
// v, position p after the partial first step; ok = false if every rejection
// try failed.  Counter (mm, block, 0, 0), key (seed, purpose 2 | species | face | step).
PF_D InjSample inject_sample(const InjectDev& d, int mm, long long step, int s, const Mesh& mesh, double dth) {
    const int f = d.face, ax = f >> 1;
    const double sgn = (f & 1) ? -1.0 : 1.0;
    const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
    const double nax[3] = {(double)mesh.nx, (double)mesh.ny, (double)mesh.nz};
    const unsigned long long key1 = stream_key(2, s, f, step);
    unsigned long long m = (unsigned long long)mm;
    U64x4 b0 = philox4x64(m, 0, 0, 0, d.seed, key1);
    U64x4 b1 = philox4x64(m, 1, 0, 0, d.seed, key1);
    InjSample r;
    double vn = 0.0;
    r.ok = flux_normal(m, d.seed, key1, sgn * d.drift[ax] / d.vth, vn);
    double g1, g2;
    box_muller(u01(b1.v[0]), u01(b1.v[1]), g1, g2);
    r.p0[ax] = sgn > 0 ? 0.0 : nax[ax];
    r.p0[t1] = u01(b0.v[0]) * nax[t1];
    r.p0[t2] = u01(b0.v[1]) * nax[t2];
    double frac = u01(b0.v[2]);
    r.v[ax] = sgn * (d.vth * vn);
    r.v[t1] = d.drift[t1] + d.vth * g1;
    r.v[t2] = d.drift[t2] + d.vth * g2;
    double sl = frac * dth;
    for (int c = 0; c < 3; ++c) r.p[c] = r.p0[c] + r.v[c] * sl;
    return r;
}

// ---- photoelectron emission (Sec. 5.2.2) ----------------------------------------
struct PhotoArgs {
    const PhotoDev* tets;
    const long long* Q;
    long long* carry;
    int* cnt;
    const long long* base;
    const long long* total;
    long long* next_id;        // per species
    long long ne;
    int species;
    double vth;
    unsigned long long seed;
    const long long* step;
    double dth;                // dt / h of the IFE mesh: emission works in IFE cell units
    double inv_r;              // 1 / refine (a power of two): IFE to PIC cell units, exact
};

struct PhotoSample {
    double p0[3], p[3], v[3];
    bool ok;
};

// particle m of this step's emissions from tet d: point on Gamma_h (triangle by
// area, then sqrt(r1), r2), flux-weighted normal speed (zero drift), Gaussian
// tangential speeds, then a fraction U of one step.  Blocks of counter (m, b):
// 0 -> (triangle, r1, r2, U), 1 -> tangential normals, 2.. -> normal speed.
PF_D PhotoSample photo_sample(const PhotoDev& d, unsigned long long m, unsigned long long seed,
                              unsigned long long key1, double vth, double dth) {
    PhotoSample r;
    U64x4 b0 = philox4x64(m, 0, 0, 0, seed, key1);
    U64x4 b1 = philox4x64(m, 1, 0, 0, seed, key1);
    double vn = 0.0;
    r.ok = flux_normal(m, seed, key1, 0.0, vn);
    double g1, g2;
    box_muller(u01(b1.v[0]), u01(b1.v[1]), g1, g2);
    const double ut = u01(b0.v[0]), r1 = u01(b0.v[1]), r2 = u01(b0.v[2]), U = u01(b0.v[3]);
    const int k = (d.ntri > 1 && ut * d.A >= d.area0) ? 1 : 0;
    const double sq = sqrt(r1);
    const double a0 = 1.0 - sq, a1 = sq * (1.0 - r2), a2 = sq * r2;
    const double sl = U * dth;
    for (int c = 0; c < 3; ++c) {
        r.p0[c] = (a0 * d.P[k][0][c] + a1 * d.P[k][1][c]) + a2 * d.P[k][2][c];
        r.v[c] = ((vth * vn) * d.n[c] + (vth * g1) * d.t1[c]) + (vth * g2) * d.t2[c];
        r.p[c] = r.p0[c] + r.v[c] * sl;
    }
    return r;
}

// emitting tet of emission m: the last tet whose base is <= m (tets with no
// emission this step share the base of the next one and come before it)
PF_D long long photo_tet_of(const long long* base, long long ne, long long m) {
    long long lo = 0, hi = ne;          // first index with base > m
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (base[mid] <= m) lo = mid + 1;
        else hi = mid;
    }
    return lo - 1;
}

// ---- FP32 sampling for the MIXED path -----------------------------------------
// The same Philox counters and keys as above; uniforms from the top 24 bits,
// ((x >> 40) + 0.5) 2^-24, strictly inside (0, 1) and exact in FP32, so an
// injected particle is the FP64 sample to FP32 precision.
PF_D float u01f(unsigned long long x) { return ((float)(x >> 40) + 0.5f) * 5.9604644775390625e-8f; }

PF_D void box_muller_f(float u1, float u2, float& z0, float& z1) {
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}

PF_D bool flux_normal_f(unsigned long long m, unsigned long long seed, unsigned long long key1, float s, float& v) {
    const float mu = 0.5f * (s + sqrtf(s * s + 4.0f));
    for (int t = 0; t < MAX_TRIES; ++t) {
        U64x4 r = philox4x64(m, 2 + t, 0, 0, seed, key1);
        float z, z1;
        box_muller_f(u01f(r.v[0]), u01f(r.v[1]), z, z1);
        const float vv = mu + z;
        const float ratio = vv / mu;
        if (vv > 0.0f && u01f(r.v[2]) < ratio * expf(1.0f - ratio)) { v = vv; return true; }
    }
    return false;
}

struct InjSampleF {
    float p0[3], p[3], v[3];
    bool ok;
};

PF_D InjSampleF inject_sample_f(const InjectDev& d, int mm, long long step, int s, const Mesh& mesh, float dth) {
    const int f = d.face, ax = f >> 1;
    const float sgn = (f & 1) ? -1.0f : 1.0f;
    const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
    const float nax[3] = {(float)mesh.nx, (float)mesh.ny, (float)mesh.nz};
    const unsigned long long key1 = stream_key(2, s, f, step);
    const unsigned long long m = (unsigned long long)mm;
    U64x4 b0 = philox4x64(m, 0, 0, 0, d.seed, key1);
    U64x4 b1 = philox4x64(m, 1, 0, 0, d.seed, key1);
    InjSampleF r;
    float vn = 0.0f;
    const float vth = (float)d.vth;
    r.ok = flux_normal_f(m, d.seed, key1, sgn * (float)d.drift[ax] / vth, vn);
    float g1, g2;
    box_muller_f(u01f(b1.v[0]), u01f(b1.v[1]), g1, g2);
    r.p0[ax] = sgn > 0.0f ? 0.0f : nax[ax];
    r.p0[t1] = u01f(b0.v[0]) * nax[t1];
    r.p0[t2] = u01f(b0.v[1]) * nax[t2];
    const float frac = u01f(b0.v[2]);
    r.v[ax] = sgn * (vth * vn);
    r.v[t1] = (float)d.drift[t1] + vth * g1;
    r.v[t2] = (float)d.drift[t2] + vth * g2;
    const float sl = frac * dth;
    for (int c = 0; c < 3; ++c) r.p[c] = r.p0[c] + r.v[c] * sl;
    return r;
}

}  // namespace pf
