// FP64 particle cycle (compiled without FMA contraction: the gather, push,
// level-set and weight arithmetic follows one fixed IEEE operation order so
// cell indices, hit decisions and fixed-point charges are reproducible).
//
// Sec. 2.1 (Fig. 1): charge weighted to nodes (scatter), field interpolated at
// particle positions (gather), velocity and position update (particle-push);
// Sec. 3.1.3: pre-load, injection at open faces, absorption at open faces;
// Sec. 5.2.2: particles hitting the object are collected and their charge is
// accumulated for surface charging.  The paper does not name its pusher or
// weighting; this file uses trilinear weights of the PIC cell, leapfrog, and
// int64 fixed-point deposits of 2^32 units per particle.
//
// Layout: per species, particles live in bins of BLK^3 cells (SoA, one
// contiguous slot range per bin).  One CTA handles one bin: it stages the
// bin's (BLK+1)^3 node-field tile in shared memory with a TMA tile load,
// pushes the bin's particles, deposits stayers into a shared int64 tile and
// compacts them in place; particles that leave the bin go to a mover list,
// from which a rebin kernel reinserts them (overflowing bins spill to the
// next step's mover list).
#include <math.h>

#include "internal.h"
#include "sampling.cuh"

namespace pf {

__constant__ TetTables cTp;
cudaError_t set_particle_tables(const TetTables& t) { return cudaMemcpyToSymbol(cTp, &t, sizeof(TetTables)); }

constexpr double TWO32 = 4294967296.0;

// ---- trilinear weights, fixed order: w_l = (wx[a] * wy[b]) * wz[c] ---------------
struct Wts {
    int ci, cj, ck;
    double w[8];
};
PF_D Wts weights(double x, double y, double z) {
    Wts r;
    double cx = floor(x), cy = floor(y), cz = floor(z);
    double fx = x - cx, fy = y - cy, fz = z - cz;
    double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
#pragma unroll
    for (int l = 0; l < 8; ++l) r.w[l] = (wx[l & 1] * wy[(l >> 1) & 1]) * wz[(l >> 2) & 1];
    r.ci = (int)cx; r.cj = (int)cy; r.ck = (int)cz;
    return r;
}

// 7 rounded weights + remainder: exactly 2^32 units per particle
PF_D void fixed_weights(const Wts& w, long long W[8]) {
    long long rest = 1ll << 32;
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        W[l] = __double2ll_rn(w.w[l] * TWO32);
        rest -= W[l];
    }
    W[7] = rest;
}

// node field at the 8 corners, accumulated left to right in node order
template <class EA>
PF_D void gather(const Wts& w, const EA& ea, double& ex, double& ey, double& ez) {
    double4 e0 = ea(w.ci, w.cj, w.ck);
    ex = w.w[0] * e0.x; ey = w.w[0] * e0.y; ez = w.w[0] * e0.z;
#pragma unroll
    for (int l = 1; l < 8; ++l) {
        double4 e = ea(w.ci + (l & 1), w.cj + ((l >> 1) & 1), w.ck + ((l >> 2) & 1));
        ex = ex + w.w[l] * e.x;
        ey = ey + w.w[l] * e.y;
        ez = ez + w.w[l] * e.z;
    }
}

struct EGlobal {
    const double4* E;
    Mesh m;
    PF_D double4 operator()(int i, int j, int k) const { return E[node_id(m, i, j, k)]; }
};
struct ETile {
    const double4* T;
    int x0, y0, z0;
    PF_D double4 operator()(int i, int j, int k) const {
        return T[(i - x0) + TILE * ((j - y0) + TILE * (k - z0))];
    }
};

PF_D bool outside(const Mesh& m, double x, double y, double z) {
    return (x < 0.0) | (x >= (double)m.nx) | (y < 0.0) | (y >= (double)m.ny) | (z < 0.0) | (z >= (double)m.nz);
}

// cell of the crossing point of a particle that entered the object
PF_D int hit_target(const Launch& L, double xo, double yo, double zo, double xn, double yn, double zn) {
    double Lo = level_set(L.obj, xo, yo, zo);
    double Ln = level_set(L.obj, xn, yn, zn);
    double t = Lo / (Lo - Ln);
    double xc = xo + t * (xn - xo), yc = yo + t * (yn - yo), zc = zo + t * (zn - zo);
    // the crossing point's cell on the IFE mesh (refine times finer; exact scaling)
    const Mesh& f = L.fmesh;
    double fi = floor(L.rf * xc), fj = floor(L.rf * yc), fk = floor(L.rf * zc);
    fi = fi < 0.0 ? 0.0 : (fi > (double)(f.nx - 1) ? (double)(f.nx - 1) : fi);
    fj = fj < 0.0 ? 0.0 : (fj > (double)(f.ny - 1) ? (double)(f.ny - 1) : fj);
    fk = fk < 0.0 ? 0.0 : (fk > (double)(f.nz - 1) ? (double)(f.nz - 1) : fk);
    return L.cell_acc[cell_id(f, (int)fi, (int)fj, (int)fk)];
}

enum { ALIVE = 0, ABSORBED = 1, COLLECTED = 2, NONE = 3 };

// boundary test, then object test (codes above); acc = surface slot for hits
PF_D int classify(const Launch& L, double xo, double yo, double zo, double x, double y, double z, int& acc) {
    if (outside(L.mesh, x, y, z)) return ABSORBED;
    if (level_set(L.obj, x, y, z) < 0.0) {
        acc = hit_target(L, xo, yo, zo, x, y, z);
        return COLLECTED;
    }
    return ALIVE;
}

// entries of a mover list: its counter may pass the capacity (reservations are
// made before the capacity check), so reads are clamped to the capacity
PF_D long long list_len(const unsigned long long* n, long long cap) {
    long long v = (long long)*n;
    return v < cap ? v : cap;
}

// the bin of a cell inside the mesh (non-negative indices; bin edge 2^bsh)
PF_D int block_of(const Launch& L, int ci, int cj, int ck) {
    return (ci >> L.bsh) + L.nbx * ((cj >> L.bsh) + L.nby * (ck >> L.bsh));
}

// deposit with weights w of a cell of the IFE mesh (the PIC mesh when refine == 1)
PF_D void global_deposit(const Launch& L, unsigned long long* W, const Wts& w) {
    long long Wf[8];
    fixed_weights(w, Wf);
#pragma unroll
    for (int l = 0; l < 8; ++l)
        atomicAdd(&W[node_id(L.fmesh, w.ci + (l & 1), w.cj + ((l >> 1) & 1), w.ck + ((l >> 2) & 1))],
                  (unsigned long long)Wf[l]);
}
// deposit of a particle at (x, y, z) (PIC cell units) on the IFE mesh
PF_D void deposit_at(const Launch& L, unsigned long long* W, double x, double y, double z) {
    if (L.refine == 1) global_deposit(L, W, weights(x, y, z));
    else global_deposit(L, W, weights(L.rf * x, L.rf * y, L.rf * z));
}

PF_D void put(const PArr& a, long long i, double x, double y, double z, double vx, double vy, double vz,
              long long id, bool track) {
    a.x[i] = x; a.y[i] = y; a.z[i] = z; a.vx[i] = vx; a.vy[i] = vy; a.vz[i] = vz;
    if (track) a.id[i] = id;
}

// count one event per lane into a shared counter (warp-aggregated)
PF_D void count_event(unsigned long long* sctr, bool ev) {
    unsigned m = __ballot_sync(0xffffffffu, ev);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(sctr, (unsigned long long)__popc(m));
}

// ------------------------------------------------------------------------------------
// fused gather + push + boundary + object hit + deposit + in-place compaction
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_push_bins(Launch L, const __grid_constant__ CUtensorMap tmE) {
    __shared__ alignas(128) double4 Et[TILE_N];
    // fixed-point tile (low 16 bits / signed high part) with 8 interleaved
    // copies per node, copy = lane & 7, to spread the atomics over the banks
    __shared__ int Wlo[8 * TILE_N];
    __shared__ int Whi[8 * TILE_N];
    __shared__ alignas(8) unsigned long long bar;
    __shared__ int wcnt[8];
    __shared__ unsigned sctr[NCTR];
    __shared__ int s_ok;
    const int s = blockIdx.y;
    const int b = blockIdx.x;
    const SpeciesDev& S = L.sp[s];
    const int n = S.bcount[b];
    if (n == 0) return;
    const int bx = b % L.nbx, by = (b / L.nbx) % L.nby, bz = b / (L.nbx * L.nby);
    const int x0 = bx * BLK, y0 = by * BLK, z0 = bz * BLK;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) { mbar_init(&bar, 1); fence_barrier_init(); }
    for (int t = tid; t < 8 * TILE_N; t += blockDim.x) { Wlo[t] = 0; Whi[t] = 0; }
    if (tid < NCTR) sctr[tid] = 0u;
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bar, TILE_N * (unsigned)sizeof(double4));
        tma_load_4d(Et, &tmE, &bar, 0, x0, y0, z0);
        bool ok = mbar_wait_bounded(&bar, 0);
        if (!ok) {
            atomicOr(L.err, ERR_TMA_TIMEOUT);
            mbar_wait_bounded(&bar, 0);      // give the copy in flight a second bounded chance
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const ETile ea{Et, x0, y0, z0};
    const long long start = S.bstart[b];
    const bool track = L.track;
    int nstay = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        int code = NONE, acc = -1;
        double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
        long long id = 0;
        Wts w;
        if (i < n) {
            const long long g = start + i;
            x = S.bins.x[g]; y = S.bins.y[g]; z = S.bins.z[g];
            vx = S.bins.vx[g]; vy = S.bins.vy[g]; vz = S.bins.vz[g];
            if (track) id = S.bins.id[g];
            w = weights(x, y, z);
            double ex, ey, ez;
            gather(w, ea, ex, ey, ez);
            vx = vx + S.k * ex; vy = vy + S.k * ey; vz = vz + S.k * ez;
            const double xo = x, yo = y, zo = z;
            x = x + vx * L.dth; y = y + vy * L.dth; z = z + vz * L.dth;
            if (S.reflect) reflect_d(L.mesh, S.reflect, x, y, z, vx, vy, vz);
            code = classify(L, xo, yo, zo, x, y, z, acc);
        }
        bool stay = false, mover = false;
        if (code == ALIVE) {
            w = weights(x, y, z);
            stay = (w.ci >= x0) & (w.ci < x0 + BLK) & (w.cj >= y0) & (w.cj < y0 + BLK) & (w.ck >= z0) &
                   (w.ck < z0 + BLK);
            mover = !stay;
            if (L.refine != 1) {
                deposit_at(L, S.W, x, y, z);      // hybrid grid: straight onto the IFE nodes
            } else if (stay) {
                long long Wf[8];
                fixed_weights(w, Wf);
                const long long W7[7] = {Wf[0], Wf[1], Wf[2], Wf[3], Wf[4], Wf[5], Wf[6]};
                const int t0 = (w.ci - x0) + TILE * ((w.cj - y0) + TILE * (w.ck - z0));
                tile_deposit(Wlo, Whi, 8 * t0 + (lane & 7), W7);
            } else {
                global_deposit(L, S.W, w);
            }
        } else if (code == COLLECTED) {
            if (acc >= 0) atomicAdd(&S.surf[acc], 1ull);
        }
        count_event32(&sctr[C_PUSHED], code != NONE);
        count_event32(&sctr[C_ABSORBED], code == ABSORBED);
        count_event32(&sctr[C_COLLECTED], code == COLLECTED);
        count_event32(&sctr[C_LOST], code == COLLECTED && acc < 0);
        // block-wide compaction of stayers (all reads of this chunk are done
        // before the barrier, so in-place writes cannot clobber unread slots)
        unsigned bal = __ballot_sync(0xffffffffu, stay);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int q = 0; q < nw; ++q) { int v = wcnt[q]; off += (q < wid) ? v : 0; tot += v; }
        if (stay) {
            long long dst = start + nstay + off + __popc(bal & ((1u << lane) - 1));
            put(S.bins, dst, x, y, z, vx, vy, vz, id, track);
        }
        long long slot = warp_reserve(S.mov_out_n, mover);
        if (mover) {
            if (slot < S.mcap) put(S.mov_out, slot, x, y, z, vx, vy, vz, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
        nstay += tot;
        __syncthreads();
    }
    if (tid == 0) S.bcount[b] = nstay;
    for (int t = tid; t < TILE_N; t += blockDim.x) {
        long long v = 0;
        for (int c = 0; c < 8; ++c) v += tile_value(Wlo[t * 8 + c], Whi[t * 8 + c]);
        if (!v) continue;
        int tx = t % TILE, ty = (t / TILE) % TILE, tz = t / (TILE * TILE);
        int gi = x0 + tx, gj = y0 + ty, gk = z0 + tz;
        if (gi <= L.mesh.nx && gj <= L.mesh.ny && gk <= L.mesh.nz) atomicAdd(&S.W[node_id(L.mesh, gi, gj, gk)], (unsigned long long)v);
    }
    if (tid < NCTR && sctr[tid]) atomicAdd(&S.ctr[tid], (unsigned long long)sctr[tid]);
}

// particles waiting in the mover list (spilled last step): same arithmetic,
// node field read from global memory; every survivor goes back to the list
// of this step's movers
__global__ void k_push_movers(Launch L) {
    __shared__ unsigned long long sctr[NCTR];
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    if (threadIdx.x < NCTR) sctr[threadIdx.x] = 0ull;
    __syncthreads();
    const long long n = list_len(S.mov_in_n, S.mcap);
    const EGlobal ea{L.E, L.mesh};
    const bool track = L.track;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += stride) {
        long long i = base + threadIdx.x;
        int code = NONE, acc = -1;
        double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
        long long id = 0;
        if (i < n) {
            x = S.mov_in.x[i]; y = S.mov_in.y[i]; z = S.mov_in.z[i];
            vx = S.mov_in.vx[i]; vy = S.mov_in.vy[i]; vz = S.mov_in.vz[i];
            if (track) id = S.mov_in.id[i];
            Wts w = weights(x, y, z);
            double ex, ey, ez;
            gather(w, ea, ex, ey, ez);
            vx = vx + S.k * ex; vy = vy + S.k * ey; vz = vz + S.k * ez;
            const double xo = x, yo = y, zo = z;
            x = x + vx * L.dth; y = y + vy * L.dth; z = z + vz * L.dth;
            if (S.reflect) reflect_d(L.mesh, S.reflect, x, y, z, vx, vy, vz);
            code = classify(L, xo, yo, zo, x, y, z, acc);
            if (code == ALIVE) deposit_at(L, S.W, x, y, z);
            else if (code == COLLECTED && acc >= 0) atomicAdd(&S.surf[acc], 1ull);
        }
        count_event(&sctr[C_PUSHED], code != NONE);
        count_event(&sctr[C_ABSORBED], code == ABSORBED);
        count_event(&sctr[C_COLLECTED], code == COLLECTED);
        count_event(&sctr[C_LOST], code == COLLECTED && acc < 0);
        bool alive = code == ALIVE;
        long long slot = warp_reserve(S.mov_out_n, alive);
        if (alive) {
            if (slot < S.mcap) put(S.mov_out, slot, x, y, z, vx, vy, vz, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

// ------------------------------------------------------------------------------------
// injection (reading of Sec. 3.1.3 / Sec. 5.2.2; see inject_one)
// ------------------------------------------------------------------------------------
// count = floor(carry + rate) per stream, ids consecutive per species in face order
__global__ void k_inject_counts(InjArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int q = 0; q < a.nst; ++q) {
        const InjectDev& d = a.st[q];
        double cr = a.carry[q] + d.rate;
        double nf = floor(cr);
        a.carry[q] = cr - nf;
        int cnt = (int)nf;
        if (cnt > d.maxcnt) cnt = d.maxcnt;
        a.count[q] = cnt;
        a.idbase[q] = a.next_id[d.species];
        a.next_id[d.species] += cnt;
    }
}

__global__ void k_inject(Launch L, InjArgs a) {
    __shared__ unsigned long long sctr[NCTR];
    const int q = blockIdx.y;
    const InjectDev d = a.st[q];
    const int s = d.species;
    const SpeciesDev& S = L.sp[s];
    if (threadIdx.x < NCTR) sctr[threadIdx.x] = 0ull;
    __syncthreads();
    const int cnt = a.count[q];
    const long long idb = a.idbase[q];
    const bool track = L.track;
    for (int base = blockIdx.x * blockDim.x; base < cnt; base += gridDim.x * blockDim.x) {
        int mm = base + threadIdx.x;
        int code = NONE, acc = -1;
        bool rejected = false;
        double p[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        if (mm < cnt) {
            InjSample sm = inject_sample(d, mm, *a.step, s, L.mesh, L.dth);
            double p0[3] = {sm.p0[0], sm.p0[1], sm.p0[2]};
            bool ok = sm.ok;
            for (int c = 0; c < 3; ++c) { p[c] = sm.p[c]; v[c] = sm.v[c]; }
            if (S.reflect) reflect_d(L.mesh, S.reflect, p[0], p[1], p[2], v[0], v[1], v[2]);
            if (!ok || level_set(L.obj, p0[0], p0[1], p0[2]) < 0.0) {
                rejected = true;
            } else {
                code = classify(L, p0[0], p0[1], p0[2], p[0], p[1], p[2], acc);
                if (code == ALIVE) deposit_at(L, S.W, p[0], p[1], p[2]);
                else if (code == COLLECTED && acc >= 0) atomicAdd(&S.surf[acc], 1ull);
            }
        }
        count_event(&sctr[C_INJECTED], code != NONE);
        count_event(&sctr[C_REJECTED], rejected);
        count_event(&sctr[C_ABSORBED], code == ABSORBED);
        count_event(&sctr[C_COLLECTED], code == COLLECTED);
        count_event(&sctr[C_LOST], code == COLLECTED && acc < 0);
        bool alive = code == ALIVE;
        long long slot = warp_reserve(S.mov_out_n, alive);
        if (alive) {
            if (slot < S.mcap) put(S.mov_out, slot, p[0], p[1], p[2], v[0], v[1], v[2], idb + mm, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

// ------------------------------------------------------------------------------------
// rebin: movers -> bins; a full bin sends the particle to next step's mover list
// ------------------------------------------------------------------------------------
__global__ void k_rebin(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    const long long n = list_len(S.mov_out_n, S.mcap);
    const bool track = L.track;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += stride) {
        long long i = base + threadIdx.x;
        bool spill = false;
        double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
        long long id = 0;
        if (i < n) {
            x = S.mov_out.x[i]; y = S.mov_out.y[i]; z = S.mov_out.z[i];
            vx = S.mov_out.vx[i]; vy = S.mov_out.vy[i]; vz = S.mov_out.vz[i];
            if (track) id = S.mov_out.id[i];
            int b = block_of(L, (int)floor(x), (int)floor(y), (int)floor(z));
            int slot = warp_inc(&S.bcount[b]);
            if (slot < S.bcap[b]) put(S.bins, S.bstart[b] + slot, x, y, z, vx, vy, vz, id, track);
            else spill = true;
        }
        long long slot = warp_reserve(S.mov_in_n, spill);
        if (spill) {
            if (slot < S.mcap) put(S.mov_in, slot, x, y, z, vx, vy, vz, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
}

__global__ void k_step_advance(long long* step) { *step += 1; }

__global__ void k_clamp_counts(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < L.nblocks && S.bcount[b] > S.bcap[b]) S.bcount[b] = S.bcap[b];
    if (b == 0) {
        unsigned long long sp = *S.mov_in_n;
        S.ctr[C_SPILLED] = sp < (unsigned long long)S.mcap ? sp : (unsigned long long)S.mcap;
        if (sp > (unsigned long long)S.mcap) *S.mov_in_n = S.mcap;
    }
}

// ------------------------------------------------------------------------------------
// loading, bin construction, flattening, deposit of everything, leapfrog start
// ------------------------------------------------------------------------------------
__global__ void k_load(Launch L, int s, int ppc, double vth, double dx, double dy, double dz,
                       unsigned long long seed, PArr out, unsigned long long* nout, long long cap) {
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const Mesh& m = L.mesh;
    if (g >= m.ncells * (long long)ppc) return;
    long long c = g / ppc;
    int pc = (int)(g % ppc);
    int i = (int)(c % m.nx), j = (int)((c / m.nx) % m.ny), k = (int)(c / ((long long)m.nx * m.ny));
    unsigned long long key1 = stream_key(1, s, 0, 0);
    U64x4 b0 = philox4x64((unsigned long long)c, (unsigned long long)pc, 0, 0, seed, key1);
    U64x4 b1 = philox4x64((unsigned long long)c, (unsigned long long)pc, 1, 0, seed, key1);
    double x = (double)i + u01(b0.v[0]);
    double y = (double)j + u01(b0.v[1]);
    double z = (double)k + u01(b0.v[2]);
    if (level_set(L.obj, x, y, z) < 0.0) return;
    double g0, g1, g2, g3;
    box_muller(u01(b1.v[0]), u01(b1.v[1]), g0, g1);
    box_muller(u01(b1.v[2]), u01(b1.v[3]), g2, g3);
    unsigned long long slot = warp_inc64(nout);
    if ((long long)slot >= cap) return;
    put(out, (long long)slot, x, y, z, dx + vth * g0, dy + vth * g1, dz + vth * g2, c * ppc + pc, true);
}

__global__ void k_bin_count(Launch L, PArr a, long long n, int* cnt) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = block_of(L, (int)floor(a.x[i]), (int)floor(a.y[i]), (int)floor(a.z[i]));
    warp_inc(&cnt[b]);
}

// capacity per bin: count + 25% + 64 slack, multiple of 32
__global__ void k_bin_caps(int nb, const int* cnt, int* cap, int* cnt_copy) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int c = cnt[b];
    int cp = ((c + c / 4 + 64) + 31) & ~31;
    cap[b] = cp < BIN_MAX ? cp : BIN_MAX;   // larger loads wait in the mover list
    cnt_copy[b] = 0;
}

// exclusive scan of the bin capacities, one block of BIN_SCAN_THREADS: each
// thread sums a contiguous run of bins, the runs' totals are scanned across
// the block, then each thread writes its run's starts
__global__ void k_bin_scan(int nb, const int* cap, long long* start, long long* total) {
    __shared__ long long wsum[BIN_SCAN_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (nb + BIN_SCAN_THREADS - 1) / BIN_SCAN_THREADS;
    const int b0 = t * per, b1 = min(b0 + per, nb);
    long long mine = 0;
    for (int b = b0; b < b1; ++b) mine += cap[b];
    long long inc = mine;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long v = lane < BIN_SCAN_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < BIN_SCAN_THREADS / 32) wsum[lane] = v;   // inclusive over warps
    }
    __syncthreads();
    long long run = inc - mine + (w > 0 ? wsum[w - 1] : 0);
    for (int b = b0; b < b1; ++b) { start[b] = run; run += cap[b]; }
    if (t == BIN_SCAN_THREADS - 1) *total = wsum[BIN_SCAN_THREADS / 32 - 1];
}

// a bin already at capacity sends the particle to the waiting (mover) list
__global__ void k_bin_scatter(Launch L, int s, PArr a, long long n, bool track) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SpeciesDev& S = L.sp[s];
    int b = block_of(L, (int)floor(a.x[i]), (int)floor(a.y[i]), (int)floor(a.z[i]));
    int slot = warp_inc(&S.bcount[b]);
    long long id = track ? a.id[i] : 0;
    if (slot < S.bcap[b]) {
        put(S.bins, S.bstart[b] + slot, a.x[i], a.y[i], a.z[i], a.vx[i], a.vy[i], a.vz[i], id, track);
    } else {
        unsigned long long q = atomicAdd(S.mov_in_n, 1ull);
        if ((long long)q < S.mcap) put(S.mov_in, (long long)q, a.x[i], a.y[i], a.z[i], a.vx[i], a.vy[i], a.vz[i], id, track);
        else atomicAdd(&S.ctr[C_DROPPED], 1ull);
    }
}

__global__ void k_flatten(Launch L, int s, PArr out, unsigned long long* nout) {
    const SpeciesDev& S = L.sp[s];
    int b = blockIdx.x;
    int n = S.bcount[b];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = n ? atomicAdd(nout, (unsigned long long)n) : 0ull;
    __syncthreads();
    long long st = S.bstart[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        long long g = st + i;
        put(out, (long long)base + i, S.bins.x[g], S.bins.y[g], S.bins.z[g], S.bins.vx[g], S.bins.vy[g],
            S.bins.vz[g], L.track ? S.bins.id[g] : 0, L.track);
    }
}

__global__ void k_flatten_list(Launch L, int s, PArr out, unsigned long long* nout) {
    const SpeciesDev& S = L.sp[s];
    long long n = list_len(S.mov_in_n, S.mcap);
    __shared__ unsigned long long base;
    if (threadIdx.x == 0 && blockIdx.x == 0) base = 0;
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) base = n ? atomicAdd(nout, (unsigned long long)n) : 0ull;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
        put(out, (long long)base + i, S.mov_in.x[i], S.mov_in.y[i], S.mov_in.z[i], S.mov_in.vx[i], S.mov_in.vy[i],
            S.mov_in.vz[i], L.track ? S.mov_in.id[i] : 0, L.track);
}

// scatter of every particle (bins + waiting movers) with global atomics
__global__ void k_deposit_bins(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    int b = blockIdx.x;
    int n = S.bcount[b];
    long long st = S.bstart[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        long long g = st + i;
        deposit_at(L, S.W, S.bins.x[g], S.bins.y[g], S.bins.z[g]);
    }
}
__global__ void k_deposit_list(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    long long n = list_len(S.mov_in_n, S.mcap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        deposit_at(L, S.W, S.mov_in.x[i], S.mov_in.y[i], S.mov_in.z[i]);
}

// v <- v - (k/2) E(x)
__global__ void k_half_kick_bins(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    int b = blockIdx.x;
    int n = S.bcount[b];
    long long st = S.bstart[b];
    const EGlobal ea{L.E, L.mesh};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        long long g = st + i;
        double ex, ey, ez;
        gather(weights(S.bins.x[g], S.bins.y[g], S.bins.z[g]), ea, ex, ey, ez);
        S.bins.vx[g] = S.bins.vx[g] - S.khalf * ex;
        S.bins.vy[g] = S.bins.vy[g] - S.khalf * ey;
        S.bins.vz[g] = S.bins.vz[g] - S.khalf * ez;
    }
}
__global__ void k_half_kick_list(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    long long n = list_len(S.mov_in_n, S.mcap);
    const EGlobal ea{L.E, L.mesh};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double ex, ey, ez;
        gather(weights(S.mov_in.x[i], S.mov_in.y[i], S.mov_in.z[i]), ea, ex, ey, ez);
        S.mov_in.vx[i] = S.mov_in.vx[i] - S.khalf * ex;
        S.mov_in.vy[i] = S.mov_in.vy[i] - S.khalf * ey;
        S.mov_in.vz[i] = S.mov_in.vz[i] - S.khalf * ez;
    }
}

// ------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------
static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

Launch make_launch(Ctx& c) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.mesh = c.pmesh; L.obj = c.obj; L.dth = c.dth;
    L.fmesh = c.mesh; L.refine = c.refine; L.rf = (double)c.refine;
    L.nbx = c.nbx; L.nby = c.nby; L.nbz = c.nbz; L.nblocks = c.nblocks;
    L.bsh = c.bin_edge == 8 ? 3 : 2;
    L.nspecies = (int)c.sp.size();
    L.track = c.track;
    L.cell_acc = c.cell_acc;
    L.E = c.Ep; L.Ef = c.Efp;   // the node field at the PIC nodes
    L.err = c.err_word;
    for (int s = 0; s < L.nspecies; ++s) {
        Species& q = c.sp[s];
        SpeciesDev& d = L.sp[s];
        d.k = q.k; d.khalf = 0.5 * q.k;
        d.bins = q.bins; d.binsF = q.binsF;
        d.bstart = q.bstart; d.bcap = q.bcap; d.bcount = q.bcount; d.bstay = q.bstay;
        d.mov_in = q.mov[0]; d.mov_out = q.mov[1];
        d.movF_in = q.movF[0]; d.movF_out = q.movF[1];
        d.mov_in_n = q.mov_n; d.mov_out_n = q.mov_n + 1;
        d.mcap = q.mcap;
        d.W = q.W; d.surf = q.surf; d.ctr = q.ctr;
        d.reflect = q.reflect;
    }
    return L;
}

static InjArgs inj_args(Ctx& c) {
    InjArgs a;
    a.st = c.inj_dev; a.nst = (int)c.inj.size();
    a.count = c.inj_count; a.idbase = c.inj_base; a.carry = c.inj_carry; a.next_id = c.next_id;
    a.step = (const long long*)(c.scal + 42);
    return a;
}

cudaError_t launch_load_maxwellian(Ctx& c, int s, int ppc, double vth, const double drift[3],
                                   unsigned long long seed, PArr flat, unsigned long long* nflat, long long cap) {
    Launch L = make_launch(c);
    long long n = c.pmesh.ncells * (long long)ppc;
    k_load<<<nb(n), 256, 0, c.stream>>>(L, s, ppc, vth, drift[0], drift[1], drift[2], seed, flat, nflat, cap);
    return cudaGetLastError();
}

cudaError_t launch_flatten(Ctx& c, int s, PArr flat, unsigned long long* nflat) {
    Launch L = make_launch(c);
    if (c.sp[s].bcount) k_flatten<<<c.nblocks, 256, 0, c.stream>>>(L, s, flat, nflat);
    if (c.sp[s].mov_n) k_flatten_list<<<1, 256, 0, c.stream>>>(L, s, flat, nflat);
    return cudaGetLastError();
}

// (re)build the bins of species s from a flat list of n particles on the device
cudaError_t launch_build_bins(Ctx& c, int s, PArr flat, long long n, bool) {
    Species& q = c.sp[s];
    cudaError_t e;
    int* cnt = nullptr;
    long long* tot = nullptr;
    long long total = 0;
    e = lib_malloc(&cnt, sizeof(int) * c.nblocks);
    if (e != cudaSuccess) return e;
    e = lib_malloc(&tot, sizeof(long long));
    if (e != cudaSuccess) { lib_free(cnt); return e; }
    cudaMemsetAsync(cnt, 0, sizeof(int) * c.nblocks, c.stream);
    Launch L = make_launch(c);
    if (n > 0) k_bin_count<<<nb(n), 256, 0, c.stream>>>(L, flat, n, cnt);
    if (!q.bcap) {
        lib_malloc(&q.bcap, sizeof(int) * c.nblocks);
        lib_malloc(&q.bcount, sizeof(int) * c.nblocks);
        lib_malloc(&q.bstart, sizeof(long long) * c.nblocks);
    }
    k_bin_caps<<<nb(c.nblocks), 256, 0, c.stream>>>(c.nblocks, cnt, q.bcap, q.bcount);
    k_bin_scan<<<1, BIN_SCAN_THREADS, 0, c.stream>>>(c.nblocks, q.bcap, q.bstart, tot);
    e = cudaMemcpyAsync(&total, tot, sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) { lib_free(cnt); lib_free(tot); return e; }
    if (total > q.cap) {
        double** arr[6] = {&q.bins.x, &q.bins.y, &q.bins.z, &q.bins.vx, &q.bins.vy, &q.bins.vz};
        for (auto a : arr) { lib_free(*a); *a = nullptr; }
        lib_free(q.bins.id); q.bins.id = nullptr;
        for (auto a : arr) {
            e = lib_malloc(a, sizeof(double) * total);
            if (e != cudaSuccess) { lib_free(cnt); lib_free(tot); return e; }
        }
        if (c.track) {
            e = lib_malloc(&q.bins.id, sizeof(long long) * total);
            if (e != cudaSuccess) { lib_free(cnt); lib_free(tot); return e; }
        }
        q.cap = total;
    }
    L = make_launch(c);
    cudaMemsetAsync(q.mov_n, 0, 2 * sizeof(unsigned long long), c.stream);
    if (n > 0) k_bin_scatter<<<nb(n), 256, 0, c.stream>>>(L, s, flat, n, c.track != 0);
    k_clamp_counts<<<dim3(nb(c.nblocks), (unsigned)c.sp.size()), 256, 0, c.stream>>>(L);
    e = cudaStreamSynchronize(c.stream);
    lib_free(cnt);
    lib_free(tot);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_deposit_all(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    cudaMemsetAsync(c.Wall, 0, sizeof(unsigned long long) * MAX_SPECIES * c.mesh.nnodes, c.stream);
    if (ns == 0) return cudaGetLastError();
    k_deposit_bins<<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L);
    k_deposit_list<<<dim3(64, ns), 256, 0, c.stream>>>(L);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_half_kick(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    if (ns == 0) return cudaSuccess;
    k_half_kick_bins<<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L);
    k_half_kick_list<<<dim3(64, ns), 256, 0, c.stream>>>(L);
    c.launches += 2;
    return cudaGetLastError();
}

// push of all bins (+ node-field tiles by TMA) and of waiting movers
// what precedes a push: the step's mover-list counts and node charges start at zero
cudaError_t launch_push_prep(Ctx& c) {
    int ns = (int)c.sp.size();
    for (int s = 0; s < ns; ++s)
        cudaMemsetAsync(c.sp[s].mov_n + 1, 0, sizeof(unsigned long long), c.stream);
    cudaMemsetAsync(c.Wall, 0, sizeof(unsigned long long) * ns * c.mesh.nnodes, c.stream);
    return cudaGetLastError();
}

cudaError_t launch_push_bins(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    k_push_bins<<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L, c.tmapE);
    c.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_push(Ctx& c) {
    cudaError_t e = launch_push_prep(c);
    return e == cudaSuccess ? launch_push_bins(c) : e;
}

cudaError_t launch_movers(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    k_push_movers<<<dim3(152, ns), 256, 0, c.stream>>>(L);
    c.launches += 1;
    return cudaGetLastError();
}

// ---- photoelectron emission (FP64 state) -------------------------------------
// scan kernels of setup.cu (graph-safe here: the tile buffer is preallocated)
__global__ void k_scan_tiles(const int* in, long long n, long long* out, long long* tile_sum);
__global__ void k_scan_sums(long long* tile_sum, long long ntiles, long long* total);
__global__ void k_scan_add(long long* out, long long n, const long long* tile_sum);

// this step's count per emitting tet from the fixed-point carry
__global__ void k_photo_counts(PhotoArgs a) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= a.ne) return;
    const long long tot = a.carry[e] + a.Q[e];
    a.cnt[e] = (int)(tot >> PHOTO_RATE_BITS);
    a.carry[e] = tot & ((1ll << PHOTO_RATE_BITS) - 1);
}

__global__ void k_photo(Launch L, PhotoArgs a) {
    __shared__ unsigned long long sctr[NCTR];
    const SpeciesDev& S = L.sp[a.species];
    if (threadIdx.x < NCTR) sctr[threadIdx.x] = 0ull;
    __syncthreads();
    const long long total = *a.total;
    const long long idb = a.next_id[a.species];
    const unsigned long long key1 = stream_key(3, a.species, 0, *a.step);
    const bool track = L.track;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < total; base += stride) {
        const long long m = base + threadIdx.x;
        bool emitted = false, alive = false, out = false;
        double p[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        if (m < total) {
            const PhotoDev& d = a.tets[photo_tet_of(a.base, a.ne, m)];
            const PhotoSample sm = photo_sample(d, (unsigned long long)m, a.seed, key1, a.vth, a.dth);
            for (int c = 0; c < 3; ++c) { p[c] = sm.p[c] * a.inv_r; v[c] = sm.v[c]; }   // to PIC units
            if (S.reflect) reflect_d(L.mesh, S.reflect, p[0], p[1], p[2], v[0], v[1], v[2]);
            emitted = sm.ok && !(level_set(L.obj, p[0], p[1], p[2]) < 0.0);
            if (emitted) {
                atomicAdd(&S.surf[d.acc], (unsigned long long)-1ll);   // the electron leaves +e behind
                out = outside(L.mesh, p[0], p[1], p[2]);
                alive = !out;
                if (alive) deposit_at(L, S.W, p[0], p[1], p[2]);
            }
        }
        count_event(&sctr[C_INJECTED], emitted);
        count_event(&sctr[C_REJECTED], m < total && !emitted);
        count_event(&sctr[C_ABSORBED], out);
        long long slot = warp_reserve(S.mov_out_n, alive);
        if (alive) {
            if (slot < S.mcap) put(S.mov_out, slot, p[0], p[1], p[2], v[0], v[1], v[2], idb + m, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

__global__ void k_photo_ids(long long* next_id, const long long* total) { *next_id += *total; }

PhotoArgs photo_args(Ctx& c) {
    PhotoArgs a;
    a.tets = c.ph_tets; a.Q = c.ph_Q; a.carry = c.ph_carry; a.cnt = c.ph_cnt; a.base = c.ph_base;
    a.total = c.ph_total; a.next_id = c.next_id; a.ne = c.ph_ne; a.species = c.ph_species; a.vth = c.ph_vth;
    a.seed = c.ph_seed; a.step = (const long long*)(c.scal + 42);
    a.dth = c.dt / c.mesh.h;
    a.inv_r = 1.0 / (double)c.refine;
    return a;
}

// counts and their scan for this step (both precisions)
cudaError_t launch_photo_counts(Ctx& c) {
    PhotoArgs a = photo_args(c);
    const long long ne = c.ph_ne, ntiles = (ne + 2047) / 2048;
    k_photo_counts<<<nb(ne), 256, 0, c.stream>>>(a);
    k_scan_tiles<<<(unsigned)ntiles, 256, 0, c.stream>>>(c.ph_cnt, ne, c.ph_base, c.ph_tiles);
    k_scan_sums<<<1, 32, 0, c.stream>>>(c.ph_tiles, ntiles, c.ph_total);
    k_scan_add<<<nb(ne), 256, 0, c.stream>>>(c.ph_base, ne, c.ph_tiles);
    c.launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_photo(Ctx& c) {
    if (c.ph_species < 0 || c.ph_ne <= 0) return cudaSuccess;
    cudaError_t e = launch_photo_counts(c);
    if (e != cudaSuccess) return e;
    k_photo<<<4 * 152, 256, 0, c.stream>>>(make_launch(c), photo_args(c));
    k_photo_ids<<<1, 1, 0, c.stream>>>(c.next_id + c.ph_species, c.ph_total);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_inject(Ctx& c) {
    if (!c.inj.empty()) {
        Launch L = make_launch(c);
        InjArgs a = inj_args(c);
        k_inject_counts<<<1, 32, 0, c.stream>>>(a);
        int maxc = 1;
        for (auto& d : c.inj) maxc = d.maxcnt > maxc ? d.maxcnt : maxc;
        unsigned gx = (unsigned)((maxc + 255) / 256);
        if (gx > 1024) gx = 1024;
        k_inject<<<dim3(gx, (unsigned)c.inj.size()), 256, 0, c.stream>>>(L, a);
        c.launches += 2;
    }
    return launch_photo(c);
}

cudaError_t launch_rebin(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    for (int s = 0; s < ns; ++s) cudaMemsetAsync(c.sp[s].mov_n, 0, sizeof(unsigned long long), c.stream);
    k_rebin<<<dim3(4 * 152, ns), 256, 0, c.stream>>>(L);
    k_clamp_counts<<<dim3(nb(c.nblocks), ns), 256, 0, c.stream>>>(L);
    k_step_advance<<<1, 1, 0, c.stream>>>((long long*)(c.scal + 42));
    c.launches += 3;
    return cudaGetLastError();
}

}  // namespace pf
