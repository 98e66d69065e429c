// MIXED-precision particle cycle: the same steps as particles.cu (Sec. 2.1
// gather / push / scatter, Sec. 3.1.3 and Sec. 5.2.2 injection, absorption and
// collection) with the state a particle carries cut to 28 bytes: a packed
// int32 cell (i | j<<11 | k<<22), the FP32 offset inside the cell and the
// FP32 velocity.  Positions never lose precision far from the origin because
// the offset is relative to the cell.  Node charges stay int64 with exactly
// 2^32 units per particle; the weights are FP32, rounded to 2^-19 of a particle
// inside a bin (2^-32 for movers).  Injection samples in FP32 from the same
// random streams as the FP64 path.
#include <math.h>

#include "internal.h"
#include "sampling.cuh"

namespace pf {

// kernels defined in particles.cu (bin construction and count clamping do not
// depend on the particle representation)
__global__ void k_bin_count(Launch L, PArr a, long long n, int* cnt);
__global__ void k_bin_caps(int nb, const int* cnt, int* cap, int* cnt_copy);
__global__ void k_bin_scan(int nb, const int* cap, long long* start, long long* total);
__global__ void k_clamp_counts(Launch L);

struct ObjF {
    int kind;
    float a0, a1, a2, a3, a4, a5, a6, a7, a8, a9, a10, a11;
};

static ObjF obj_f(const Object& o) {
    ObjF f;
    f.kind = o.kind;
    f.a0 = (float)o.a0; f.a1 = (float)o.a1; f.a2 = (float)o.a2;
    f.a3 = (float)o.a3; f.a4 = (float)o.a4; f.a5 = (float)o.a5;
    f.a6 = (float)o.a6; f.a7 = (float)o.a7; f.a8 = (float)o.a8;
    f.a9 = (float)o.a9; f.a10 = (float)o.a10; f.a11 = (float)o.a11;
    return f;
}

PF_D float level_set_f(const ObjF& o, float x, float y, float z) {
    if (o.kind == 1) {
        float dx = x - o.a0, dy = y - o.a1, dz = z - o.a2;
        return (dx * dx + dy * dy + dz * dz) - o.a3;
    } else if (o.kind == 2) {
        float dx = x - o.a1, dy = y - o.a2;
        float r2 = dx * dx + dy * dy;
        float zs = (r2 < o.a3) ? o.a5 - sqrtf(o.a4 - r2) : o.a0;
        return z - zs;
    } else if (o.kind == 3) {
        return o.a0 * x + o.a1 * y + o.a2 * z - o.a3;
    } else if (o.kind == 4) {   // rim crater, parameters as in level_set
        const float dx = x - o.a0, dy = y - o.a1;
        const float r = sqrtf(dx * dx + dy * dy);
        float zs;
        if (r <= o.a2) {
            zs = o.a5;
        } else if (r <= o.a3) {
            const float t = (r - o.a2) / o.a9;
            zs = o.a5 + o.a7 * ((t * t) * (3.0f - 2.0f * t));
        } else if (r < o.a4) {
            const float t = (r - o.a3) / o.a10;
            zs = o.a6 - o.a8 * ((t * t) * (3.0f - 2.0f * t));
        } else {
            zs = o.a11;
        }
        return z - zs;
    }
    return 1.0f;
}

PF_D int pack_cell(int i, int j, int k) { return i | (j << 11) | (k << 22); }
PF_D void unpack_cell(int c, int& i, int& j, int& k) {
    unsigned u = (unsigned)c;
    i = (int)(u & 2047u);
    j = (int)((u >> 11) & 2047u);
    k = (int)(u >> 22);
}

struct WF {
    float w[8];
};
PF_D WF weights_f(float fx, float fy, float fz) {
    WF r;
    float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
#pragma unroll
    for (int l = 0; l < 8; ++l) r.w[l] = (wx[l & 1] * wy[(l >> 1) & 1]) * wz[(l >> 2) & 1];
    return r;
}

PF_D void fixed_weights_f(const WF& w, long long W[8]) {
    long long rest = 1ll << 32;
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        // w < 1 except at a cell corner; 2^32 saturates to 2^32 - 1 and the
        // remainder weight below restores the exact total
        W[l] = (long long)__float2uint_rn(w.w[l] * 4294967296.0f);
        rest -= W[l];
    }
    W[7] = rest;
}

struct EGlobalF {
    const float4* E;
    Mesh m;
    PF_D float4 operator()(int i, int j, int k) const { return E[node_id(m, i, j, k)]; }
};

template <class EA>
PF_D void gather_f(int i, int j, int k, const WF& w, const EA& ea, float& ex, float& ey, float& ez) {
    ex = 0.f; ey = 0.f; ez = 0.f;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        float4 e = ea(i + (l & 1), j + ((l >> 1) & 1), k + ((l >> 2) & 1));
        ex += w.w[l] * e.x;
        ey += w.w[l] * e.y;
        ez += w.w[l] * e.z;
    }
}

// one particle: kick, drift in cell-relative coordinates, cell change,
// boundary test, object test (codes as in particles.cu)
enum { ALIVE = 0, ABSORBED = 1, COLLECTED = 2, NONE = 3 };

struct PF32 {
    int i, j, k;
    float fx, fy, fz, vx, vy, vz;
};

PF_D void advance_axis(float& f, int& c) {
    float s = floorf(f);
    f -= s;
    c += (int)s;
    if (f >= 1.0f) { f = 0.0f; c += 1; }   // -tiny - (-1) rounded up to 1
}

// reflecting faces (bit f = face f, minus face first per axis) on the cell +
// offset state: the mirror of c + f is -c - f at the minus face and 2n - c - f
// at the plus face, split again into a cell and an offset in [0, 1); a mirror
// that rounds onto n takes the last offset below 1 of cell n - 1
PF_D void reflect_axis_f(int& c, float& f, float& v, int n, int lo, int hi) {
    if (lo && c < 0) {
        if (f == 0.0f) {
            c = -c;
        } else {
            c = -c - 1; f = 1.0f - f;
            if (f >= 1.0f) { f = 0.0f; c += 1; }
        }
        v = -v;
    }
    if (hi && c >= n) {
        if (f == 0.0f) {
            c = 2 * n - c;
        } else {
            c = 2 * n - c - 1; f = 1.0f - f;
            if (f >= 1.0f) { f = 0.0f; c += 1; }
        }
        if (c >= n) { c = n - 1; f = 0.99999994f; }
        v = -v;
    }
}
PF_D void reflect_cell(const Mesh& m, int mask, PF32& p) {
    reflect_axis_f(p.i, p.fx, p.vx, m.nx, mask & 1, mask & 2);
    reflect_axis_f(p.j, p.fy, p.vy, m.ny, mask & 4, mask & 8);
    reflect_axis_f(p.k, p.fz, p.vz, m.nz, mask & 16, mask & 32);
}
// the same on a plain FP32 coordinate (injected particles, before the cell split)
PF_D void reflect_axis_pf(float& x, float& v, int n, int lo, int hi) {
    const float nf = (float)n;
    if (lo && x < 0.0f) { x = -x; v = -v; }
    if (hi && x >= nf) {
        x = (2.0f * nf) - x;
        if (x >= nf) x = __int_as_float(__float_as_int(nf) - 1);
        v = -v;
    }
}

PF_D int hit_cell_f(const Launch& L, const ObjF& of, float xo, float yo, float zo, float xn, float yn, float zn) {
    float Lo = level_set_f(of, xo, yo, zo), Ln = level_set_f(of, xn, yn, zn);
    float t = Lo / (Lo - Ln);
    float xc = xo + t * (xn - xo), yc = yo + t * (yn - yo), zc = zo + t * (zn - zo);
    // the crossing point's cell on the IFE mesh (refine times finer; exact scaling)
    const float r = (float)L.refine;
    int ci = min(max((int)floorf(r * xc), 0), L.fmesh.nx - 1);
    int cj = min(max((int)floorf(r * yc), 0), L.fmesh.ny - 1);
    int ck = min(max((int)floorf(r * zc), 0), L.fmesh.nz - 1);
    return L.cell_acc[cell_id(L.fmesh, ci, cj, ck)];
}

template <class EA>
PF_D int push_one(const Launch& L, const ObjF& of, float kf, float dthf, int refl, PF32& p, const EA& ea, int& acc) {
    WF w = weights_f(p.fx, p.fy, p.fz);
    float ex, ey, ez;
    gather_f(p.i, p.j, p.k, w, ea, ex, ey, ez);
    p.vx += kf * ex; p.vy += kf * ey; p.vz += kf * ez;
    float xo = (float)p.i + p.fx, yo = (float)p.j + p.fy, zo = (float)p.k + p.fz;
    p.fx += p.vx * dthf; p.fy += p.vy * dthf; p.fz += p.vz * dthf;
    advance_axis(p.fx, p.i); advance_axis(p.fy, p.j); advance_axis(p.fz, p.k);
    if (refl) reflect_cell(L.mesh, refl, p);
    if (p.i < 0 || p.i >= L.mesh.nx || p.j < 0 || p.j >= L.mesh.ny || p.k < 0 || p.k >= L.mesh.nz) return ABSORBED;
    float xn = (float)p.i + p.fx, yn = (float)p.j + p.fy, zn = (float)p.k + p.fz;
    if (level_set_f(of, xn, yn, zn) < 0.0f) {
        acc = hit_cell_f(L, of, xo, yo, zo, xn, yn, zn);
        return COLLECTED;
    }
    return ALIVE;
}

// deposit on the IFE mesh: with refine r the IFE cell of (i + f) is r i +
// floor(r f) and its offset frac(r f) (exact in FP32: r is a power of two)
PF_D void global_deposit_f(const Launch& L, unsigned long long* W, const PF32& p) {
    long long Wf[8];
    int i = p.i, j = p.j, k = p.k;
    float fx = p.fx, fy = p.fy, fz = p.fz;
    if (L.refine != 1) {
        const float r = (float)L.refine;
        const float sx = floorf(r * fx), sy = floorf(r * fy), sz = floorf(r * fz);
        i = L.refine * i + (int)sx; j = L.refine * j + (int)sy; k = L.refine * k + (int)sz;
        fx = r * fx - sx; fy = r * fy - sy; fz = r * fz - sz;
    }
    fixed_weights_f(weights_f(fx, fy, fz), Wf);
#pragma unroll
    for (int l = 0; l < 8; ++l)
        atomicAdd(&W[node_id(L.fmesh, i + (l & 1), j + ((l >> 1) & 1), k + ((l >> 2) & 1))],
                  (unsigned long long)Wf[l]);
}

// asynchronous 4-byte global -> shared copies (cp.async), committed in groups
PF_D void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
PF_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
PF_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
PF_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

PF_D void load_p(const PArrF& a, long long g, PF32& p) {
    unpack_cell(a.cell[g], p.i, p.j, p.k);
    p.fx = a.fx[g]; p.fy = a.fy[g]; p.fz = a.fz[g];
    p.vx = a.vx[g]; p.vy = a.vy[g]; p.vz = a.vz[g];
}
PF_D void store_p(const PArrF& a, long long g, const PF32& p, long long id, bool track) {
    a.cell[g] = pack_cell(p.i, p.j, p.k);
    a.fx[g] = p.fx; a.fy[g] = p.fy; a.fz[g] = p.fz;
    a.vx[g] = p.vx; a.vy[g] = p.vy; a.vz[g] = p.vz;
    if (track) a.id[g] = id;
}

PF_D void count_event(unsigned long long* sctr, bool ev) {
    unsigned m = __ballot_sync(0xffffffffu, ev);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(sctr, (unsigned long long)__popc(m));
}

PF_D long long list_len(const unsigned long long* n, long long cap) {
    long long v = (long long)*n;
    return v < cap ? v : cap;
}

// the bin of a cell inside the mesh (non-negative indices; bin edge 2^bsh)
PF_D int block_of(const Launch& L, int ci, int cj, int ck) {
    return (ci >> L.bsh) + L.nbx * ((cj >> L.bsh) + L.nby * (ck >> L.bsh));
}

// ------------------------------------------------------------------------------------
// fused gather + push + boundary + collection + deposit + compaction (one bin per CTA)
// ------------------------------------------------------------------------------------
// A bin of B^3 cells reads and deposits through a TL^3 node tile, TL = B + 1.
// gather from the staged node-field tile; t0 = tile index of the cell's corner 0
template <int TL>
PF_D void gather_tile(const float4* Et, int t0, const WF& w, float& ex, float& ey, float& ez) {
    ex = 0.f; ey = 0.f; ez = 0.f;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
        const float4 e = Et[t0 + tile_corner<TL>(l)];
        ex += w.w[l] * e.x;
        ey += w.w[l] * e.y;
        ez += w.w[l] * e.z;
    }
}

template <int TL>
PF_D int tile_index(int i, int j, int k, int x0, int y0, int z0) {
    return (i - x0) + TL * ((j - y0) + TL * (k - z0));
}

// a bin's deposit tile: 8 interleaved 32-bit copies per node (copy = lane & 7),
// units of 2^-19 particle (see k_push_bins_m).  One particle: 7 rounded
// weights and the remainder, so it adds exactly 2^19.
template <int TL>
PF_D void tile_deposit19(unsigned* Wt, int t0, const WF& w) {
    unsigned rest = 1u << 19;
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const unsigned W = __float2uint_rn(w.w[l] * 524288.0f);
        rest -= W;
        atomicAdd(&Wt[t0 + 8 * tile_corner<TL>(l)], W);
    }
    atomicAdd(&Wt[t0 + 8 * tile_corner<TL>(7)], rest);
}
// add the tile to the node charges (2^32 units per particle), all threads of the block
template <int TL>
PF_D void tile_flush19(const Launch& L, unsigned long long* W, const unsigned* Wt, int x0, int y0, int z0) {
    for (int t = threadIdx.x; t < TL * TL * TL; t += blockDim.x) {
        long long v = 0;
        for (int c = 0; c < 8; ++c) {
            long long u = (long long)Wt[t * 8 + c];
            if (u >= (3ll << 30)) u -= 1ll << 32;     // a (small) negative copy total
            v += u;
        }
        if (!v) continue;
        int tx = t % TL, ty = (t / TL) % TL, tz = t / (TL * TL);
        int gi = x0 + tx, gj = y0 + ty, gk = z0 + tz;
        if (gi <= L.mesh.nx && gj <= L.mesh.ny && gk <= L.mesh.nz)
            atomicAdd(&W[node_id(L.mesh, gi, gj, gk)], (unsigned long long)(v * 8192));
    }
}

// One CTA per (bin, species); warps take chunks of 32 particles in turn
// (chunk c to warp c mod 8, prefetching the next) and never wait at a block
// barrier.  Stayers are compacted in place: chunk c writes its stayers right
// after those of chunks 0..c-1.  Each chunk publishes its own stayer count in
// shared memory as soon as it has it; the warp of chunk c adds the counts of
// chunks c-7..c-1 (one per lane: the other warps' latest chunks) to its own
// running total up to chunk c-8, so no warp waits on a chain of publications.
// Writes land only on slots of chunks <= c, all of which were read before
// their counts were published, so no unread particle is overwritten.
// A warp's next PUSH_DEPTH chunks are in flight at any time: each lane copies
// its particle's seven words into the warp's stage in shared memory with
// cp.async (no registers held while the loads travel) and reads them back
// when the chunk comes up.
// HYBRID: the IFE mesh is finer than the PIC mesh, stayers deposit straight
// onto its nodes (a separate instantiation keeps the common path's registers)
constexpr int PUSH_WARPS = 8;   // 256 threads
constexpr int PUSH_DEPTH = 3;   // chunks in flight per warp

// the push's dynamic shared memory for bins of edge B: node-field tile, deposit
// tile, chunk counts, cp.async stages (in that order; every part a multiple of 16 bytes)
template <int B>
struct PushSmem {
    static constexpr int TL = B + 1, TN = TL * TL * TL;
    static constexpr size_t et = sizeof(float4) * TN;
    static constexpr size_t wt = sizeof(unsigned) * 8 * TN;
    static constexpr size_t agg = sizeof(int) * ((((BIN_MAX + 31) / 32) + 3) & ~3);
    static constexpr size_t stg = sizeof(unsigned) * PUSH_WARPS * PUSH_DEPTH * 7 * 32;
    static constexpr size_t bytes = et + wt + agg + stg;
    static_assert(et % 16 == 0 && wt % 16 == 0 && agg % 16 == 0, "16-byte parts");
};

template <bool HYBRID, int B>
__global__ void __launch_bounds__(256, 5) k_push_bins_m(Launch L, ObjF of, float dthf,
                                                     const __grid_constant__ CUtensorMap tmE) {
    using SM = PushSmem<B>;
    constexpr int TL = SM::TL, TN = SM::TN;
    extern __shared__ __align__(128) unsigned char push_smem[];
    float4* Et = reinterpret_cast<float4*>(push_smem);   // the bin's node-field tile (TMA destination)
    // deposits of the bin's stayers in units of 2^-19 particle, 8 interleaved
    // copies per node (copy = lane & 7) so that the lanes of one atomic
    // instruction spread over the banks.  A particle adds 7 rounded weights and
    // the remainder 2^19 - sum (at least -4), so a copy, reached by at most
    // BIN_MAX / 8 + 1 particles, holds a value in [-2^14, 2^31]: exact in 32
    // bits modulo 2^32.  The flush multiplies by 2^13 (2^32 units per particle).
    unsigned* Wt = reinterpret_cast<unsigned*>(push_smem + SM::et);
    // stayers of chunk c plus one, for each chunk c (0: not yet published)
    int* agg = reinterpret_cast<int*>(push_smem + SM::et + SM::wt);
    __shared__ int s_total, s_fail;   // stayers of the bin plus one; a wait gave up
    // per warp and stage: cell, fx, fy, fz, vx, vy, vz of 32 particles
    typedef unsigned Stage[PUSH_DEPTH][7][32];
    Stage* stg = reinterpret_cast<Stage*>(push_smem + SM::et + SM::wt + SM::agg);
    __shared__ alignas(8) unsigned long long bar;
    __shared__ unsigned sctr[NCTR];
    __shared__ int s_ok;
    const int s = blockIdx.y;
    const int b = blockIdx.x;
    const SpeciesDev& S = L.sp[s];
    const int n = S.bcount[b];
    if (n == 0) {
        if (threadIdx.x == 0) S.bstay[b] = 0;
        return;
    }
    const int bx = b % L.nbx, by = (b / L.nbx) % L.nby, bz = b / (L.nbx * L.nby);
    const int x0 = bx * B, y0 = by * B, z0 = bz * B;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int nch = (n + 31) >> 5;
    const long long start = S.bstart[b];
    // copies of chunk cc (this warp's) into stage slot sl; one group per call
    auto stage = [&](int cc, int sl) {
        const int ii = cc * 32 + lane;
        if (cc < nch && ii < n) {
            const long long g = start + ii;
            unsigned(&d)[7][32] = stg[wid][sl];
            cp_async4(&d[0][lane], S.binsF.cell + g);
            cp_async4(&d[1][lane], S.binsF.fx + g);
            cp_async4(&d[2][lane], S.binsF.fy + g);
            cp_async4(&d[3][lane], S.binsF.fz + g);
            cp_async4(&d[4][lane], S.binsF.vx + g);
            cp_async4(&d[5][lane], S.binsF.vy + g);
            cp_async4(&d[6][lane], S.binsF.vz + g);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < PUSH_DEPTH; ++d) stage(wid + d * nw, d);
    if (tid == 0) { mbar_init(&bar, 1); fence_barrier_init(); }
    for (int t = tid; t < 8 * TN; t += blockDim.x) Wt[t] = 0u;
    for (int t = tid; t < nch; t += blockDim.x) agg[t] = 0;
    if (tid < NCTR) sctr[tid] = 0u;
    if (tid == 0) { s_total = 0; s_fail = 0; }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bar, TN * (unsigned)sizeof(float4));
        tma_load_4d(Et, &tmE, &bar, 0, x0, y0, z0);
        bool ok = mbar_wait_bounded(&bar, 0);
        if (!ok) {
            atomicOr(L.err, ERR_TMA_TIMEOUT);
            mbar_wait_bounded(&bar, 0);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {   // (the bin is left as it was; the error flag reports it)
        cp_async_wait_all();
        if (tid == 0) S.bstay[b] = n;
        return;
    }
    const bool track = L.track;
    const float kf = (float)S.k;
    const int refl = S.reflect;
    const int copy = lane & 7;
    volatile int* vagg = agg;
    volatile int* vfail = &s_fail;
    int run = 0;   // stayers of chunks 0..c-nw (this warp's previous chunk included)
    unsigned c_push = 0, c_abs = 0, c_col = 0, c_lost = 0;
    int sl = 0;   // stage slot of the current chunk
    for (int c = wid; c < nch; c += nw) {
        const int i = c * 32 + lane;
        int code = NONE, acc = -1;
        PF32 p;
        long long id = 0;
        cp_async_wait<PUSH_DEPTH - 1>();   // this chunk's group (each lane reads only its own copies)
        {
            const unsigned(&d)[7][32] = stg[wid][sl];
            unpack_cell((int)d[0][lane], p.i, p.j, p.k);
            p.fx = __uint_as_float(d[1][lane]); p.fy = __uint_as_float(d[2][lane]);
            p.fz = __uint_as_float(d[3][lane]); p.vx = __uint_as_float(d[4][lane]);
            p.vy = __uint_as_float(d[5][lane]); p.vz = __uint_as_float(d[6][lane]);
        }
        if (track && i < n) id = S.binsF.id[start + i];
        if (i < n) {
            // kick with the field gathered at the old position, then drift
            const WF w = weights_f(p.fx, p.fy, p.fz);
            float ex, ey, ez;
            gather_tile<TL>(Et, tile_index<TL>(p.i, p.j, p.k, x0, y0, z0), w, ex, ey, ez);
            p.vx += kf * ex; p.vy += kf * ey; p.vz += kf * ez;
            const float xo = (float)p.i + p.fx, yo = (float)p.j + p.fy, zo = (float)p.k + p.fz;
            p.fx += p.vx * dthf; p.fy += p.vy * dthf; p.fz += p.vz * dthf;
            advance_axis(p.fx, p.i); advance_axis(p.fy, p.j); advance_axis(p.fz, p.k);
            if (refl) reflect_cell(L.mesh, refl, p);
            if (p.i < 0 || p.i >= L.mesh.nx || p.j < 0 || p.j >= L.mesh.ny || p.k < 0 || p.k >= L.mesh.nz) {
                code = ABSORBED;
            } else {
                const float xn = (float)p.i + p.fx, yn = (float)p.j + p.fy, zn = (float)p.k + p.fz;
                if (level_set_f(of, xn, yn, zn) < 0.0f) {
                    acc = hit_cell_f(L, of, xo, yo, zo, xn, yn, zn);
                    code = COLLECTED;
                } else {
                    code = ALIVE;
                }
            }
        }
        // refill the slot (its values have been used, so its reads are done)
        stage(c + PUSH_DEPTH * nw, sl);
        sl = sl + 1 == PUSH_DEPTH ? 0 : sl + 1;
        bool stay = false, mover = false;
        if (code == ALIVE) {
            stay = (p.i >= x0) & (p.i < x0 + B) & (p.j >= y0) & (p.j < y0 + B) & (p.k >= z0) & (p.k < z0 + B);
            mover = !stay;
            if (HYBRID && stay) {
                global_deposit_f(L, S.W, p);   // hybrid grid: straight onto the IFE nodes
            } else if (stay) {   // (movers deposit in the rebin, with every mover of the step)
                tile_deposit19<TL>(Wt, 8 * tile_index<TL>(p.i, p.j, p.k, x0, y0, z0) + copy, weights_f(p.fx, p.fy, p.fz));
            }
        } else if (code == COLLECTED) {
            if (acc >= 0) atomicAdd(&S.surf[acc], 1ull);
        }
        c_push += code != NONE;
        c_abs += code == ABSORBED;
        c_col += code == COLLECTED;
        c_lost += code == COLLECTED && acc < 0;
        // publish this chunk's count, then add those of chunks c-7..c-1 (bounded waits)
        const unsigned bal = __ballot_sync(0xffffffffu, stay);
        if (lane == 0) vagg[c] = __popc(bal) + 1;
        unsigned got = 0;
        bool ok = true;
        if (lane >= 1 && lane < nw && c - lane >= 0) {
            int v;
            long long spins = 0;
            while ((v = vagg[c - lane]) == 0)
                if (++spins > (1ll << 26) || *vfail) { ok = false; break; }
            got = ok ? (unsigned)(v - 1) : 0u;
        }
        if (!__all_sync(0xffffffffu, ok)) {   // give up: this bin's stayers are dropped
            if (lane == 0) { *vfail = 1; atomicOr(L.err, ERR_CHUNK_TIMEOUT); }
            break;
        }
        const int before = run + (int)__reduce_add_sync(0xffffffffu, got);
        run = before + __popc(bal);
        if (lane == 0 && c == nch - 1) s_total = run + 1;
        if (stay) store_p(S.binsF, start + before + __popc(bal & ((1u << lane) - 1)), p, id, track);
        long long slot = warp_reserve(S.mov_out_n, mover);
        if (mover) {
            if (slot < S.mcap) store_p(S.movF_out, slot, p, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    cp_async_wait_all();   // (a warp that gave up may still have copies in flight)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_push += __shfl_xor_sync(0xffffffffu, c_push, o);
        c_abs += __shfl_xor_sync(0xffffffffu, c_abs, o);
        c_col += __shfl_xor_sync(0xffffffffu, c_col, o);
        c_lost += __shfl_xor_sync(0xffffffffu, c_lost, o);
    }
    if (lane == 0) {
        if (c_push) atomicAdd(&sctr[C_PUSHED], c_push);
        if (c_abs) atomicAdd(&sctr[C_ABSORBED], c_abs);
        if (c_col) atomicAdd(&sctr[C_COLLECTED], c_col);
        if (c_lost) atomicAdd(&sctr[C_LOST], c_lost);
    }
    __syncthreads();
    if (tid == 0) {
        S.bcount[b] = (s_fail || s_total == 0) ? 0 : s_total - 1;
        S.bstay[b] = S.bcount[b];
    }
    tile_flush19<TL>(L, S.W, Wt, x0, y0, z0);
    if (tid < NCTR && sctr[tid]) atomicAdd(&S.ctr[tid], (unsigned long long)sctr[tid]);
}

__global__ void k_push_movers_m(Launch L, ObjF of, float dthf) {
    __shared__ unsigned long long sctr[NCTR];
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    if (threadIdx.x < NCTR) sctr[threadIdx.x] = 0ull;
    __syncthreads();
    const long long n = list_len(S.mov_in_n, S.mcap);
    const EGlobalF ea{L.Ef, L.mesh};
    const bool track = L.track;
    const float kf = (float)S.k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += stride) {
        long long i = base + threadIdx.x;
        int code = NONE, acc = -1;
        PF32 p;
        long long id = 0;
        if (i < n) {
            load_p(S.movF_in, i, p);
            if (track) id = S.movF_in.id[i];
            code = push_one(L, of, kf, dthf, S.reflect, p, ea, acc);
            if (code == COLLECTED && acc >= 0) atomicAdd(&S.surf[acc], 1ull);
        }
        count_event(&sctr[C_PUSHED], code != NONE);
        count_event(&sctr[C_ABSORBED], code == ABSORBED);
        count_event(&sctr[C_COLLECTED], code == COLLECTED);
        count_event(&sctr[C_LOST], code == COLLECTED && acc < 0);
        bool alive = code == ALIVE;
        long long slot = warp_reserve(S.mov_out_n, alive);
        if (alive) {
            if (slot < S.mcap) store_p(S.movF_out, slot, p, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

// injection: FP32 sampling (same random streams as the FP64 path) and FP32
// tests, stored as cell + FP32 offset
__global__ void k_inject_m(Launch L, InjArgs a, ObjF of, float dthf) {
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
    const float nxf = (float)L.mesh.nx, nyf = (float)L.mesh.ny, nzf = (float)L.mesh.nz;
    for (int base = blockIdx.x * blockDim.x; base < cnt; base += gridDim.x * blockDim.x) {
        int mm = base + threadIdx.x;
        int code = NONE, acc = -1;
        bool rejected = false;
        PF32 p;
        if (mm < cnt) {
            // FP32 sample (the MIXED state is FP32); tests on the FP32 level set
            InjSampleF sm = inject_sample_f(d, mm, *a.step, s, L.mesh, dthf);
            if (S.reflect) {
                reflect_axis_pf(sm.p[0], sm.v[0], L.mesh.nx, S.reflect & 1, S.reflect & 2);
                reflect_axis_pf(sm.p[1], sm.v[1], L.mesh.ny, S.reflect & 4, S.reflect & 8);
                reflect_axis_pf(sm.p[2], sm.v[2], L.mesh.nz, S.reflect & 16, S.reflect & 32);
            }
            if (!sm.ok || level_set_f(of, sm.p0[0], sm.p0[1], sm.p0[2]) < 0.0f) {
                rejected = true;
            } else if (sm.p[0] < 0.0f || sm.p[0] >= nxf || sm.p[1] < 0.0f || sm.p[1] >= nyf || sm.p[2] < 0.0f ||
                       sm.p[2] >= nzf) {
                code = ABSORBED;
            } else {
                const float fi = floorf(sm.p[0]), fj = floorf(sm.p[1]), fk = floorf(sm.p[2]);
                p.i = (int)fi; p.j = (int)fj; p.k = (int)fk;
                p.fx = sm.p[0] - fi; p.fy = sm.p[1] - fj; p.fz = sm.p[2] - fk;
                if (p.fx >= 1.0f) p.fx = 0.99999994f;
                if (p.fy >= 1.0f) p.fy = 0.99999994f;
                if (p.fz >= 1.0f) p.fz = 0.99999994f;
                p.vx = sm.v[0]; p.vy = sm.v[1]; p.vz = sm.v[2];
                if (level_set_f(of, sm.p[0], sm.p[1], sm.p[2]) < 0.0f) {
                    acc = hit_cell_f(L, of, sm.p0[0], sm.p0[1], sm.p0[2], sm.p[0], sm.p[1], sm.p[2]);
                    code = COLLECTED;
                    if (acc >= 0) atomicAdd(&S.surf[acc], 1ull);
                } else {
                    code = ALIVE;   // deposits in the rebin
                }
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
            if (slot < S.mcap) store_p(S.movF_out, slot, p, idb + mm, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

// rebin: every particle of this step's mover list (bin leavers of the push,
// survivors of the spill list, injected and photoemitted particles) deposits
// its charge here, in one warp-coherent pass, then joins its bin or, if the
// bin is full, next step's spill list
// DEFER: a mover stored into a bin deposits later with the bin's other arrivals
// (k_deposit_arrivals_m); one that waits in the list deposits here
template <bool DEFER>
__global__ void k_rebin_m(Launch L) {
    const int s = blockIdx.y;
    const SpeciesDev& S = L.sp[s];
    const long long n = list_len(S.mov_out_n, S.mcap);
    const bool track = L.track;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += stride) {
        long long i = base + threadIdx.x;
        bool spill = false;
        PF32 p;
        long long id = 0;
        if (i < n) {
            load_p(S.movF_out, i, p);
            if (track) id = S.movF_out.id[i];
            int b = block_of(L, p.i, p.j, p.k);
            int slot = warp_inc(&S.bcount[b]);
            if (slot < S.bcap[b]) store_p(S.binsF, S.bstart[b] + slot, p, id, track);
            else spill = true;
            if (!DEFER || spill) global_deposit_f(L, S.W, p);
        }
        long long slot = warp_reserve(S.mov_in_n, spill);
        if (spill) {
            if (slot < S.mcap) store_p(S.movF_in, slot, p, id, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
}

// FP64 flat list -> MIXED bins (load, explicit particles, rebuild)
__global__ void k_bin_scatter_m(Launch L, int s, PArr a, long long n, bool track) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SpeciesDev& S = L.sp[s];
    double fi = floor(a.x[i]), fj = floor(a.y[i]), fk = floor(a.z[i]);
    PF32 p;
    p.i = (int)fi; p.j = (int)fj; p.k = (int)fk;
    p.fx = (float)(a.x[i] - fi); p.fy = (float)(a.y[i] - fj); p.fz = (float)(a.z[i] - fk);
    if (p.fx >= 1.0f) p.fx = 0.99999994f;
    if (p.fy >= 1.0f) p.fy = 0.99999994f;
    if (p.fz >= 1.0f) p.fz = 0.99999994f;
    p.vx = (float)a.vx[i]; p.vy = (float)a.vy[i]; p.vz = (float)a.vz[i];
    int b = block_of(L, p.i, p.j, p.k);
    int slot = warp_inc(&S.bcount[b]);
    long long id = track ? a.id[i] : 0;
    if (slot < S.bcap[b]) {
        store_p(S.binsF, S.bstart[b] + slot, p, id, track);
    } else {   // a full bin: the particle waits in the mover list
        unsigned long long q = atomicAdd(S.mov_in_n, 1ull);
        if ((long long)q < S.mcap) store_p(S.movF_in, (long long)q, p, id, track);
        else atomicAdd(&S.ctr[C_DROPPED], 1ull);
    }
}

PF_D void put_d(const PArr& o, long long g, const PF32& p, long long id, bool track) {
    o.x[g] = (double)p.i + (double)p.fx; o.y[g] = (double)p.j + (double)p.fy; o.z[g] = (double)p.k + (double)p.fz;
    o.vx[g] = p.vx; o.vy[g] = p.vy; o.vz[g] = p.vz;
    if (track) o.id[g] = id;
}

__global__ void k_flatten_m(Launch L, int s, PArr out, unsigned long long* nout) {
    const SpeciesDev& S = L.sp[s];
    int b = blockIdx.x;
    int n = S.bcount[b];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = n ? atomicAdd(nout, (unsigned long long)n) : 0ull;
    __syncthreads();
    long long st = S.bstart[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        PF32 p;
        load_p(S.binsF, st + i, p);
        put_d(out, (long long)base + i, p, L.track ? S.binsF.id[st + i] : 0, true);
    }
}

__global__ void k_flatten_list_m(Launch L, int s, PArr out, unsigned long long* nout) {
    const SpeciesDev& S = L.sp[s];
    long long n = list_len(S.mov_in_n, S.mcap);
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = n ? atomicAdd(nout, (unsigned long long)n) : 0ull;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        PF32 p;
        load_p(S.movF_in, i, p);
        put_d(out, (long long)base + i, p, L.track ? S.movF_in.id[i] : 0, true);
    }
}

// every binned particle's deposit (a full recount of the node charges) with
// the 2^-32 weights of global_deposit_f: on the PIC mesh through a shared tile
// of split 32-bit counters (tile_deposit; integer sums, so the node charges
// equal those of one global atomic per weight), on a finer IFE mesh straight
// to its nodes
template <bool HYBRID, int B>
__global__ void k_deposit_bins_m(Launch L) {
    constexpr int TL = B + 1, TN = TL * TL * TL;
    __shared__ int Wlo[8 * TN];
    __shared__ int Whi[8 * TN];
    const SpeciesDev& S = L.sp[blockIdx.y];
    const int b = blockIdx.x;
    const int n = S.bcount[b];
    if (n == 0) return;
    const long long st = S.bstart[b];
    if (HYBRID) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            PF32 p;
            load_p(S.binsF, st + i, p);
            global_deposit_f(L, S.W, p);
        }
        return;
    }
    const int bx = b % L.nbx, by = (b / L.nbx) % L.nby, bz = b / (L.nbx * L.nby);
    const int x0 = bx * B, y0 = by * B, z0 = bz * B;
    for (int t = threadIdx.x; t < 8 * TN; t += blockDim.x) { Wlo[t] = 0; Whi[t] = 0; }
    __syncthreads();
    const int copy = threadIdx.x & 7;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        PF32 p;
        load_p(S.binsF, st + i, p);
        long long Wf[8];
        fixed_weights_f(weights_f(p.fx, p.fy, p.fz), Wf);
        unsigned W7[7];
#pragma unroll
        for (int l = 0; l < 7; ++l) W7[l] = (unsigned)Wf[l];
        tile_deposit<unsigned, TL>(Wlo, Whi, 8 * tile_index<TL>(p.i, p.j, p.k, x0, y0, z0) + copy, W7);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TN; t += blockDim.x) {
        long long v = 0;
        for (int c = 0; c < 8; ++c) v += tile_value(Wlo[t * 8 + c], Whi[t * 8 + c]);
        if (!v) continue;
        const int tx = t % TL, ty = (t / TL) % TL, tz = t / (TL * TL);
        const int gi = x0 + tx, gj = y0 + ty, gk = z0 + tz;
        if (gi <= L.mesh.nx && gj <= L.mesh.ny && gk <= L.mesh.nz)
            atomicAdd(&S.W[node_id(L.mesh, gi, gj, gk)], (unsigned long long)v);
    }
}
__global__ void k_deposit_list_m(Launch L) {
    const SpeciesDev& S = L.sp[blockIdx.y];
    long long n = list_len(S.mov_in_n, S.mcap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        PF32 p;
        load_p(S.movF_in, i, p);
        global_deposit_f(L, S.W, p);
    }
}

__global__ void k_half_kick_bins_m(Launch L) {
    const SpeciesDev& S = L.sp[blockIdx.y];
    int b = blockIdx.x;
    int n = S.bcount[b];
    long long st = S.bstart[b];
    const EGlobalF ea{L.Ef, L.mesh};
    const float kh = (float)S.khalf;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        PF32 p;
        load_p(S.binsF, st + i, p);
        float ex, ey, ez;
        gather_f(p.i, p.j, p.k, weights_f(p.fx, p.fy, p.fz), ea, ex, ey, ez);
        S.binsF.vx[st + i] = p.vx - kh * ex;
        S.binsF.vy[st + i] = p.vy - kh * ey;
        S.binsF.vz[st + i] = p.vz - kh * ez;
    }
}
__global__ void k_half_kick_list_m(Launch L) {
    const SpeciesDev& S = L.sp[blockIdx.y];
    long long n = list_len(S.mov_in_n, S.mcap);
    const EGlobalF ea{L.Ef, L.mesh};
    const float kh = (float)S.khalf;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        PF32 p;
        load_p(S.movF_in, i, p);
        float ex, ey, ez;
        gather_f(p.i, p.j, p.k, weights_f(p.fx, p.fy, p.fz), ea, ex, ey, ez);
        S.movF_in.vx[i] = p.vx - kh * ex;
        S.movF_in.vy[i] = p.vy - kh * ey;
        S.movF_in.vz[i] = p.vz - kh * ez;
    }
}

// ------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------
static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t set_mixed_tables(const TetTables&) { return cudaSuccess; }

static InjArgs inj_args_m(Ctx& c) {
    InjArgs a;
    a.st = c.inj_dev; a.nst = (int)c.inj.size();
    a.count = c.inj_count; a.idbase = c.inj_base; a.carry = c.inj_carry; a.next_id = c.next_id;
    a.step = (const long long*)(c.scal + 42);
    return a;
}

__global__ void k_inject_counts(InjArgs a);   // particles.cu
__global__ void k_step_advance(long long* step);

// one push launch; the kernel's dynamic shared-memory limit is raised once
// to what bins of edge B need (above the 48 KB default at B = 8)
template <bool HYBRID, int B>
static cudaError_t push_bins_m(dim3 grid, cudaStream_t st, const Launch& L, const ObjF& of, float dthf,
                               const CUtensorMap& tm) {
    static_assert(PushSmem<B>::bytes <= 200 * 1024, "push shared memory");
    void* kern = (void*)k_push_bins_m<HYBRID, B>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PushSmem<B>::bytes);
    if (e != cudaSuccess) return e;
    k_push_bins_m<HYBRID, B><<<grid, 256, PushSmem<B>::bytes, st>>>(L, of, dthf, tm);
    return cudaGetLastError();
}

// what precedes a push: the step's mover-list counts and node charges start at zero
cudaError_t launch_push_prep_mixed(Ctx& c) {
    int ns = (int)c.sp.size();
    for (int s = 0; s < ns; ++s) cudaMemsetAsync(c.sp[s].mov_n + 1, 0, sizeof(unsigned long long), c.stream);
    cudaMemsetAsync(c.Wall, 0, sizeof(unsigned long long) * ns * c.mesh.nnodes, c.stream);
    return cudaGetLastError();
}

cudaError_t launch_push_mixed(Ctx& c) {
    cudaError_t e = launch_push_prep_mixed(c);
    return e == cudaSuccess ? launch_push_bins_mixed(c) : e;
}

cudaError_t launch_push_bins_mixed(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    const dim3 grid(c.nblocks, ns);
    const ObjF of = obj_f(c.obj);
    const float dthf = (float)c.dth;
    cudaError_t e;
    if (c.bin_edge == 8)
        e = c.refine == 1 ? push_bins_m<false, 8>(grid, c.stream, L, of, dthf, c.tmapEf)
                          : push_bins_m<true, 8>(grid, c.stream, L, of, dthf, c.tmapEf);
    else
        e = c.refine == 1 ? push_bins_m<false, 4>(grid, c.stream, L, of, dthf, c.tmapEf)
                          : push_bins_m<true, 4>(grid, c.stream, L, of, dthf, c.tmapEf);
    c.launches += 1;
    return e;
}

cudaError_t launch_movers_mixed(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    k_push_movers_m<<<dim3(152, ns), 256, 0, c.stream>>>(L, obj_f(c.obj), (float)c.dth);
    c.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_photo_mixed(Ctx& c);

cudaError_t launch_inject_mixed(Ctx& c) {
    if (!c.inj.empty()) {
        Launch L = make_launch(c);
        InjArgs a = inj_args_m(c);
        k_inject_counts<<<1, 32, 0, c.stream>>>(a);
        int maxc = 1;
        for (auto& d : c.inj) maxc = d.maxcnt > maxc ? d.maxcnt : maxc;
        unsigned gx = (unsigned)((maxc + 255) / 256);
        if (gx > 1024) gx = 1024;
        k_inject_m<<<dim3(gx, (unsigned)c.inj.size()), 256, 0, c.stream>>>(L, a, obj_f(c.obj), (float)c.dth);
        c.launches += 2;
    }
    return launch_photo_mixed(c);
}

// ---- photoelectron emission (MIXED state) ----------------------------------
// The emitted counts are small, so the sample is taken in FP64 exactly as on the
// FP64 path and then stored as cell + FP32 offset.
PhotoArgs photo_args(Ctx& c);                 // particles.cu
cudaError_t launch_photo_counts(Ctx& c);
__global__ void k_photo_ids(long long* next_id, const long long* total);

__global__ void k_photo_m(Launch L, PhotoArgs a) {
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
        PF32 p;
        if (m < total) {
            const PhotoDev& d = a.tets[photo_tet_of(a.base, a.ne, m)];
            PhotoSample sm = photo_sample(d, (unsigned long long)m, a.seed, key1, a.vth, a.dth);
            for (int c = 0; c < 3; ++c) sm.p[c] *= a.inv_r;   // IFE to PIC cell units (exact)
            if (S.reflect) reflect_d(L.mesh, S.reflect, sm.p[0], sm.p[1], sm.p[2], sm.v[0], sm.v[1], sm.v[2]);
            emitted = sm.ok && !(level_set(L.obj, sm.p[0], sm.p[1], sm.p[2]) < 0.0);
            if (emitted) {
                atomicAdd(&S.surf[d.acc], (unsigned long long)-1ll);   // the electron leaves +e behind
                out = (sm.p[0] < 0.0) | (sm.p[0] >= (double)L.mesh.nx) | (sm.p[1] < 0.0) |
                      (sm.p[1] >= (double)L.mesh.ny) | (sm.p[2] < 0.0) | (sm.p[2] >= (double)L.mesh.nz);
                alive = !out;
                if (alive) {
                    const double fi = floor(sm.p[0]), fj = floor(sm.p[1]), fk = floor(sm.p[2]);
                    p.i = (int)fi; p.j = (int)fj; p.k = (int)fk;
                    p.fx = (float)(sm.p[0] - fi); p.fy = (float)(sm.p[1] - fj); p.fz = (float)(sm.p[2] - fk);
                    if (p.fx >= 1.0f) p.fx = 0.99999994f;
                    if (p.fy >= 1.0f) p.fy = 0.99999994f;
                    if (p.fz >= 1.0f) p.fz = 0.99999994f;
                    p.vx = (float)sm.v[0]; p.vy = (float)sm.v[1]; p.vz = (float)sm.v[2];   // deposits in the rebin
                }
            }
        }
        count_event(&sctr[C_INJECTED], emitted);
        count_event(&sctr[C_REJECTED], m < total && !emitted);
        count_event(&sctr[C_ABSORBED], out);
        long long slot = warp_reserve(S.mov_out_n, alive);
        if (alive) {
            if (slot < S.mcap) store_p(S.movF_out, slot, p, idb + m, track);
            else atomicAdd(&S.ctr[C_DROPPED], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < NCTR && sctr[threadIdx.x]) atomicAdd(&S.ctr[threadIdx.x], sctr[threadIdx.x]);
}

cudaError_t launch_photo_mixed(Ctx& c) {
    if (c.ph_species < 0 || c.ph_ne <= 0) return cudaSuccess;
    cudaError_t e = launch_photo_counts(c);
    if (e != cudaSuccess) return e;
    k_photo_m<<<4 * 152, 256, 0, c.stream>>>(make_launch(c), photo_args(c));
    k_photo_ids<<<1, 1, 0, c.stream>>>(c.next_id + c.ph_species, c.ph_total);
    c.launches += 2;
    return cudaGetLastError();
}

// the bin's arrivals of this step, slots [bstay, bcount), deposit through a
// shared tile of split 32-bit counters with the 2^-32 weights of
// global_deposit_f (integer sums: the node charges equal those of one global
// atomic per weight, with an eighth of the global atomics or fewer)
template <int B>
__global__ void k_deposit_arrivals_m(Launch L) {
    constexpr int TL = B + 1, TN = TL * TL * TL;
    __shared__ int Wlo[8 * TN];
    __shared__ int Whi[8 * TN];
    const SpeciesDev& S = L.sp[blockIdx.y];
    const int b = blockIdx.x;
    const int n0 = S.bstay[b], n1 = S.bcount[b];   // (bcount clamped to the capacity)
    if (n1 <= n0) return;
    const long long st = S.bstart[b];
    const int bx = b % L.nbx, by = (b / L.nbx) % L.nby, bz = b / (L.nbx * L.nby);
    const int x0 = bx * B, y0 = by * B, z0 = bz * B;
    for (int t = threadIdx.x; t < 8 * TN; t += blockDim.x) { Wlo[t] = 0; Whi[t] = 0; }
    __syncthreads();
    const int copy = threadIdx.x & 7;
    for (int i = n0 + threadIdx.x; i < n1; i += blockDim.x) {
        PF32 p;
        load_p(S.binsF, st + i, p);
        long long Wf[8];
        fixed_weights_f(weights_f(p.fx, p.fy, p.fz), Wf);
        unsigned W7[7];
#pragma unroll
        for (int l = 0; l < 7; ++l) W7[l] = (unsigned)Wf[l];
        tile_deposit<unsigned, TL>(Wlo, Whi, 8 * tile_index<TL>(p.i, p.j, p.k, x0, y0, z0) + copy, W7);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TN; t += blockDim.x) {
        long long v = 0;
        for (int c = 0; c < 8; ++c) v += tile_value(Wlo[t * 8 + c], Whi[t * 8 + c]);
        if (!v) continue;
        const int tx = t % TL, ty = (t / TL) % TL, tz = t / (TL * TL);
        const int gi = x0 + tx, gj = y0 + ty, gk = z0 + tz;
        if (gi <= L.mesh.nx && gj <= L.mesh.ny && gk <= L.mesh.nz)
            atomicAdd(&S.W[node_id(L.mesh, gi, gj, gk)], (unsigned long long)v);
    }
}

cudaError_t launch_rebin_mixed(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    for (int s = 0; s < ns; ++s) cudaMemsetAsync(c.sp[s].mov_n, 0, sizeof(unsigned long long), c.stream);
    const bool defer = c.refine == 1;   // (a finer IFE mesh takes the deposits node by node)
    if (defer) k_rebin_m<true><<<dim3(4 * 152, ns), 256, 0, c.stream>>>(L);
    else k_rebin_m<false><<<dim3(4 * 152, ns), 256, 0, c.stream>>>(L);
    k_clamp_counts<<<dim3(nb(c.nblocks), ns), 256, 0, c.stream>>>(L);
    if (defer) {
        if (c.bin_edge == 8) k_deposit_arrivals_m<8><<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L);
        else k_deposit_arrivals_m<4><<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L);
    }
    k_step_advance<<<1, 1, 0, c.stream>>>((long long*)(c.scal + 42));
    c.launches += defer ? 4 : 3;
    return cudaGetLastError();
}

cudaError_t launch_deposit_all_mixed(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    cudaMemsetAsync(c.Wall, 0, sizeof(unsigned long long) * MAX_SPECIES * c.mesh.nnodes, c.stream);
    if (ns == 0) return cudaGetLastError();
    const dim3 grid(c.nblocks, ns);
    if (c.bin_edge == 8) {
        if (c.refine > 1) k_deposit_bins_m<true, 8><<<grid, 256, 0, c.stream>>>(L);
        else k_deposit_bins_m<false, 8><<<grid, 256, 0, c.stream>>>(L);
    } else {
        if (c.refine > 1) k_deposit_bins_m<true, 4><<<grid, 256, 0, c.stream>>>(L);
        else k_deposit_bins_m<false, 4><<<grid, 256, 0, c.stream>>>(L);
    }
    k_deposit_list_m<<<dim3(64, ns), 256, 0, c.stream>>>(L);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_half_kick_mixed(Ctx& c) {
    Launch L = make_launch(c);
    int ns = (int)c.sp.size();
    if (ns == 0) return cudaSuccess;
    k_half_kick_bins_m<<<dim3(c.nblocks, ns), 256, 0, c.stream>>>(L);
    k_half_kick_list_m<<<dim3(64, ns), 256, 0, c.stream>>>(L);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_flatten_mixed_to_f64(Ctx& c, int s, PArr flat, unsigned long long* nflat) {
    Launch L = make_launch(c);
    if (c.sp[s].bcount) k_flatten_m<<<c.nblocks, 256, 0, c.stream>>>(L, s, flat, nflat);
    if (c.sp[s].mov_n) k_flatten_list_m<<<1, 256, 0, c.stream>>>(L, s, flat, nflat);
    return cudaGetLastError();
}

void free_parrf(PArrF& a) {
    if (a.base) {
        lib_free(a.base);
    } else {
        lib_free(a.cell); lib_free(a.fx); lib_free(a.fy); lib_free(a.fz); lib_free(a.vx); lib_free(a.vy);
        lib_free(a.vz); lib_free(a.id);
    }
    a = PArrF{};
}

// the seven 4-byte arrays (and 8-byte ids first, for their alignment) in one allocation
cudaError_t alloc_parrf(PArrF& a, long long n, bool id) {
    free_parrf(a);
    const size_t m = (size_t)(n > 0 ? n : 1);
    const size_t mid = id ? sizeof(long long) * m : 0;
    char* b = nullptr;
    cudaError_t e = lib_malloc(&b, mid + 7 * sizeof(float) * m);
    if (e != cudaSuccess) return e;
    a.base = b;
    if (id) a.id = (long long*)b;
    char* f = b + mid;
    a.cell = (int*)f;
    float** arr[6] = {&a.fx, &a.fy, &a.fz, &a.vx, &a.vy, &a.vz};
    for (int d = 0; d < 6; ++d) *arr[d] = (float*)(f + sizeof(float) * m * (d + 1));
    return cudaSuccess;
}

// (re)build MIXED bins of species s from a flat FP64 list of n particles
cudaError_t launch_build_bins_mixed(Ctx& c, int s, PArr flat, long long n, bool) {
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
        lib_malloc(&q.bstay, sizeof(int) * c.nblocks);
    }
    cudaMemsetAsync(q.bstay, 0, sizeof(int) * c.nblocks, c.stream);
    k_bin_caps<<<nb(c.nblocks), 256, 0, c.stream>>>(c.nblocks, cnt, q.bcap, q.bcount);
    k_bin_scan<<<1, BIN_SCAN_THREADS, 0, c.stream>>>(c.nblocks, q.bcap, q.bstart, tot);
    e = cudaMemcpyAsync(&total, tot, sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) { lib_free(cnt); lib_free(tot); return e; }
    if (total > q.cap) {
        e = alloc_parrf(q.binsF, total, c.track != 0);
        if (e != cudaSuccess) { lib_free(cnt); lib_free(tot); return e; }
        q.cap = total;
    }
    L = make_launch(c);
    cudaMemsetAsync(q.mov_n, 0, 2 * sizeof(unsigned long long), c.stream);
    if (n > 0) k_bin_scatter_m<<<nb(n), 256, 0, c.stream>>>(L, s, flat, n, c.track != 0);
    k_clamp_counts<<<dim3(nb(c.nblocks), (unsigned)c.sp.size()), 256, 0, c.stream>>>(L);
    e = cudaStreamSynchronize(c.stream);
    lib_free(cnt);
    lib_free(tot);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace pf
