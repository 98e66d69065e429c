// Device helpers shared by the libpifepic kernels: level sets, the 5-tet
// split tables, Philox4x64-10, warp-aggregated counters, and the
// mbarrier / TMA primitives used to stage node-field tiles in shared memory.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define PF_HD __host__ __device__ __forceinline__
#define PF_D __device__ __forceinline__

namespace pf {

constexpr int BLK = 4;                    // particle bin = BLK^3 cells
constexpr int TILE = BLK + 1;             // node tile edge
constexpr int TILE_N = TILE * TILE * TILE;
constexpr int MAX_SPECIES = 8;
constexpr int NCTR = 8;                   // per-species device counters
enum { C_PUSHED = 0, C_ABSORBED, C_COLLECTED, C_LOST, C_INJECTED, C_REJECTED, C_SPILLED, C_DROPPED };
enum { ERR_TMA_TIMEOUT = 1, ERR_CAPACITY = 2, ERR_BARRIER_TIMEOUT = 4, ERR_CHUNK_TIMEOUT = 8 };

// ---------------------------------------------------------------------------
// Object level sets in cell units (Sec. 2.1 interface Gamma; L >= 0 plasma).
// Each is a fixed sequence of IEEE double operations (this translation unit
// is compiled without FMA contraction) so hit decisions are reproducible.
// ---------------------------------------------------------------------------
struct Object {
    int kind;          // 0 none, 1 sphere, 2 cap crater, 3 plane, 4 rim crater
    double a0, a1, a2, a3, a4, a5, a6, a7, a8, a9, a10, a11;
    double eps_minus, eps_plus;
    // layered object: bedrock (permittivity eps_bed) below the plane z = zb
    // (cell units) inside the object; L_b = z - zb < 0 there
    int bed;
    double zb, eps_bed;
};

PF_HD double level_set(const Object& o, double x, double y, double z) {
    if (o.kind == 1) {                       // sphere: a0..a2 centre, a3 = r^2
        double dx = x - o.a0, dy = y - o.a1, dz = z - o.a2;
        return ((dx * dx + dy * dy) + dz * dz) - o.a3;
    } else if (o.kind == 2) {                // crater: zg, xc, yc, a^2, Rs^2, zc
        double dx = x - o.a1, dy = y - o.a2;
        double r2 = dx * dx + dy * dy;
        double zs = (r2 < o.a3) ? o.a5 - sqrt(o.a4 - r2) : o.a0;
        return z - zs;
    } else if (o.kind == 3) {                // plane: n.xi - d0
        return ((o.a0 * x + o.a1 * y) + o.a2 * z) - o.a3;
    } else if (o.kind == 4) {                // rim crater (see pifepic_set_object)
        // a0, a1 centre; a2, a3, a4 inner-rim, top-rim, outer-rim radii;
        // a5 floor, a6 rim top, a11 ground heights; a7 = depth + height;
        // a8 height; a9, a10 widths of the inner wall and the outer flank
        double dx = x - o.a0, dy = y - o.a1;
        double r = sqrt(dx * dx + dy * dy);
        double zs;
        if (r <= o.a2) {
            zs = o.a5;
        } else if (r <= o.a3) {
            double t = (r - o.a2) / o.a9;
            zs = o.a5 + o.a7 * ((t * t) * (3.0 - 2.0 * t));
        } else if (r < o.a4) {
            double t = (r - o.a3) / o.a10;
            zs = o.a6 - o.a8 * ((t * t) * (3.0 - 2.0 * t));
        } else {
            zs = o.a11;
        }
        return z - zs;
    }
    return 1.0;
}
// bedrock level set of a layered object at a node of height k (cell units)
PF_HD double bed_level(const Object& o, int k) { return (double)k - o.zb; }

// ---------------------------------------------------------------------------
// Mesh and 5-tet split (reading of Sec. 3.1.1): tet 0 = the 4 vertices of the
// cube with global parity even, tets 1..4 = corner tets (o, o^1, o^2, o^4) for
// the odd vertices o.  Local vertex l = a + 2b + 4c <-> offset (a, b, c).
// ---------------------------------------------------------------------------
struct Mesh {
    int nx, ny, nz, NX, NY, NZ;
    long long nnodes, ncells;
    double h;
    // the regular stencil's h/6 and h/12, once per mesh instead of once per
    // row (the same IEEE quotients, in FP64 and from the FP32 h in FP32)
    double h6, h12;
    float h6f, h12f;
};

// Reflecting particle faces (the symmetry plane of Sec. 5.2.2), bit f of the
// mask for face f = x-, x+, y-, y+, z-, z+.  A coordinate beyond a reflecting
// face is mirrored back, xi -> -xi at the minus face and xi -> 2n - xi at the
// plus face, and the normal velocity reversed; per axis the minus face is
// tested first.  A mirror landing exactly on n (the box is [0, n)) takes the
// largest double below n (n >= 1: one less in the bit pattern).
PF_D void reflect_axis_d(double& x, double& v, int n, int lo, int hi) {
    const double nd = (double)n;
    if (lo && x < 0.0) { x = -x; v = -v; }
    if (hi && x >= nd) {
        x = (2.0 * nd) - x;
        if (x >= nd) x = __longlong_as_double(__double_as_longlong(nd) - 1);
        v = -v;
    }
}
PF_D void reflect_d(const Mesh& m, int mask, double& x, double& y, double& z, double& vx, double& vy,
                    double& vz) {
    reflect_axis_d(x, vx, m.nx, mask & 1, mask & 2);
    reflect_axis_d(y, vy, m.ny, mask & 4, mask & 8);
    reflect_axis_d(z, vz, m.nz, mask & 16, mask & 32);
}

struct TetTables {
    int vert[2][5][4];         // [cube parity][tet][k] local vertex
    double grad[2][5][4][3];   // P1 basis gradients for h = 1
    double vol[5];             // volumes for h = 1
    int slot[27];              // stencil slot of offset (dx,dy,dz), -1 if none
    int off[19][3];            // offset of each slot
};

PF_HD long long node_id(const Mesh& m, int i, int j, int k) {
    return (long long)i + (long long)m.NX * ((long long)j + (long long)m.NY * k);
}
PF_HD long long cell_id(const Mesh& m, int i, int j, int k) {
    return (long long)i + (long long)m.nx * ((long long)j + (long long)m.ny * k);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): multipliers and Weyl key increments as
// published; round: (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)).
// ---------------------------------------------------------------------------
struct U64x4 { unsigned long long v[4]; };

PF_HD void mulhilo64(unsigned long long a, unsigned long long b, unsigned long long& hi,
                     unsigned long long& lo) {
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    lo = (unsigned long long)p;
    hi = (unsigned long long)(p >> 64);
#endif
}

PF_HD U64x4 philox4x64(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                       unsigned long long c3, unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned long long hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, hi0, lo0);
        mulhilo64(M1, c2, hi1, lo1);
        unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    U64x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

PF_HD unsigned long long stream_key(int purpose, int species, int face, long long step) {
    return ((unsigned long long)purpose << 56) | ((unsigned long long)species << 48) |
           ((unsigned long long)face << 40) | ((unsigned long long)step & ((1ull << 40) - 1));
}

// open uniform from the top 52 bits; exact in double
PF_HD double u01(unsigned long long x) { return ((double)(x >> 12) + 0.5) * 2.220446049250313e-16; }

// ---------------------------------------------------------------------------
// warp-aggregated atomic increment: returns this lane's slot
// ---------------------------------------------------------------------------
PF_D long long warp_reserve(unsigned long long* counter, bool want) {
    unsigned mask = __ballot_sync(0xffffffffu, want);
    if (!want) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return (long long)(base + __popc(mask & ((1u << lane) - 1)));
}

// atomicAdd(p, 1) with one atomic per group of active lanes that share the
// address (match_any): each lane gets a distinct value, as if the lanes had
// added one by one in lane order.  Lanes hitting one counter (particles of one
// bin in a warp) no longer serialise on it.
PF_D int warp_inc(int* p) {
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, (unsigned long long)p);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(p, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + __popc(grp & ((1u << lane) - 1));
}
// the same for one counter shared by all active lanes
PF_D unsigned long long warp_inc64(unsigned long long* p) {
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(p, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    return base + __popc(act & ((1u << lane) - 1));
}

constexpr int BIN_MAX = 32767;
constexpr int BIN_SCAN_THREADS = 1024;   // k_bin_scan's block
// corner offsets in a TL^3 node tile (TL = bin edge + 1), node order
// 000,100,010,110,001,101,011,111
template <int TL = TILE>
PF_HD constexpr int tile_corner(int l) {
    return (l & 1) + TL * ((l >> 1) & 1) + TL * TL * ((l >> 2) & 1);
}

// Shared-memory fixed-point deposit of one particle with native 32-bit atomics.
// The tile keeps 8 interleaved copies per node (index 8 * node + copy; base =
// 8 * corner-0 node + copy).  W[l] (l < 7, 0 <= W[l] <= 2^32) are the rounded
// weights of corners 0..6; each goes in as its low 16 bits and its high part
// W >> 16 (two signed counters).  Corner 7 receives minus the low parts and
// 2^16 minus the high parts of the other seven: exactly 2^32 - sum W[l], the
// remainder weight, so the particle adds exactly 2^32 and every node the same
// integer as an int64 deposit.  Per copy at most BIN_MAX / 8 + 1 particles
// reach a node, each moving a counter by less than 7 * 2^16, so both counters
// stay inside 32 bits and tile_value() is exact.
template <typename WT, int TL = TILE>
PF_D void tile_deposit(int* lo, int* hi, int base, const WT (&W)[7]) {
    int slo = 0, shi = 0;
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const int a = (int)(W[l] & 0xFFFF), b = (int)(W[l] >> 16);
        atomicAdd(&lo[base + 8 * tile_corner<TL>(l)], a);
        atomicAdd(&hi[base + 8 * tile_corner<TL>(l)], b);
        slo += a;
        shi += b;
    }
    atomicAdd(&lo[base + 8 * tile_corner<TL>(7)], -slo);
    atomicAdd(&hi[base + 8 * tile_corner<TL>(7)], 65536 - shi);
}
PF_D long long tile_value(int lo, int hi) { return (long long)lo + ((long long)hi << 16); }

// warp-aggregated event count into a 32-bit shared counter
PF_D void count_event32(unsigned* c, bool ev) {
    const unsigned m = __ballot_sync(0xffffffffu, ev);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(c, (unsigned)__popc(m));
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (cp.async.bulk.tensor) helpers
// ---------------------------------------------------------------------------
PF_D unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

PF_D void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
PF_D void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
PF_D bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
PF_D void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
PF_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4-D tiled TMA load (components, x, y, z) of one node tile into shared memory
PF_D void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1, int c2,
                      int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// bounded wait on phase 0 of an mbarrier; false on timeout (~2^31 cycles)
PF_D bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

}  // namespace pf
