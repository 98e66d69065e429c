// Grid-wide synchronisation of the persistent PCG kernels (pcg_coop.cu,
// pcg_mg.cu): deterministic exchanges of block partials over a monotonic
// arrival counter, the fixed-point exchange of the FP32 inner loops, and a
// plain grid barrier.  Every wait is bounded (about a second at 2 GHz); a
// timeout sets ERR_BARRIER_TIMEOUT and the caller ends its solve.
#pragma once
#include "field_common.cuh"
#include "internal.h"

namespace pf {

struct ExchShared {
    double sh[4 * 32];
    double bc[4];
    int ok;
};

// grid exchange number e: publish this block's NV partials, wait for every
// block, return the grid totals (same in every block); false after a timeout.
// The barrier is one monotonic counter: each block adds 1 with release
// semantics and waits (acquire) until the count reaches the next multiple of
// the grid size -- no generation word, no reset, one atomic per block.
template <typename A, int NV, typename Args>
static __device__ __forceinline__ bool exchange(const Args& a, int& e, A (&v)[NV], A (&tot)[NV], ExchShared& xs) {
    A* sh = (A*)xs.sh;
    block_sum_t<A, NV>(v, sh);                // ends with __syncthreads: the block's z stores are issued
    const unsigned G = gridDim.x;
    A* val = (A*)a.val + (size_t)(e & 1) * 4 * G;
    const bool first_of_launch = e == 0;
    ++e;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) __stcg(val + (size_t)q * G + blockIdx.x, v[q]);
        const unsigned long long t = atom_add_release(a.arrivals, 1ull);
        // (a test can make the launch's first exchange wait for arrivals that
        // never come, to see the bounded wait give up and report)
        const unsigned long long target = (t / G + 1) * G + (first_of_launch ? (unsigned long long)*a.hold : 0ull);
        int ok = 1;
        if (ld_acquire(a.arrivals) < target) {
            const long long c0 = clock64();
            while (ld_acquire(a.arrivals) < target)
                if (clock64() - c0 > (1ll << 31)) { ok = 0; atomicOr(a.err, ERR_BARRIER_TIMEOUT); break; }
        }
        xs.ok = ok;
    }
    __syncthreads();
    if (!xs.ok) return false;
    A s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = threadIdx.x < G ? __ldcg(val + (size_t)q * G + threadIdx.x) : (A)0;
    block_sum_t<A, NV>(s, sh);
    A* bc = (A*)xs.bc;
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) bc[q] = s[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = bc[q];
    return true;
}

// ---- fixed-point exchange (FP32 inner loop of the register-resident kernel) ----
//
// The arrival and the partial travel in one fire-and-forget atomic: a block
// adds to one 64-bit word per value
//     (rint(v 2^k) << 2W) + (fits ? 1 : 1 + 2^W)
// -- bits 0..W-1 count arrivals, bits W..2W-1 blocks whose scaled partial did
// not fit, bits 2W..63 the two's-complement sum.  W = 8 (at most 255 blocks):
// partials below 2^39, a 48-bit sum, the scale 2^k puts the value's previous
// total near 2^32; W = 9 (at most 511 blocks): partials below 2^36, a 46-bit
// sum, previous total near 2^29.  No field carries into the next within one
// exchange.  A block polls the word until its growth since the previous use
// shows every arrival; the growth then holds the integer total, each partial
// exact to 2^-32 (2^-29) of the previous total.  Integer sums do not depend on the
// arrival order: results stay deterministic run to run.  A word is reused only
// after the other exchange kind (a full barrier) has passed, so its value is
// stable from the last arrival until every block has read it.  If a partial
// did not fit, or the total kept fewer than 2^26 (2^23) units (the value fell
// far below its previous total), every block sees it and redoes the values
// with the partial exchange above.
constexpr int FX_LINE = 16;                  // words per 128-byte line
template <int W>
struct FxLayout {
    static_assert(W == 8 || W == 9, "layouts for up to 255 or 511 blocks");
    static constexpr int SUM = 2 * W;                                        // sum field shift
    static constexpr unsigned long long MASK = (1ull << W) - 1;
    static constexpr float FIT = W == 8 ? 549755813888.0f : 68719476736.0f;   // 2^39, 2^36
    static constexpr int SCALE = W == 8 ? 32 : 29;
    static constexpr long long MIN = W == 8 ? (1ll << 26) : (1ll << 23);
};

// ref: the previous totals (positive, normal); prev: this lane's word value
// after its last use (lanes 0..NV-1 of warp 0).  Returns 1 with the totals in
// tot, -1 if the values must be redone, 0 after a timeout.
template <int NV, bool REL, int W, typename Args>
static __device__ __forceinline__ int exchange_fx(const Args& a, unsigned long long* words, unsigned long long& prev,
                                                  const float (&ref)[NV], float (&v)[NV], float (&tot)[NV],
                                                  ExchShared& xs) {
    block_sum_t<float, NV>(v, (float*)xs.sh);   // totals in thread 0; ends with __syncthreads
    float* bc = (float*)xs.bc;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const bool act = lane < NV;
        float mine = 0.0f, rf = ref[0];
#pragma unroll
        for (int q = 0; q < NV; ++q) {      // lane q takes value q (the block total sits in thread 0)
            const float t = __shfl_sync(0xffffffffu, v[q], 0);
            if (lane == q) { mine = t; rf = ref[q]; }
        }
        using FL = FxLayout<W>;
        const int k = FL::SCALE - ilogbf(rf);
        const float sc = ldexpf(mine, k);
        const bool fits = fabsf(sc) < FL::FIT;
        const long long fx = fits ? __float2ll_rn(sc) : 0ll;
        unsigned long long* w = words + lane * FX_LINE;
        if (act) {
            const unsigned long long add = ((unsigned long long)fx << FL::SUM) + (fits ? 1ull : 1ull + (1ull << W));
            if (REL) red_add_release(w, add);
            else red_add_relaxed(w, add);
        }
        const unsigned long long G = gridDim.x;
        unsigned long long d = 0;
        bool done = !act, timeout = false;
        const long long c0 = clock64();
        for (;;) {
            if (!done) {
                d = ld_acquire(w) - prev;
                done = (d & FL::MASK) == G;
            }
            if (__all_sync(0xffffffffu, done)) break;
            if (__any_sync(0xffffffffu, clock64() - c0 > (1ll << 31))) { timeout = true; break; }
        }
        bool good = true;
        if (act && !timeout) {
            prev += d;
            const long long val = (long long)d >> FL::SUM;
            good = ((d >> W) & FL::MASK) == 0 && (val >= FL::MIN || val <= -FL::MIN);
            bc[lane] = ldexpf((float)val, -k);
        }
        const bool all_good = __all_sync(0xffffffffu, good);
        if (lane == 0) {
            if (timeout) atomicOr(a.err, ERR_BARRIER_TIMEOUT);
            xs.ok = timeout ? 0 : (all_good ? 1 : 2);
        }
    }
    __syncthreads();
    // (the next exchange rewrites bc and ok only after its block sum's barrier)
    const int ok = xs.ok;
    if (ok == 1) {
#pragma unroll
        for (int q = 0; q < NV; ++q) tot[q] = bc[q];
    }
    return ok == 1 ? 1 : (ok == 2 ? -1 : 0);
}

// an FP32 exchange: fixed-point when the previous totals give a scale, else
// (or when the fixed-point totals cannot be trusted) the partial exchange
template <int NV, bool REL, int W, typename Args>
static __device__ __forceinline__ bool exchange_f32(const Args& a, int& e, unsigned long long* words,
                                                    unsigned long long& prev, const float (&ref)[NV], bool use_fx,
                                                    float (&v)[NV], float (&tot)[NV], ExchShared& xs) {
    if (use_fx) {
        float vc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) vc[q] = v[q];
        const int rc = exchange_fx<NV, REL, W>(a, words, prev, ref, vc, tot, xs);
        if (rc == 1) return true;
        if (rc == 0) return false;
    }
    return exchange<float, NV>(a, e, v, tot, xs);
}

// a previous total usable as the fixed-point scale
static __device__ __forceinline__ bool fx_ref_ok(float r) { return r > 1e-30f && r < 1e30f; }


// grid barrier number e (shares the arrival counter and the bounded wait of
// the exchanges, carries no values); false after a timeout.  The block's
// stores before the call are visible to every block after it returns.
template <typename Args>
static __device__ __forceinline__ bool grid_barrier(const Args& a, int& e, ExchShared& xs) {
    __syncthreads();
    const unsigned G = gridDim.x;
    const bool first_of_launch = e == 0;
    ++e;
    if (threadIdx.x == 0) {
        const unsigned long long t = atom_add_release(a.arrivals, 1ull);
        const unsigned long long target = (t / G + 1) * G + (first_of_launch ? (unsigned long long)*a.hold : 0ull);
        int ok = 1;
        if (ld_acquire(a.arrivals) < target) {
            const long long c0 = clock64();
            while (ld_acquire(a.arrivals) < target)
                if (clock64() - c0 > (1ll << 31)) { ok = 0; atomicOr(a.err, ERR_BARRIER_TIMEOUT); break; }
        }
        xs.ok = ok;
    }
    __syncthreads();
    return xs.ok != 0;
}

}  // namespace pf
