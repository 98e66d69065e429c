// Persistent cooperative PCG (Sec. 2.5: the matrix solve is a PCG iteration
// stopped on the relative residual; the Jacobi preconditioner is this build's
// reading).  One launch runs the whole solve: every block keeps iterating,
// separated by grid-wide exchanges, so the loop pays no kernel launches.
//
//  FP64 mode : Jacobi PCG in FP64.
//  MIXED mode: FP64 iterative refinement around FP32 Jacobi PCG solves; the
//              refinement residuals are FP64, the inner vectors, operator and
//              reductions FP32.
//
// Reductions are deterministic: each block writes its partial, and after the
// exchange every block sums all partials in the same order (or, in the FP32
// inner loop of the register-resident kernel, adds them as integers), so all
// blocks take the same decisions and two runs give identical results.
// Exchange waits are bounded (about a second); a timeout raises an error bit
// and ends the solve.
//
// Two kernels: k_pcg_reg keeps the vectors in registers (meshes with at most 8
// nodes per thread of a full grid, e.g. 64^3); k_pcg_glob keeps them in
// global memory / L2 (larger meshes, e.g. 160 x 160 x 80).
#include <math.h>

#include <type_traits>

#include "field_common.cuh"
#include "internal.h"
#include "pcg_sync.cuh"

namespace pf {

constexpr int COOP_MAX_OUTER = 12;   // MIXED: refinement steps at most
// MIXED, pipelined inner loop: an inner solve whose FP64 residual ends more
// than 30x (in norm) above its recurrence residual switches the context to the
// classic loop (the sphere meshes measure about 8x, mostly-Neumann craters 80x)
constexpr double PIPE_GAP2 = 900.0;
constexpr int PIPE_STALL = 40;

// ---- register-resident PCG --------------------------------------------------
//
// When a full-occupancy grid gives every thread at most 8 nodes, block b owns
// the contiguous nodes [b*M, (b+1)*M) and its thread t the nodes
// b*M + t + s*REG_THREADS (s < NPT); all PCG vectors of those nodes live in
// registers.  Only z = D^-1 r, which the operator reads at neighbouring nodes,
// goes through global memory (it stays in L2): before each matrix product a
// block copies the window of z its rows touch -- its own range plus one
// z-plane, one row and one node on each side, contiguous in node order -- into
// shared memory with 16-byte loads, one round trip instead of one per node.
//
// Both modes run Jacobi PCG with the q recurrence: two grid exchanges per
// iteration, one per reduction.  Inner-loop dot products, block sums and the
// scalars alpha and beta are in the working precision (FP32 in MIXED mode; the
// outer FP64 residual corrects what FP32 inner products lose).  An exchange
// is a monotonic arrival counter (below) with the block partials in one of two
// slots by exchange parity, so a block that races ahead into the next exchange
// never overwrites partials a slower block is still summing; the FP32 inner
// loop of MIXED mode uses the fixed-point exchange instead, which needs no
// second round trip for the partials.  z alternates between two copies by
// iteration parity: the update writes the copy that the previous iteration's
// staging read, whose readers the previous r.z exchange (release/acquire)
// already ordered before the writer.  So the p.q exchange orders no global
// data (the products write none) and its fixed-point atomic is relaxed: the
// release fence is about a third of an exchange's latency.  MIXED wraps FP32
// inner solves in FP64 refinement as the global-memory kernel does.  (The pipelined form of PCG would need one
// exchange per iteration, but its recurrences stagnated on meshes with mostly
// Neumann faces, in FP32 and with FP64 recurrences alike, so it is not used.)

constexpr int REG_THREADS = 512;

struct RegArgs {
    FieldArgs f;
    const double* b;
    double* u;                 // FP64 unknown (warm start in, solution out)
    const double* g;           // Dirichlet values
    double* phi;
    void* zg[2];               // exchanged vector z (T), two guarded copies
    long long M;               // nodes per block
    int woff[19];              // staged rows: window offset of each stencil slot
    double* val;               // [2][4][G] block partials
    unsigned long long* arrivals;  // grows by G per exchange
    unsigned long long* fx;        // fixed-point exchange words: pq at [0], r.r and r.z at [FX_LINE], [2 FX_LINE];
                                   // pipelined loop: two sets of three at [(3 + 3 set + q) FX_LINE]
    int* classic;                  // MIXED: 1 once a solve found the pipelined recurrences too inexact
    const int* hold;               // arrivals the launch's first exchange waits for beyond the grid (tests)
    PcgState* S;
    long long* it_total;
    long long* outer_total;
    int* err;
};

static __device__ __forceinline__ unsigned pack_ijk(int i, int j, int k) {
    return (unsigned)i | ((unsigned)j << 11) | ((unsigned)k << 22);
}
template <typename T, typename LD>
static __device__ __forceinline__ T row_at(const FieldArgs& f, long long n, unsigned pk, LD ld, const T* coef) {
    return apply_row_ld<T>(f, n, (int)(pk & 2047u), (int)((pk >> 11) & 2047u), (int)(pk >> 22), ld, coef);
}

// the window of z a block's rows read: [ws, we), both multiples of the 16-byte
// vector, we <= N rounded up (inside the padded allocation)
template <typename T>
static __host__ __device__ __forceinline__ void z_window(long long N, long long NX, long long NXY, long long b0,
                                                         long long b1, long long& ws, long long& we) {
    constexpr long long VEC = 16 / sizeof(T);
    const long long halo = NXY + NX + 1;
    ws = b0 - halo;
    if (ws < 0) ws = 0;
    ws -= ws % VEC;
    we = b1 + halo;
    if (we > N) we = N;
    we = (we + VEC - 1) / VEC * VEC;
}

// the zero-padded window of the staged-rows variant: [ws, we) around the
// block's range without clamping to the mesh, so that every stencil slot of
// every owned node indexes inside it; entries outside [0, N) read as zero
template <typename T>
static __host__ __device__ __forceinline__ void z_window_padded(long long NX, long long NXY, long long b0,
                                                                long long b1, long long& ws, long long& we) {
    constexpr long long VEC = 16 / sizeof(T);
    const long long halo = NXY + NX + 1;
    ws = b0 - halo;
    ws = (ws >= 0) ? ws - ws % VEC : -(((-ws) + VEC - 1) / VEC) * VEC;
    we = (b1 + halo + VEC - 1) / VEC * VEC;
}

// Jacobi PCG, vectors in registers.  FP64 mode: one pass in FP64.  MIXED: FP64
// refinement (true residual of u in FP64) around FP32 inner solves for x.
// ROWS: the block's operator rows are built once into shared memory ([node][19]
// coefficients) and every matrix product is a branch-free 19-term sum over a
// zero-padded window; otherwise rows are evaluated from the mesh each time.
template <bool MIXED, int NPT, bool ROWS>
__global__ void __launch_bounds__(REG_THREADS, 1) k_pcg_reg(RegArgs a) {
    using T = typename std::conditional<MIXED, float, double>::type;
    using V = typename std::conditional<MIXED, float4, double2>::type;
    constexpr int VEC = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char win_raw[];
    __shared__ ExchShared xs;
    const FieldArgs& f = a.f;
    const long long N = f.m.nnodes;
    const long long NXY = (long long)f.m.NX * f.m.NY;
    const long long b0 = (long long)blockIdx.x * a.M;
    const long long b1 = b0 + a.M < N ? b0 + a.M : N;
    const int nown = (int)(b1 - b0);
    // staged rows come first (19 T per owned node, rounded to 16 bytes), then the window
    const size_t rows_bytes = ROWS ? ((size_t)a.M * 19 * sizeof(T) + 15) / 16 * 16 : 0;
    T* rows = (T*)win_raw;
    T* win = (T*)(win_raw + rows_bytes);
    long long ws, we;
    if (ROWS) z_window_padded<T>(f.m.NX, NXY, b0, b1, ws, we);
    else z_window<T>(N, f.m.NX, NXY, b0, b1, ws, we);
    const int nvec = (int)((we - ws) / VEC);
    const long long nvec_in = (N + VEC - 1) / VEC;   // vectors of z inside the padded allocation
    T* const zbuf[2] = {(T*)a.zg[0], (T*)a.zg[1]};
    int zc = 0;   // the copy the next staging reads
    const T* coef = MIXED ? (const T*)f.coeff : (const T*)f.coef;
    const T* dinv = MIXED ? (const T*)f.invdiagf : (const T*)f.invdiag;
    const double tol2 = a.S->tol2, inner_red2 = a.S->inner_red2, margin2 = a.S->margin2;
    const int maxit = a.S->maxit;
    auto ldw = [&](long long m) { return win[m - ws]; };
    auto ldu = [&](long long m) { return __ldcg(a.u + m); };
    int e = 0;
    if (ROWS) {
        for (int li = threadIdx.x; li < nown; li += REG_THREADS) {
            const long long n = b0 + li;
            int i, j, kk;
            node_ijk(f.m, n, i, j, kk);
            T c[19];
            row_coeffs<T>(f, n, i, j, kk, coef, c);
#pragma unroll
            for (int q = 0; q < 19; ++q) rows[li * 19 + q] = c[q];
        }
        // rows are read only after the first exchange's __syncthreads
    }
    unsigned pk[NPT];
    T dv[NPT];
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
        const long long n = b0 + threadIdx.x + s * REG_THREADS;
        pk[s] = 0;
        dv[s] = (T)0;
        if (n < b1) {
            int i, j, kk;
            node_ijk(f.m, n, i, j, kk);
            pk[s] = pack_ijk(i, j, kk);
            dv[s] = dinv[n];
        }
    }
    // this launch's starting values of the fixed-point words (read before the
    // first exchange, so before any block of this launch adds to them)
    unsigned long long fxa = 0, fxb = 0;
    if (MIXED && threadIdx.x < 2) {
        fxa = ld_relaxed(a.fx);
        fxb = ld_relaxed(a.fx + (1 + threadIdx.x) * FX_LINE);
    }
    // pipelined loop: two word sets used in turn (a set is reused only after an
    // exchange on the other one, so every block has read its last total);
    // fxp0 belongs to the set of the next exchange, fxp1 to the other one
    unsigned long long fxp0 = 0, fxp1 = 0;
    int pset = 0;
    if (MIXED && threadIdx.x < 3) {
        fxp0 = ld_relaxed(a.fx + (3 + threadIdx.x) * FX_LINE);
        fxp1 = ld_relaxed(a.fx + (6 + threadIdx.x) * FX_LINE);
    }
    // MIXED inner loop: pipelined unless an earlier solve of this context found
    // its recurrences too far from the true residual (then the classic loop)
    bool pipe = MIXED && *a.classic == 0;
    bool switched = false;
    // copy the window of zg that this block's rows read into shared memory (the
    // last exchange ordered every block's stores to zg and every read of the
    // previous window)
    auto stage = [&](const T* zg) {
        V* dst = (V*)win;
        if (ROWS) {
            const long long v0 = ws / VEC;   // exact: ws is a multiple of VEC
            for (int c = threadIdx.x; c < nvec; c += REG_THREADS) {
                const long long gv = v0 + c;
                V val = {};
                if (gv >= 0 && gv < nvec_in) val = __ldcg((const V*)zg + gv);
                dst[c] = val;
            }
        } else {
            const V* src = (const V*)(zg + ws);
            for (int c = threadIdx.x; c < nvec; c += REG_THREADS) dst[c] = __ldcg(src + c);
        }
        __syncthreads();
    };
    // row n (slot s of this thread) of the operator times the staged window
    auto apply = [&](int s, long long n) -> T {
        if (ROWS) {
            const int li = threadIdx.x + s * REG_THREADS;
            const T* rw = rows + li * 19;
            const T* wc = win + (n - ws);
            T az = rw[0] * wc[0];
#pragma unroll
            for (int q = 1; q < 19; ++q) az += rw[q] * wc[a.woff[q]];
            return az;
        }
        return row_at<T>(f, n, pk[s], ldw, coef);
    };
    int it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    T rr_exit = (T)0;     // recurrence residual at the end of the last inner solve
    bool conv = false, alive = true;
    for (;;) {
        // true residual of u in FP64 (neighbours of u through L2); z = D^-1 r, p = z
        T x[NPT], r[NPT], z[NPT], p[NPT], q[NPT];
        double v3[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int s = 0; s < NPT; ++s) {
            const long long n = b0 + threadIdx.x + s * REG_THREADS;
            x[s] = r[s] = z[s] = p[s] = q[s] = (T)0;
            if (n < b1) {
                const double bn = a.b[n];
                const double rn = (f.ntype[n] == -3) ? 0.0
                                                     : bn - apply_row64(f, n, (int)(pk[s] & 2047u),
                                                                        (int)((pk[s] >> 11) & 2047u), (int)(pk[s] >> 22),
                                                                        ldu, f.coef);
                r[s] = (T)rn;
                z[s] = dv[s] * r[s];
                p[s] = z[s];
                zbuf[zc][n] = z[s];
                v3[0] += bn * bn;
                v3[1] += rn * rn;
                v3[2] += (double)r[s] * (double)z[s];
            }
        }
        double t3[3];
        if (!(alive = exchange<double, 3>(a, e, v3, t3, xs))) break;
        if (outer == 0) bb = t3[0];
        rr = t3[1];
        T rz = (T)t3[2];
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        // the pipelined recurrences drift from the true residual by the rounding
        // they amplify; if the last inner solve ended far above what it claimed,
        // finish with the classic loop (and keep it for this context's next solves)
        if (MIXED && pipe && outer > 0 && !conv && rr > PIPE_GAP2 * (double)rr_exit) {
            pipe = false;
            switched = true;
        }
        if (conv || it >= maxit || (MIXED && outer >= COOP_MAX_OUTER)) break;
        // inner target: the final tolerance, or (MIXED) max(margin tol |b|, reduction |r0|) (set_refinement)
        const T rr_stop = (T)(MIXED ? fmax(margin2 * tol2 * bb, inner_red2 * rr) : tol2 * bb);
        ++outer;
        T rr_in = (T)rr;
        if (MIXED && pipe) {
          if constexpr (MIXED) {
            // Pipelined Jacobi PCG (Ghysels and Vanroose): the recurrences for
            // u = D^-1 r, w = A u, m = D^-1 w, and A p, D^-1 A p, A D^-1 A p
            // move the matrix product behind the iteration's one exchange, which
            // carries r.u, w.u and r.r and also publishes m for the product.
            // u starts as z (written above, ordered by the residual exchange).
            T w[NPT], sv[NPT], nz[NPT];
            stage(zbuf[zc]);
#pragma unroll
            for (int s = 0; s < NPT; ++s) {
                const long long n = b0 + threadIdx.x + s * REG_THREADS;
                w[s] = sv[s] = nz[s] = (T)0;
                if (n < b1) w[s] = apply(s, n);
            }
            float ref[3] = {0.0f, 0.0f, 0.0f};
            bool have_ref = false;
            T gam_old = (T)1, al_old = (T)1;
            bool first = true;
            // progress: the recurrence residual must halve within PIPE_STALL
            // iterations, else (FP32 pipelined recurrences can stall and drift
            // on hard meshes) the inner solve ends and the classic loop takes over
            T rr_mark = rr_in;
            int it_mark = it;
            for (;;) {
                T v[3] = {(T)0, (T)0, (T)0};
#pragma unroll
                for (int s = 0; s < NPT; ++s) {
                    const long long n = b0 + threadIdx.x + s * REG_THREADS;
                    if (n < b1) {
                        zbuf[zc ^ 1][n] = dv[s] * w[s];
                        v[0] += r[s] * z[s];
                        v[1] += w[s] * z[s];
                        v[2] += r[s] * r[s];
                    }
                }
                T t[3];
                alive = exchange_f32<3, true, 8>(a, e, a.fx + (3 + 3 * pset) * FX_LINE, fxp0, ref, have_ref, v, t,
                                                 xs);
                if (!alive) break;
                {
                    const unsigned long long tmp = fxp0;
                    fxp0 = fxp1;
                    fxp1 = tmp;
                    pset ^= 1;
                }
                zc ^= 1;
                rr_in = t[2];
                if (rr_in <= rr_stop || it >= maxit) break;
                if (rr_in <= (T)0.25 * rr_mark) {
                    rr_mark = rr_in;
                    it_mark = it;
                } else if (it - it_mark > PIPE_STALL) {
                    pipe = false;
                    switched = true;
                    break;
                }
                const T gam = t[0], dl = t[1];
                T be, al;
                if (first) {
                    be = (T)0;
                    al = gam / dl;
                } else {
                    be = gam / gam_old;
                    al = gam / (dl - be * gam / al_old);
                }
                stage(zbuf[zc]);
#pragma unroll
                for (int s = 0; s < NPT; ++s) {
                    const long long n = b0 + threadIdx.x + s * REG_THREADS;
                    if (n < b1) {
                        const T nn = apply(s, n);
                        const T m = dv[s] * w[s];
                        if (first) {
                            nz[s] = nn; q[s] = m; sv[s] = w[s]; p[s] = z[s];
                        } else {
                            nz[s] = nn + be * nz[s];
                            q[s] = m + be * q[s];
                            sv[s] = w[s] + be * sv[s];
                            p[s] = z[s] + be * p[s];
                        }
                        x[s] = x[s] + al * p[s];
                        r[s] = r[s] - al * sv[s];
                        z[s] = z[s] - al * q[s];
                        w[s] = w[s] - al * nz[s];
                    }
                }
                first = false;
                gam_old = gam;
                al_old = al;
                ref[0] = t[0]; ref[1] = t[1]; ref[2] = t[2];
                have_ref = fx_ref_ok(t[0]) && fx_ref_ok(t[1]) && fx_ref_ok(t[2]);
                ++it;
            }
          }
        } else {
            T beta = (T)0;
            float pq_prev = 0.0f;     // no scale for the first p.q of an inner solve
            bool first = true;
            for (;;) {
                stage(zbuf[zc]);
                // p = z + beta p, q = A z + beta q (= A p); first pass: q = A z
                T v1[1] = {(T)0};
                const T bt = beta;
#pragma unroll
                for (int s = 0; s < NPT; ++s) {
                    const long long n = b0 + threadIdx.x + s * REG_THREADS;
                    if (n < b1) {
                        const T az = apply(s, n);
                        if (first) {
                            q[s] = az;
                        } else {
                            p[s] = z[s] + bt * p[s];
                            q[s] = az + bt * q[s];
                        }
                        v1[0] += p[s] * q[s];
                    }
                }
                first = false;
                T pq[1];
                if constexpr (MIXED) {
                    const float rf[1] = {pq_prev};
                    alive = exchange_f32<1, false, 8>(a, e, a.fx, fxa, rf, fx_ref_ok(pq_prev), v1, pq, xs);
                    pq_prev = pq[0];
                } else {
                    alive = exchange<T, 1>(a, e, v1, pq, xs);
                }
                if (!alive) break;
                const T al = rz / pq[0];
                T v2[2] = {(T)0, (T)0};
#pragma unroll
                for (int s = 0; s < NPT; ++s) {
                    const long long n = b0 + threadIdx.x + s * REG_THREADS;
                    if (n < b1) {
                        x[s] = x[s] + al * p[s];
                        r[s] = r[s] - al * q[s];
                        z[s] = dv[s] * r[s];
                        zbuf[zc ^ 1][n] = z[s];
                        v2[0] += r[s] * r[s];
                        v2[1] += r[s] * z[s];
                    }
                }
                T t2[2];
                if constexpr (MIXED) {
                    const float rf[2] = {rr_in, rz};
                    alive = exchange_f32<2, true, 8>(a, e, a.fx + FX_LINE, fxb, rf, fx_ref_ok(rr_in) && fx_ref_ok(rz),
                                                     v2, t2, xs);
                } else {
                    alive = exchange<T, 2>(a, e, v2, t2, xs);
                }
                if (!alive) break;
                zc ^= 1;
                beta = t2[1] / rz;
                rz = t2[1];
                rr_in = t2[0];
                ++it;
                if (rr_in <= rr_stop || it >= maxit) break;
            }
        }
        if (!alive) break;
        rr_exit = rr_in;
        // u += x; MIXED: an exchange so that the next residual sees the new u
#pragma unroll
        for (int s = 0; s < NPT; ++s) {
            const long long n = b0 + threadIdx.x + s * REG_THREADS;
            if (n < b1) a.u[n] = a.u[n] + (double)x[s];
        }
        if (!MIXED) {
            rr = (double)rr_in;
            conv = rr <= tol2 * bb;
            break;
        }
        T v0[1] = {(T)0}, t0s[1];
        if (!(alive = exchange<T, 1>(a, e, v0, t0s, xs))) break;
    }
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
        const long long n = b0 + threadIdx.x + s * REG_THREADS;
        if (n < b1) a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        PcgState* S = a.S;
        S->bb = bb;
        S->rr = rr;
        S->it = it;
        S->outer_it = outer;
        S->converged = alive && conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += MIXED ? outer : 0;
        if (MIXED && switched) *a.classic = 1;
    }
}

// ---- global-memory PCG for meshes beyond the register-resident kernel -----------
//
// Vectors in global memory (a 2M-node mesh keeps them in L2), otherwise the
// same iteration as k_pcg_reg: Jacobi PCG with the q recurrence, two
// exchanges per iteration (MIXED: the fixed-point exchange for up to 511
// blocks, the p.q one relaxed, z in two copies by iteration parity; FP64: the
// partial exchange), FP32 inner arithmetic in MIXED mode, FP64 refinement
// residual.  Regular rows are the branch-free
// masked stencil selected by a per-node kind word (made once per mesh);
// interface rows use their patch coefficients.  Each thread takes its nodes
// four at a time and issues every load of the four before any store, so the
// L2 round trips of a group overlap; two 512-thread blocks per SM (64
// registers, a few spilled) hide more latency than one block without spills.

constexpr int GLOB_THREADS = 512;
constexpr int GLOB_UNROLL = 4;

struct GlobArgs {
    FieldArgs f;
    const unsigned short* kind;   // [N] row kinds
    const double* b;
    double* u;
    const double* g;
    double* phi;
    void *r, *z, *z2, *p, *q, *x;   // working-precision vectors (z in two guarded copies)
    double* val;
    unsigned long long* arrivals;
    unsigned long long* fx;         // fixed-point exchange words (as RegArgs::fx)
    const int* hold;                // as RegArgs::hold
    PcgState* S;
    long long* it_total;
    long long* outer_total;
    int* err;
};

__global__ void k_row_kind(FieldArgs f, unsigned short* kind) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= f.m.nnodes) return;
    int i, j, k;
    node_ijk(f.m, n, i, j, k);
    kind[n] = row_kind(f, n, i, j, k);
}

// x must be readable (and finite) up to NXY + NX + 1 entries outside [0, N):
// the masked stencil of a boundary node reads its absent neighbours and
// multiplies them by zero (the context's z / zf carry a zeroed guard)
template <typename T>
static __device__ __forceinline__ T glob_row(const GlobArgs& a, const T* x, long long n, unsigned kd, int NX,
                                             int NXY, T h, T ep, T em, const T* coef) {
    if (kd & RK_DIRICHLET) return (T)0;
    if (kd & RK_GENERAL) {
        int i, j, k;
        node_ijk(a.f.m, n, i, j, k);
        return apply_row<T, true>(a.f, n, i, j, k, x, coef);
    }
    return regular_row_masked_ld<T>([&](int o) { return __ldcg(x + n + o); }, NX, NXY, kd, h, h_over6<T>(a.f.m),
                                    h_over12<T>(a.f.m), ep, em);
}

template <bool MIXED>
__global__ void __launch_bounds__(GLOB_THREADS, 2) k_pcg_glob(GlobArgs a) {
    using T = typename std::conditional<MIXED, float, double>::type;
    __shared__ ExchShared xs;
    const FieldArgs& f = a.f;
    const long long N = f.m.nnodes;
    const long long TT = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T* r = (T*)a.r;
    T* const zb[2] = {(T*)a.z, (T*)a.z2};
    int zc = 0;   // the copy the next products read
    T* p = (T*)a.p;
    T* q = (T*)a.q;
    T* x = (T*)a.x;
    const T* coef = MIXED ? (const T*)f.coeff : (const T*)f.coef;
    const T* dinv = MIXED ? (const T*)f.invdiagf : (const T*)f.invdiag;
    const int NX = f.m.NX, NXY = f.m.NX * f.m.NY;
    const T hT = (T)f.m.h, ep = (T)f.o.eps_plus, em = (T)f.o.eps_minus;
    const double tol2 = a.S->tol2, inner_red2 = a.S->inner_red2, margin2 = a.S->margin2;
    const int maxit = a.S->maxit;
    int e = 0, it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    bool conv = false, alive = true;
    // this launch's starting values of the fixed-point words (before any block adds)
    unsigned long long fxa = 0, fxb = 0;
    if (MIXED && threadIdx.x < 2) {
        fxa = ld_relaxed(a.fx);
        fxb = ld_relaxed(a.fx + (1 + threadIdx.x) * FX_LINE);
    }
    for (;;) {
        // true residual of u in FP64; z = D^-1 r, p = z, x = 0
        double v3[3] = {0.0, 0.0, 0.0};
        for (long long n = t0; n < N; n += TT) {
            int i, j, k;
            node_ijk(f.m, n, i, j, k);
            const double bn = a.b[n];
            const double rn =
                (f.ntype[n] == -3) ? 0.0
                                   : bn - apply_row64(f, n, i, j, k, [&](long long m) { return __ldcg(a.u + m); }, f.coef);
            const T rt = (T)rn, zt = dinv[n] * rt;
            r[n] = rt; zb[zc][n] = zt; p[n] = zt; x[n] = (T)0;
            v3[0] += bn * bn;
            v3[1] += rn * rn;
            v3[2] += (double)rt * (double)zt;
        }
        double t3[3];
        if (!(alive = exchange<double, 3>(a, e, v3, t3, xs))) break;
        if (outer == 0) bb = t3[0];
        rr = t3[1];
        T rz = (T)t3[2];
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        if (conv || it >= maxit || (MIXED && outer >= COOP_MAX_OUTER)) break;
        const T rr_stop = (T)(MIXED ? fmax(margin2 * tol2 * bb, inner_red2 * rr) : tol2 * bb);
        ++outer;
        T beta = (T)0, rr_in = (T)rr;
        float pq_prev = 0.0f;     // no scale for the first p.q of an inner solve
        bool first = true;
        for (;;) {
            // p = z + beta p, q = A z + beta q (first pass: p = z, q = A z)
            const T* z = zb[zc];
            T v1[1] = {(T)0};
            for (long long n0 = t0; n0 < N; n0 += GLOB_UNROLL * TT) {
                T az[GLOB_UNROLL], zl[GLOB_UNROLL], pl[GLOB_UNROLL], ql[GLOB_UNROLL];
#pragma unroll
                for (int u = 0; u < GLOB_UNROLL; ++u) {
                    const long long n = n0 + u * TT;
                    az[u] = zl[u] = pl[u] = ql[u] = (T)0;
                    if (n < N) {
                        az[u] = glob_row<T>(a, z, n, a.kind[n], NX, NXY, hT, ep, em, coef);
                        zl[u] = __ldcg(z + n);
                        if (!first) { pl[u] = __ldcg(p + n); ql[u] = __ldcg(q + n); }
                    }
                }
#pragma unroll
                for (int u = 0; u < GLOB_UNROLL; ++u) {
                    const long long n = n0 + u * TT;
                    if (n < N) {
                        const T pn = first ? zl[u] : zl[u] + beta * pl[u];
                        const T qn = first ? az[u] : az[u] + beta * ql[u];
                        p[n] = pn; q[n] = qn;
                        v1[0] += pn * qn;
                    }
                }
            }
            first = false;
            T pq[1];
            if constexpr (MIXED) {
                const float rf[1] = {pq_prev};
                alive = exchange_f32<1, false, 9>(a, e, a.fx, fxa, rf, fx_ref_ok(pq_prev), v1, pq, xs);
                pq_prev = pq[0];
            } else {
                alive = exchange<T, 1>(a, e, v1, pq, xs);
            }
            if (!alive) break;
            const T al = rz / pq[0];
            T* zn_out = zb[zc ^ 1];
            T v2[2] = {(T)0, (T)0};
            for (long long n0 = t0; n0 < N; n0 += GLOB_UNROLL * TT) {
                T xl[GLOB_UNROLL], rl[GLOB_UNROLL], pl[GLOB_UNROLL], ql[GLOB_UNROLL], dl[GLOB_UNROLL];
#pragma unroll
                for (int u = 0; u < GLOB_UNROLL; ++u) {
                    const long long n = n0 + u * TT;
                    xl[u] = rl[u] = pl[u] = ql[u] = dl[u] = (T)0;
                    if (n < N) {
                        xl[u] = __ldcg(x + n); rl[u] = __ldcg(r + n); pl[u] = __ldcg(p + n); ql[u] = __ldcg(q + n);
                        dl[u] = dinv[n];
                    }
                }
#pragma unroll
                for (int u = 0; u < GLOB_UNROLL; ++u) {
                    const long long n = n0 + u * TT;
                    if (n < N) {
                        const T rn = rl[u] - al * ql[u];
                        const T zn = dl[u] * rn;
                        x[n] = xl[u] + al * pl[u];
                        r[n] = rn;
                        zn_out[n] = zn;
                        v2[0] += rn * rn;
                        v2[1] += rn * zn;
                    }
                }
            }
            T t2[2];
            if constexpr (MIXED) {
                const float rf[2] = {rr_in, rz};
                alive = exchange_f32<2, true, 9>(a, e, a.fx + FX_LINE, fxb, rf, fx_ref_ok(rr_in) && fx_ref_ok(rz), v2,
                                                 t2, xs);
            } else {
                alive = exchange<T, 2>(a, e, v2, t2, xs);
            }
            if (!alive) break;
            zc ^= 1;
            beta = t2[1] / rz;
            rz = t2[1];
            rr_in = t2[0];
            ++it;
            if (rr_in <= rr_stop || it >= maxit) break;
        }
        if (!alive) break;
        for (long long n = t0; n < N; n += TT) a.u[n] = a.u[n] + (double)__ldcg(x + n);
        if (!MIXED) {
            rr = (double)rr_in;
            conv = rr <= tol2 * bb;
            break;
        }
        T v0[1] = {(T)0}, t0s[1];
        if (!(alive = exchange<T, 1>(a, e, v0, t0s, xs))) break;
    }
    for (long long n = t0; n < N; n += TT) a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        PcgState* S = a.S;
        S->bb = bb; S->rr = rr; S->it = it; S->outer_it = outer;
        S->converged = alive && conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += MIXED ? outer : 0;
    }
}


// staged rows only in MIXED mode (19 FP64 coefficients per node do not fit
// next to an FP64 window)
static void* reg_kernel(bool mixed, int npt, bool rows) {
    if (mixed && rows) {
        switch (npt) {
            case 1: return (void*)k_pcg_reg<true, 1, true>;
            case 2: return (void*)k_pcg_reg<true, 2, true>;
            case 4: return (void*)k_pcg_reg<true, 4, true>;
            case 8: return (void*)k_pcg_reg<true, 8, true>;
            default: return nullptr;
        }
    }
    switch (npt) {
        case 1: return mixed ? (void*)k_pcg_reg<true, 1, false> : (void*)k_pcg_reg<false, 1, false>;
        case 2: return mixed ? (void*)k_pcg_reg<true, 2, false> : (void*)k_pcg_reg<false, 2, false>;
        case 4: return mixed ? (void*)k_pcg_reg<true, 4, false> : (void*)k_pcg_reg<false, 4, false>;
        case 8: return mixed ? (void*)k_pcg_reg<true, 8, false> : (void*)k_pcg_reg<false, 8, false>;
        default: return nullptr;
    }
}

// nodes per thread, grid and shared memory of the register-resident kernel for
// this mesh (stored in the context; called before any capture of the solve);
// npt = 0 if it needs more than 8 nodes per thread or a z window larger than
// shared memory
static void plan_pcg_reg(Ctx& c);

// the register-resident plan, else the global-memory kernel's row kinds and
// FP64 correction vector (made here, before any capture of the solve)
cudaError_t plan_pcg_mg(Ctx& c);   // pcg_mg.cu: the multigrid hierarchy (MIXED), if selected

void plan_pcg(Ctx& c) {
    // the exchanges count arrivals in multiples of their grid size, which differs
    // between the solvers: a new plan starts the counters (and the pipelined
    // loop's fallback flag) afresh
    szero(c.stream, c.bar64, sizeof(unsigned long long) * BAR64_WORDS);
    szero(c.stream, (int*)(c.scal + 44), sizeof(int));
    plan_pcg_reg(c);
    lib_free(c.rowkind); lib_free(c.pcg_x);
    c.rowkind = nullptr; c.pcg_x = nullptr;
    if (plan_pcg_mg(c) != cudaSuccess) cudaGetLastError();   // (no hierarchy: the Jacobi solvers)
    if (c.pcg_npt > 0 && c.mg_nlev == 0) return;
    const long long N = c.mesh.nnodes;
    if (lib_malloc(&c.rowkind, sizeof(unsigned short) * N) != cudaSuccess ||
        lib_malloc(&c.pcg_x, sizeof(double) * N) != cudaSuccess) {
        cudaGetLastError();
        return;   // the solve then reports cudaErrorNotReady
    }
    FieldArgs f;
    f.m = c.mesh; f.o = c.obj; f.ntype = c.ntype; f.coef = c.patch_coef; f.coeff = c.patch_coeff;
    f.invdiag = c.invdiag; f.invdiagf = c.invdiagf;
    k_row_kind<<<(unsigned)((N + 255) / 256), 256, 0, c.stream>>>(f, c.rowkind);
    cudaStreamSynchronize(c.stream);
}

static void plan_pcg_reg(Ctx& c) {
    const bool mixed = c.precision == PIFEPIC_MIXED;
    c.pcg_npt = 0;
    int dev = c.device, nsm = 0, smem_max = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long N = c.mesh.nnodes;
    const size_t tsz = mixed ? sizeof(float) : sizeof(double);
    // one 512-thread block per SM (registers allow no more), on every SM even
    // for a small mesh: the FP64 passes (FP64 mode, and MIXED's refinement
    // residuals) run at 1/58 of the FP32 rate here, and spread over the device
    long long G = nsm;
    if (G > N) G = N;
    if (G > REG_THREADS) G = REG_THREADS;   // exchange totals: one partial per thread
    if (G > 255) G = 255;          // the fixed-point exchange counts arrivals in 8 bits
    if (G < 1) G = 1;
    const long long M = (N + G - 1) / G;
    G = (N + M - 1) / M;           // every block owns at least one node
    const long long npt = (M + REG_THREADS - 1) / REG_THREADS;
    int pick = npt <= 1 ? 1 : npt <= 2 ? 2 : npt <= 4 ? 4 : npt <= 8 ? 8 : 0;
    if (!pick) return;
    // largest window over the blocks, plus one vector of slack
    const long long NX = c.mesh.NX, NXY = (long long)c.mesh.NX * c.mesh.NY;
    long long wmax = 0;
    for (long long bl = 0; bl < G; ++bl) {
        long long ws, we, b0 = bl * M, b1 = b0 + M < N ? b0 + M : N;
        if (mixed) z_window<float>(N, NX, NXY, b0, b1, ws, we);
        else z_window<double>(N, NX, NXY, b0, b1, ws, we);
        if (we - ws > wmax) wmax = we - ws;
    }
    const size_t static_smem = sizeof(ExchShared) + 64;
    auto try_plan = [&](bool rows, size_t smem) {
        if (smem + static_smem > (size_t)smem_max) return false;
        void* kern = reg_kernel(mixed, pick, rows);
        // the function's limit is the whole opt-in budget, the same for every
        // context (a per-context value would leave it at the last context's
        // size, below what earlier contexts' graph nodes launch with)
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const int limit = smem_max - (int)fa.sharedSizeBytes;
        if ((long long)smem > (long long)limit ||
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, REG_THREADS, smem);
        if (per < 1) return false;
        c.pcg_npt = pick;
        c.pcg_rows = rows;
        c.pcg_G = (int)G;
        c.pcg_M = M;
        c.pcg_smem = smem;
        return true;
    };
    if (mixed) {
        long long wpad = 0;   // longest zero-padded window over the blocks
        for (long long bl = 0; bl < G; ++bl) {
            long long ws, we, b0 = bl * M, b1 = b0 + M < N ? b0 + M : N;
            z_window_padded<float>(NX, NXY, b0, b1, ws, we);
            if (we - ws > wpad) wpad = we - ws;
        }
        const size_t rows_bytes = ((size_t)M * 19 * sizeof(float) + 15) / 16 * 16;
        if (try_plan(true, rows_bytes + (size_t)wpad * sizeof(float))) return;
    }
    try_plan(false, (size_t)wmax * tsz);
}

static cudaError_t launch_reg(Ctx& c, cudaStream_t st, bool mixed) {
    RegArgs a;
    a.f.m = c.mesh; a.f.o = c.obj; a.f.ntype = c.ntype; a.f.coef = c.patch_coef; a.f.coeff = c.patch_coeff;
    a.f.invdiag = c.invdiag; a.f.invdiagf = c.invdiagf;
    a.b = c.b; a.u = c.u; a.g = c.gdir; a.phi = c.phi;
    a.zg[0] = mixed ? (void*)c.zf : (void*)c.z;
    a.zg[1] = mixed ? (void*)c.zf2 : (void*)c.z2;
    a.M = c.pcg_M;
    {
        const int NX = c.mesh.NX, NXY = c.mesh.NX * c.mesh.NY;
        const int d[19][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
                              {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {1, 0, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};
        for (int q = 0; q < 19; ++q) a.woff[q] = d[q][0] + d[q][1] * NX + d[q][2] * NXY;
    }
    a.val = c.coop_partial;
    a.arrivals = c.bar64;
    a.fx = c.bar64 + FX_LINE;
    a.classic = (int*)(c.scal + 44);
    a.S = (PcgState*)c.scal;
    a.it_total = (long long*)(c.scal + 40);
    a.outer_total = (long long*)(c.scal + 41);
    a.err = c.err_word;
    a.hold = (const int*)(c.scal + 45);
    void* args[] = {&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.pcg_G);
    cfg.blockDim = dim3(REG_THREADS);
    cfg.dynamicSmemBytes = c.pcg_smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, reg_kernel(mixed, c.pcg_npt, c.pcg_rows), args);
}

// the PCG state must already hold tol2 and maxit; writes phi
cudaError_t launch_pcg_mg(Ctx& c, cudaStream_t st);   // pcg_mg.cu

cudaError_t launch_pcg_coop(Ctx& c, cudaStream_t st) {
    bool mixed = c.precision == PIFEPIC_MIXED;
    if (c.pcg_npt < 0) plan_pcg(c);
    if (mixed && c.mg_single && c.mg_nlev > 0) {
        if (!c.rowkind) return cudaErrorNotReady;
        return launch_pcg_mg(c, st);
    }
    if (c.pcg_npt > 0) return launch_reg(c, st, mixed);
    if (!c.rowkind || !c.pcg_x) return cudaErrorNotReady;   // plan_pcg prepares the global-memory kernel
    GlobArgs a;
    a.f.m = c.mesh; a.f.o = c.obj; a.f.ntype = c.ntype; a.f.coef = c.patch_coef; a.f.coeff = c.patch_coeff;
    a.f.invdiag = c.invdiag; a.f.invdiagf = c.invdiagf;
    a.kind = c.rowkind;
    a.b = c.b; a.u = c.u; a.g = c.gdir; a.phi = c.phi;
    if (mixed) { a.r = c.rf; a.z = c.zf; a.z2 = c.zf2; a.p = c.pf; a.q = c.qf; a.x = c.uf; }
    else { a.r = c.r; a.z = c.z; a.z2 = c.z2; a.p = c.p; a.q = c.q; a.x = c.pcg_x; }
    a.fx = c.bar64 + FX_LINE;
    a.val = c.coop_partial;
    a.arrivals = c.bar64;
    a.S = (PcgState*)c.scal;
    a.it_total = (long long*)(c.scal + 40);
    a.outer_total = (long long*)(c.scal + 41);
    a.err = c.err_word;
    a.hold = (const int*)(c.scal + 45);
    int dev = c.device, nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_glob<true>, GLOB_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_glob<false>, GLOB_THREADS, 0);
    long long G = (long long)nsm * (per > 0 ? per : 1);
    if (G > GLOB_THREADS) G = GLOB_THREADS;   // an exchange reads one block partial per thread
    if (G > 511) G = 511;                     // the fixed-point exchange counts arrivals in 9 bits
    void* args[] = {&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(GLOB_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, mixed ? (void*)k_pcg_glob<true> : (void*)k_pcg_glob<false>, args);
}

}  // namespace pf
