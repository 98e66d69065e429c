// Multigrid-preconditioned PCG for the MIXED field solve (Sec. 2.5: the matrix
// solve is a PCG iteration stopped on the relative residual; the paper names
// no preconditioner -- Jacobi is the oracle's and the FP64 path's reading, a
// geometric multigrid V-cycle is the one this solver adds).
//
// Hierarchy.  Level 0 is the IFE system on the Cartesian mesh (matrix-free
// 7/19-point rows, explicit rows next to interface tets).  A coarse level has
// the nodes at the even fine indices of every axis, plus the last node when
// the fine axis has an odd number of cells, so any mesh coarsens.  The
// prolongation P is trilinear interpolation along the axes, zero on Dirichlet
// nodes; restriction is P^T; a coarse operator is the Galerkin product
// P^T A P, a 27-point row per coarse node (computed once per set-up, in FP64,
// stored in FP32 as 27 coefficient planes).  Coarsening stops at 256 nodes.
//
// V(1,1) cycle: damped Jacobi (omega 0.6) before and after the coarse
// correction, the pre-smoother from a zero start (no product), and an exact
// solve on the coarsest level (at most 256 nodes) by its dense inverse, made
// once per set-up on the host in FP64.  Symmetric and positive definite, so it
// preconditions CG.  Every level but the coarsest is spread over the grid, one
// block per SM, with grid barriers between the passes; block 0 does the
// coarsest solve.
//
// The PCG around it is the two-exchange loop (p.q, then r.z and r.r) in FP32,
// inside the FP64 iterative refinement of the other MIXED solvers.  Vectors
// live in global memory (L2).  Every wait is bounded and reports a timeout.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "field_common.cuh"
#include "internal.h"
#include "pcg_sync.cuh"

namespace cg = cooperative_groups;

namespace pf {

constexpr int MG_THREADS = 512;
// batched (cluster) solves: smaller CTAs, two per SM, so that the latency-bound
// passes of two systems interleave on one SM
constexpr int MG_CL_THREADS = 256;
constexpr int MG_CL_PER_SM = 2;
constexpr int MG_MAX_OUTER = 12;          // refinement steps at most
constexpr long long MG_COARSEST = 256;    // coarsening stops at or below this many nodes
constexpr float MG_OMEGA = 0.6f;          // damped-Jacobi weight

struct MgArgs {
    FieldArgs f;
    const unsigned short* kind;   // [N0] fine row kinds
    const double* b;              // FP64 right-hand side
    double* u;                    // FP64 unknown (start in, solution out)
    const double* g;
    double* phi;
    float *r, *p, *q, *x;         // FP32 PCG vectors
    float *z, *x0;                // level-0 cycle vectors, inside zeroed guards (the masked stencil reads past N)
    float* r0;                    // level-0 residual after pre-smoothing
    int nlev;                     // coarse levels 1..nlev (nlev the coarsest)
    MgLevel lev[MG_MAX_LEVELS];   // lev[1..nlev]
    const float* cinv;            // the coarsest operator's inverse, row-major, row stride cinv_ld (0 on empty rows)
    int cinv_ld;                  // N rounded up to a multiple of 4 (rows start 16-byte aligned)
    double* val;
    unsigned long long* arrivals;
    const int* hold;
    PcgState* S;
    long long* it_total;
    long long* outer_total;
    int* err;
};

static_assert(sizeof(MgArgs) <= 4096, "the solve arguments travel as a kernel parameter");

// ---- the grid transfer along one axis (n fine cells) ---------------------------------
// coarse parents of fine index fi: count, indices and weights
static __device__ __forceinline__ int mg_parents(int fi, int n, int (&c)[2], float (&w)[2]) {
    if ((fi & 1) == 0) { c[0] = fi >> 1; w[0] = 1.0f; return 1; }
    if (fi == n) { c[0] = (n + 1) >> 1; w[0] = 1.0f; return 1; }
    c[0] = (fi - 1) >> 1; c[1] = (fi + 1) >> 1; w[0] = w[1] = 0.5f;
    return 2;
}
// the weight of coarse index ci for fine index fi (0 when it is not a parent)
static __device__ __forceinline__ float mg_weight(int fi, int n, int ci) {
    if (fi < 0 || fi > n) return 0.0f;
    if ((fi & 1) == 0) return (fi >> 1) == ci ? 1.0f : 0.0f;
    if (fi == n) return ((n + 1) >> 1) == ci ? 1.0f : 0.0f;
    return ((fi - 1) >> 1) == ci || ((fi + 1) >> 1) == ci ? 0.5f : 0.0f;
}
// the fine index a coarse index sits on
static __device__ __forceinline__ int mg_fine_of(int ci, int n) { return min(2 * ci, n); }

struct Dims {
    int nx, ny, nz, NX, NY;
};
static __device__ __forceinline__ Dims dims_of(const MgLevel& L) { return Dims{L.nx, L.ny, L.nz, L.NX, L.NY}; }
static __device__ __forceinline__ Dims dims_of(const Mesh& m) { return Dims{m.nx, m.ny, m.nz, m.NX, m.NY}; }

// restriction: the coarse value at (ci, cj, ck) from fine vector v on fine dims d
static __device__ float mg_restrict(const float* v, const Dims& d, int ci, int cj, int ck) {
    const int Fi = mg_fine_of(ci, d.nx), Fj = mg_fine_of(cj, d.ny), Fk = mg_fine_of(ck, d.nz);
    float wx[3], wy[3], wz[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        wx[t] = mg_weight(Fi + t - 1, d.nx, ci);
        wy[t] = mg_weight(Fj + t - 1, d.ny, cj);
        wz[t] = mg_weight(Fk + t - 1, d.nz, ck);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (wz[c] == 0.0f) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (wy[b] == 0.0f) continue;
            const float wyz = wy[b] * wz[c];
            const unsigned row = (unsigned)d.NX * (unsigned)((Fj + b - 1) + d.NY * (Fk + c - 1));
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (wx[a] != 0.0f) s += (wx[a] * wyz) * __ldcg(v + row + (unsigned)(Fi + a - 1));
        }
    }
    return s;
}

// prolongation: the interpolated coarse correction at fine (i, j, k) from coarse vector vc on coarse dims cd
static __device__ float mg_prolong(const float* vc, const Dims& fd, const Dims& cd, int i, int j, int k) {
    int cx[2], cy[2], cz[2];
    float wx[2], wy[2], wz[2];
    const int nx = mg_parents(i, fd.nx, cx, wx), ny = mg_parents(j, fd.ny, cy, wy), nz = mg_parents(k, fd.nz, cz, wz);
    float s = 0.0f;
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b) {
            const unsigned row = (unsigned)cd.NX * (unsigned)(cy[b] + cd.NY * cz[c]);
            const float w = wy[b] * wz[c];
            for (int a = 0; a < nx; ++a) s += (wx[a] * w) * __ldcg(vc + row + cx[a]);
        }
    return s;
}

// a coarse row times v: 27 coefficient planes, neighbours outside the level skipped
static __device__ float mg_coarse_row(const MgLevel& L, const float* v, long long n, int i, int j, int k) {
    float s = 0.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        if (k + dz < 0 || k + dz > L.nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if (j + dy < 0 || j + dy > L.ny) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx > L.nx) continue;
                const int q = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                const unsigned m = (unsigned)((int)n + dx + L.NX * (dy + L.NY * dz));
                s += __ldg(L.coef + (unsigned)q * (unsigned)L.N + (unsigned)n) * __ldcg(v + m);
            }
        }
    }
    return s;
}

// (node counts of a level stay below 2^31: 32-bit index arithmetic)
static __device__ __forceinline__ void level_ijk(const MgLevel& L, long long n, int& i, int& j, int& k) {
    const unsigned u = (unsigned)n, NX = (unsigned)L.NX, t = u / NX;
    i = (int)(u - t * NX);
    j = (int)(t % (unsigned)L.NY);
    k = (int)(t / (unsigned)L.NY);
}
static __device__ __forceinline__ void fine_ijk(const Mesh& m, long long n, int& i, int& j, int& k) {
    const unsigned u = (unsigned)n, NX = (unsigned)m.NX, t = u / NX;
    i = (int)(u - t * NX);
    j = (int)(t % (unsigned)m.NY);
    k = (int)(t / (unsigned)m.NY);
}

// a fine row times v (v inside a zeroed guard: the masked stencil reads the
// absent neighbours of boundary nodes and multiplies them by zero)
static __device__ __forceinline__ float mg_fine_row(const FieldArgs& f, const float* v, long long n, unsigned kd) {
    if (kd & RK_DIRICHLET) return 0.0f;
    if (kd & RK_GENERAL) {
        int i, j, k;
        node_ijk(f.m, n, i, j, k);
        return apply_row<float, true>(f, n, i, j, k, v, f.coeff);
    }
    const int NX = f.m.NX, NXY = f.m.NX * f.m.NY;
    return regular_row_masked_ld<float>([&](int o) { return __ldcg(v + n + o); }, NX, NXY, kd, (float)f.m.h,
                                        h_over6<float>(f.m), h_over12<float>(f.m), (float)f.o.eps_plus,
                                        (float)f.o.eps_minus);
}

// ---- Galerkin coarse operators (set-up) ------------------------------------------------
// the 19 slots of a fine row (row_coeffs order)
__constant__ int cSlot19[19][3] = {{0, 0, 0},  {-1, 0, 0}, {1, 0, 0},  {0, -1, 0}, {0, 1, 0},  {0, 0, -1}, {0, 0, 1},
                                   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, 0, -1}, {1, 0, -1},
                                   {-1, 0, 1},  {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

// add  wI * a * P(g, J)  to acc[J - I] for every coarse parent J of fine node (gi, gj, gk)
static __device__ __forceinline__ void rap_add(double (&acc)[27], double wa, int gi, int gj, int gk, const Dims& fd,
                                               int ci, int cj, int ck) {
    int px[2], py[2], pz[2];
    float wx[2], wy[2], wz[2];
    const int nx = mg_parents(gi, fd.nx, px, wx), ny = mg_parents(gj, fd.ny, py, wy), nz = mg_parents(gk, fd.nz, pz, wz);
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                const int dx = px[a] - ci, dy = py[b] - cj, dz = pz[c] - ck;
                acc[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += wa * ((double)wx[a] * (double)wy[b] * (double)wz[c]);
            }
}

static __device__ void rap_store(const MgLevel& C, long long I, const double (&acc)[27]) {
    const bool live = acc[13] > 0.0;
    for (int q = 0; q < 27; ++q) C.coef[(long long)q * C.N + I] = live ? (float)acc[q] : 0.0f;
    C.dinv[I] = live ? (float)(1.0 / acc[13]) : 0.0f;
}

// level 1 from the fine operator (FP64 rows; Dirichlet nodes carry no correction)
__global__ void k_mg_rap0(FieldArgs f, MgLevel C) {
    const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (I >= C.N) return;
    int ci, cj, ck;
    level_ijk(C, I, ci, cj, ck);
    const Dims fd = dims_of(f.m);
    const int Fi = mg_fine_of(ci, fd.nx), Fj = mg_fine_of(cj, fd.ny), Fk = mg_fine_of(ck, fd.nz);
    double acc[27];
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
    for (int dz = -1; dz <= 1; ++dz) {
        const float wz = mg_weight(Fk + dz, fd.nz, ck);
        if (wz == 0.0f) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const float wy = mg_weight(Fj + dy, fd.ny, cj);
            if (wy == 0.0f) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const float wx = mg_weight(Fi + dx, fd.nx, ci);
                if (wx == 0.0f) continue;
                const int i = Fi + dx, j = Fj + dy, k = Fk + dz;
                const long long n = node_id(f.m, i, j, k);
                if (f.ntype[n] == -3) continue;
                const double wI = (double)wx * (double)wy * (double)wz;
                double c19[19];
                row_coeffs<double>(f, n, i, j, k, f.coef, c19);
                for (int s = 0; s < 19; ++s) {
                    if (c19[s] == 0.0) continue;
                    const int gi = i + cSlot19[s][0], gj = j + cSlot19[s][1], gk = k + cSlot19[s][2];
                    if (f.ntype[node_id(f.m, gi, gj, gk)] == -3) continue;
                    rap_add(acc, wI * c19[s], gi, gj, gk, fd, ci, cj, ck);
                }
            }
        }
    }
    rap_store(C, I, acc);
}

// level l+1 from level l's 27-point rows
__global__ void k_mg_rap(MgLevel F, MgLevel C) {
    const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (I >= C.N) return;
    int ci, cj, ck;
    level_ijk(C, I, ci, cj, ck);
    const Dims fd = dims_of(F);
    const int Fi = mg_fine_of(ci, fd.nx), Fj = mg_fine_of(cj, fd.ny), Fk = mg_fine_of(ck, fd.nz);
    double acc[27];
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
    for (int dz = -1; dz <= 1; ++dz) {
        const float wz = mg_weight(Fk + dz, fd.nz, ck);
        if (wz == 0.0f) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const float wy = mg_weight(Fj + dy, fd.ny, cj);
            if (wy == 0.0f) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const float wx = mg_weight(Fi + dx, fd.nx, ci);
                if (wx == 0.0f) continue;
                const int i = Fi + dx, j = Fj + dy, k = Fk + dz;
                const long long n = (long long)i + (long long)F.NX * (j + (long long)F.NY * k);
                if (F.dinv[n] == 0.0f) continue;
                const double wI = (double)wx * (double)wy * (double)wz;
                for (int q = 0; q < 27; ++q) {
                    const float a = F.coef[(long long)q * F.N + n];
                    if (a == 0.0f) continue;
                    const int gi = i + q % 3 - 1, gj = j + (q / 3) % 3 - 1, gk = k + q / 9 - 1;
                    const long long g = (long long)gi + (long long)F.NX * (gj + (long long)F.NY * gk);
                    if (F.dinv[g] == 0.0f) continue;
                    rap_add(acc, wI * (double)a, gi, gj, gk, fd, ci, cj, ck);
                }
            }
        }
    }
    rap_store(C, I, acc);
}

// ---- the team that solves one system ---------------------------------------------------
// GridTeam: the whole cooperative grid (one system per launch; grid barriers and
// exchanges over the arrival counter, bounded waits).  ClusterTeam: one
// thread-block cluster per system (a batch of independent systems per launch;
// the hardware cluster barrier orders global memory within the cluster, and a
// reduction reads the C block partials through distributed shared memory).
struct GridTeam {
    const MgArgs& a;
    int& e;
    ExchShared& xs;
    __device__ long long t0() const { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ long long size() const { return (long long)gridDim.x * blockDim.x; }
    __device__ bool leader() const { return blockIdx.x == 0; }
    __device__ bool sync() { return grid_barrier(a, e, xs); }
    template <typename A, int NV>
    __device__ bool reduce(A (&v)[NV], A (&tot)[NV]) { return exchange<A, NV>(a, e, v, tot, xs); }
};

struct ClusterSlots {
    double sh[4 * 32];
    double bc[4];
    double slot[2][4];    // this CTA's partials, by reduction parity
};

struct ClusterTeam {
    cg::cluster_group& cl;
    int C, rank;
    int e;
    ClusterSlots& cs;
    __device__ long long t0() const { return (long long)rank * blockDim.x + threadIdx.x; }
    __device__ long long size() const { return (long long)C * blockDim.x; }
    __device__ bool leader() const { return rank == 0; }
    __device__ bool sync() {
        cl.sync();
        return true;
    }
    // every CTA of the cluster gets the same totals (the partials summed in rank order)
    template <typename A, int NV>
    __device__ bool reduce(A (&v)[NV], A (&tot)[NV]) {
        A* sh = (A*)cs.sh;
        block_sum_t<A, NV>(v, sh);
        A* slot = (A*)cs.slot[e & 1];
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < NV; ++q) slot[q] = v[q];
        cl.sync();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                A x = (A)0;
                if (lane < C) x = cl.map_shared_rank(slot, lane)[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) ((A*)cs.bc)[q] = x;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NV; ++q) tot[q] = ((A*)cs.bc)[q];
        ++e;
        return true;
    }
};

// ---- the V-cycle ---------------------------------------------------------------------
// A pass over the nodes [0, N) of a level, strided over the grid, four nodes
// at a time: every node's value (its loads) before any node's store, so the
// L2 round trips of a group overlap.
constexpr int MG_UNROLL = 4;
template <class F, class S>
static __device__ __forceinline__ void pass4(long long N, long long t0, long long TT, F value, S store) {
    for (long long n0 = t0; n0 < N; n0 += MG_UNROLL * TT) {
        float v[MG_UNROLL];
#pragma unroll
        for (int u = 0; u < MG_UNROLL; ++u) {
            const long long n = n0 + u * TT;
            v[u] = n < N ? value(n) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < MG_UNROLL; ++u) {
            const long long n = n0 + u * TT;
            if (n < N) store(n, v[u]);
        }
    }
}

// the pre-smoothing step from a zero start, x0 = omega D^-1 r: no product, so
// the passes that produce r write it node by node
static __device__ __forceinline__ float mg_presmooth(const FieldArgs& f, long long n, float rn) {
    return MG_OMEGA * f.invdiagf[n] * rn;
}

// z = M^-1 r: one V(1,1) cycle, entered with the pre-smoothed x0 = omega D^-1 r
// written (not yet ordered: the cycle starts with a team barrier); rz gets this
// thread's partials of r.z and r.r from the last pass; false after a timeout
template <class Team>
static __device__ bool vcycle(const MgArgs& a, Team& team, float* sb, float (&rz)[2]) {
    const FieldArgs& f = a.f;
    const long long N = f.m.nnodes;
    const long long TT = team.size();
    const long long t0 = team.t0();
    const Dims d0 = dims_of(f.m);
    // level 0, down: the residual after pre-smoothing
    if (!team.sync()) return false;
    pass4(N, t0, TT, [&](long long n) { return __ldcg(a.r + n) - mg_fine_row(f, a.x0, n, a.kind[n]); },
          [&](long long n, float v) { a.r0[n] = v; });
    if (!team.sync()) return false;
    // coarse levels above the coarsest, down: restriction and pre-smoothing, then the residual
    for (int l = 1; l < a.nlev; ++l) {
        const MgLevel& L = a.lev[l];
        const float* src = l == 1 ? a.r0 : a.lev[l - 1].res;
        const Dims fd = l == 1 ? d0 : dims_of(a.lev[l - 1]);
        pass4(L.N, t0, TT,
              [&](long long c) {
                  int i, j, k;
                  level_ijk(L, c, i, j, k);
                  return mg_restrict(src, fd, i, j, k);
              },
              [&](long long c, float bc) { L.b[c] = bc; L.x[c] = MG_OMEGA * L.dinv[c] * bc; });
        if (!team.sync()) return false;
        pass4(L.N, t0, TT,
              [&](long long c) {
                  int i, j, k;
                  level_ijk(L, c, i, j, k);
                  return L.b[c] - mg_coarse_row(L, L.x, c, i, j, k);
              },
              [&](long long c, float v) { L.res[c] = v; });
        if (!team.sync()) return false;
    }
    // the coarsest level in the team's first block: restriction into shared
    // memory, then y = inverse * rhs with tpr threads per row (a power of two,
    // at most 32) whose 16-byte loads of the row all issue at once
    if (team.leader()) {
        const MgLevel& L = a.lev[a.nlev];
        const float* src = a.nlev == 1 ? a.r0 : a.lev[a.nlev - 1].res;
        const Dims fd = a.nlev == 1 ? d0 : dims_of(a.lev[a.nlev - 1]);
        const int Nc = (int)L.N, ld = a.cinv_ld;
        for (int c = threadIdx.x; c < ld; c += blockDim.x) {
            float v = 0.0f;
            if (c < Nc) {
                int i, j, k;
                level_ijk(L, c, i, j, k);
                v = mg_restrict(src, fd, i, j, k);
            }
            sb[c] = v;
        }
        __syncthreads();
        int tpr = 32;
        while (tpr > 1 && tpr * Nc > (int)blockDim.x) tpr >>= 1;
        const int rows = (int)blockDim.x / tpr, lane = (int)threadIdx.x % tpr, seg = ld >> 2;
        for (int c0 = 0; c0 < Nc; c0 += rows) {
            const int c = c0 + (int)threadIdx.x / tpr;
            float y = 0.0f;
            if (c < Nc) {
                const float4* row = reinterpret_cast<const float4*>(a.cinv + (unsigned)c * (unsigned)ld);
#pragma unroll 8
                for (int s4 = lane; s4 < seg; s4 += tpr) {
                    const float4 w = __ldg(row + s4);
                    y += w.x * sb[4 * s4] + w.y * sb[4 * s4 + 1] + w.z * sb[4 * s4 + 2] + w.w * sb[4 * s4 + 3];
                }
            }
            for (int o = tpr >> 1; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o, tpr);
            if (lane == 0 && c < Nc) L.y[c] = y;
        }
    }
    if (!team.sync()) return false;
    // coarse levels above the coarsest, up: correction, post-smoothing
    for (int l = a.nlev - 1; l >= 1; --l) {
        const MgLevel& L = a.lev[l];
        const MgLevel& Cc = a.lev[l + 1];
        const Dims fd = dims_of(L), cd = dims_of(Cc);
        pass4(L.N, t0, TT,
              [&](long long c) {
                  const float xc = L.x[c];
                  if (L.dinv[c] == 0.0f) return xc;
                  int i, j, k;
                  level_ijk(L, c, i, j, k);
                  return xc + mg_prolong(Cc.y, fd, cd, i, j, k);
              },
              [&](long long c, float v) { L.x[c] = v; });
        if (!team.sync()) return false;
        pass4(L.N, t0, TT,
              [&](long long c) {
                  int i, j, k;
                  level_ijk(L, c, i, j, k);
                  return L.x[c] + MG_OMEGA * L.dinv[c] * (L.b[c] - mg_coarse_row(L, L.x, c, i, j, k));
              },
              [&](long long c, float v) { L.y[c] = v; });
        if (!team.sync()) return false;
    }
    // level 0, up: coarse correction, post-smoothing into z with the r.z and r.r partials
    {
        const MgLevel& C1 = a.lev[1];
        const Dims cd = dims_of(C1);
        pass4(N, t0, TT,
              [&](long long n) {
                  const float xn = a.x0[n];
                  if (a.kind[n] & RK_DIRICHLET) return xn;
                  int i, j, k;
                  fine_ijk(f.m, n, i, j, k);
                  return xn + mg_prolong(C1.y, d0, cd, i, j, k);
              },
              [&](long long n, float v) { a.x0[n] = v; });
    }
    if (!team.sync()) return false;
    rz[0] = 0.0f;
    rz[1] = 0.0f;
    for (long long n0 = t0; n0 < N; n0 += MG_UNROLL * TT) {
        float zv[MG_UNROLL], rv[MG_UNROLL];
#pragma unroll
        for (int u = 0; u < MG_UNROLL; ++u) {
            const long long n = n0 + u * TT;
            zv[u] = 0.0f;
            rv[u] = 0.0f;
            if (n < N) {
                const float xn = __ldcg(a.x0 + n);
                rv[u] = __ldcg(a.r + n);
                zv[u] = xn + MG_OMEGA * f.invdiagf[n] * (rv[u] - mg_fine_row(f, a.x0, n, a.kind[n]));
            }
        }
#pragma unroll
        for (int u = 0; u < MG_UNROLL; ++u) {
            const long long n = n0 + u * TT;
            if (n < N) a.z[n] = zv[u];
            rz[0] += rv[u] * zv[u];
            rz[1] += rv[u] * rv[u];
        }
    }
    return true;
}

// the refined multigrid-preconditioned PCG of one system, by one team
template <class Team>
static __device__ void mg_pcg(const MgArgs& a, Team& team, float* sb) {
    const FieldArgs& f = a.f;
    const long long N = f.m.nnodes;
    const long long TT = team.size();
    const long long t0 = team.t0();
    float* r = a.r;
    float* p = a.p;
    float* q = a.q;
    float* x = a.x;
    const float* z = a.z;
    const double tol2 = a.S->tol2, inner_red2 = a.S->inner_red2, margin2 = a.S->margin2;
    const int maxit = a.S->maxit;
    int it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    bool conv = false, alive = true;
    for (;;) {
        // true residual of u in FP64, rounded to the FP32 inner solve; x = 0
        double v3[3] = {0.0, 0.0, 0.0};
        for (long long n = t0; n < N; n += TT) {
            int i, j, k;
            node_ijk(f.m, n, i, j, k);
            const double bn = a.b[n];
            const double rn =
                (f.ntype[n] == -3) ? 0.0
                                   : bn - apply_row64(f, n, i, j, k, [&](long long m) { return __ldcg(a.u + m); }, f.coef);
            r[n] = (float)rn;
            x[n] = 0.0f;
            a.x0[n] = mg_presmooth(f, n, (float)rn);
            v3[0] += bn * bn;
            v3[1] += rn * rn;
        }
        double t3[3];
        if (!(alive = team.template reduce<double, 3>(v3, t3))) break;
        if (outer == 0) bb = t3[0];
        rr = t3[1];
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        if (conv || it >= maxit || outer >= MG_MAX_OUTER) break;
        // inner target: max(margin tol |b|, reduction |r0|) (set_refinement)
        const float rr_stop = (float)fmax(margin2 * tol2 * bb, inner_red2 * rr);
        ++outer;
        float v2[2];
        if (!(alive = vcycle(a, team, sb, v2))) break;
        float rz = 0.0f, rr_in = (float)rr;
        bool first = true;
        for (;;) {
            // r.z and r.r from the cycle's last pass (the exchange also orders z before the product below)
            float t2[2];
            if (!(alive = team.template reduce<float, 2>(v2, t2))) break;
            rr_in = t2[1];
            if (rr_in <= rr_stop || it >= maxit) break;
            const float beta = first ? 0.0f : t2[0] / rz;
            rz = t2[0];
            // p = z + beta p, q = A z + beta q (= A p)
            float v1[1] = {0.0f};
            pass4(N, t0, TT, [&](long long n) { return mg_fine_row(f, z, n, a.kind[n]); },
                  [&](long long n, float az) {
                      const float zn = __ldcg(z + n);
                      const float pn = first ? zn : zn + beta * p[n];
                      const float qn = first ? az : az + beta * q[n];
                      p[n] = pn;
                      q[n] = qn;
                      v1[0] += pn * qn;
                  });
            float pq[1];
            if (!(alive = team.template reduce<float, 1>(v1, pq))) break;
            const float al = rz / pq[0];
            for (long long n = t0; n < N; n += TT) {
                x[n] += al * p[n];
                const float rn = r[n] - al * q[n];
                r[n] = rn;
                a.x0[n] = mg_presmooth(f, n, rn);
            }
            ++it;
            first = false;
            if (!(alive = vcycle(a, team, sb, v2))) break;
        }
        if (!alive) break;
        for (long long n = t0; n < N; n += TT) a.u[n] = a.u[n] + (double)x[n];
        // the next residual reads the neighbours' new u
        if (!(alive = team.sync())) break;
    }
    for (long long n = t0; n < N; n += TT) a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    if (team.leader() && threadIdx.x == 0) {
        PcgState* S = a.S;
        S->bb = bb; S->rr = rr; S->it = it; S->outer_it = outer;
        S->converged = alive && conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += outer;
    }
}

__global__ void __launch_bounds__(MG_THREADS, 1) k_pcg_mg(MgArgs a) {
    __shared__ ExchShared xs;
    __shared__ float sb[MG_COARSEST];   // the coarsest right-hand side (block 0)
    int e = 0;
    GridTeam team{a, e, xs};
    mg_pcg(a, team, sb);
}

// batched: one system on one cluster of C CTAs (the grid is that cluster; the
// arguments travel by value, in the kernel's parameter space, as every pass
// reads them)
__global__ void __launch_bounds__(MG_CL_THREADS, MG_CL_PER_SM) k_pcg_mg_cluster(MgArgs a, int C) {
    __shared__ ClusterSlots cs;
    __shared__ float sb[MG_COARSEST];
    cg::cluster_group cl = cg::this_cluster();
    ClusterTeam team{cl, C, (int)cl.block_rank(), 0, cs};
    mg_pcg(a, team, sb);
    cl.sync();   // (no CTA leaves while a peer may still read its shared slots)
}

// ---- host side -------------------------------------------------------------------------
void free_mg(Ctx& c) {
    for (int l = 1; l <= c.mg_nlev; ++l) {
        MgLevel& L = c.mg[l];
        lib_free(L.coef); lib_free(L.dinv); lib_free(L.b); lib_free(L.x); lib_free(L.res); lib_free(L.y);
        L = MgLevel{};
    }
    lib_free(c.mg_r0);
    lib_free(c.mg_cinv);
    c.mg_r0 = nullptr;
    c.mg_cinv = nullptr;
    c.mg_nlev = 0;
}

// the inverse of the coarsest operator (dense, FP64 Gauss-Jordan with partial
// pivoting over its non-empty rows), row-major in FP32 with rows padded to a
// multiple of 4 floats; false if singular
static bool coarsest_inverse(const MgLevel& L, const std::vector<float>& coef, const std::vector<float>& dinv,
                             std::vector<float>& out) {
    const int n = (int)L.N;
    std::vector<int> live;
    std::vector<int> pos(n, -1);
    for (int I = 0; I < n; ++I)
        if (dinv[I] != 0.0f) { pos[I] = (int)live.size(); live.push_back(I); }
    const int m = (int)live.size();
    std::vector<double> A((size_t)m * m, 0.0), B((size_t)m * m, 0.0);
    for (int r = 0; r < m; ++r) {
        const int I = live[r];
        const int i = I % L.NX, j = (I / L.NX) % L.NY, k = I / (L.NX * L.NY);
        for (int q = 0; q < 27; ++q) {
            const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
            if (i + dx < 0 || i + dx > L.nx || j + dy < 0 || j + dy > L.ny || k + dz < 0 || k + dz > L.nz) continue;
            const int J = I + dx + L.NX * (dy + L.NY * dz);
            if (pos[J] >= 0) A[(size_t)r * m + pos[J]] += (double)coef[(size_t)q * n + I];
        }
        B[(size_t)r * m + r] = 1.0;
    }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (std::fabs(A[(size_t)r * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = r;
        if (A[(size_t)piv * m + col] == 0.0) return false;
        if (piv != col)
            for (int t = 0; t < m; ++t) {
                std::swap(A[(size_t)piv * m + t], A[(size_t)col * m + t]);
                std::swap(B[(size_t)piv * m + t], B[(size_t)col * m + t]);
            }
        const double d = 1.0 / A[(size_t)col * m + col];
        for (int t = 0; t < m; ++t) { A[(size_t)col * m + t] *= d; B[(size_t)col * m + t] *= d; }
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            const double fct = A[(size_t)r * m + col];
            if (fct == 0.0) continue;
            for (int t = 0; t < m; ++t) {
                A[(size_t)r * m + t] -= fct * A[(size_t)col * m + t];
                B[(size_t)r * m + t] -= fct * B[(size_t)col * m + t];
            }
        }
    }
    const int ld = (n + 3) & ~3;
    out.assign((size_t)n * ld, 0.0f);
    for (int r = 0; r < m; ++r)
        for (int t = 0; t < m; ++t) out[(size_t)live[r] * ld + live[t]] = (float)B[(size_t)r * m + t];
    return true;
}

// the hierarchy for the context's current operator (MIXED contexts; leaves
// mg_nlev = 0 otherwise), and whether the context's own solve uses it
// (mg_single).  Built only where it is used: by the context's own solve, or
// once a batch that solves with multigrid has asked for it (mg_wanted).
cudaError_t plan_pcg_mg(Ctx& c) {
    free_mg(c);
    c.mg_single = false;
    if (c.precision != PIFEPIC_MIXED) return cudaSuccess;
    // AUTO: multigrid where the register-resident Jacobi solver does not fit
    // (planned just before this), where the Jacobi iterations grow past the
    // cap; and once a Jacobi solve of this context has ended at the cap
    // unconverged (mostly Neumann faces: poorly conditioned for Jacobi)
    const bool single = c.precond == PIFEPIC_PRECOND_MULTIGRID ||
                        (c.precond == PIFEPIC_PRECOND_AUTO && (c.pcg_npt == 0 || c.mg_escalated));
    if (!single && !c.mg_wanted) return cudaSuccess;
    const long long N0 = c.mesh.nnodes;
    int nx = c.mesh.nx, ny = c.mesh.ny, nz = c.mesh.nz;
    long long Nlast = N0;
    int nlev = 0;
    while (nlev + 1 < MG_MAX_LEVELS && Nlast > MG_COARSEST && (nx >= 2 || ny >= 2 || nz >= 2)) {
        nx = (nx + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
        MgLevel& L = c.mg[++nlev];
        L.nx = nx; L.ny = ny; L.nz = nz;
        L.NX = nx + 1; L.NY = ny + 1; L.NZ = nz + 1;
        L.N = (long long)L.NX * L.NY * L.NZ;
        Nlast = L.N;
    }
    // the coarsest level must be small enough for its dense inverse
    if (nlev == 0 || Nlast > MG_COARSEST) {
        for (int l = 1; l <= nlev; ++l) c.mg[l] = MgLevel{};
        return cudaSuccess;
    }
    cudaError_t e = cudaSuccess;
    for (int l = 1; l <= nlev && e == cudaSuccess; ++l) {
        MgLevel& L = c.mg[l];
        c.mg_nlev = l;   // so that free_mg releases what was allocated
        e = lib_malloc(&L.coef, sizeof(float) * 27 * L.N);
        if (e == cudaSuccess) e = lib_malloc(&L.dinv, sizeof(float) * L.N);
        if (e == cudaSuccess) e = lib_malloc(&L.b, sizeof(float) * L.N);
        if (e == cudaSuccess) e = lib_malloc(&L.x, sizeof(float) * L.N);
        if (e == cudaSuccess) e = lib_malloc(&L.res, sizeof(float) * L.N);
        if (e == cudaSuccess) e = lib_malloc(&L.y, sizeof(float) * L.N);
    }
    if (e == cudaSuccess) e = lib_malloc(&c.mg_r0, sizeof(float) * N0);
    if (e == cudaSuccess) e = lib_malloc(&c.mg_cinv, sizeof(float) * Nlast * ((Nlast + 3) & ~3));
    if (e != cudaSuccess) { free_mg(c); return e; }
    FieldArgs f;
    f.m = c.mesh; f.o = c.obj; f.ntype = c.ntype; f.coef = c.patch_coef; f.coeff = c.patch_coeff;
    f.invdiag = c.invdiag; f.invdiagf = c.invdiagf;
    k_mg_rap0<<<(unsigned)((c.mg[1].N + 127) / 128), 128, 0, c.stream>>>(f, c.mg[1]);
    for (int l = 2; l <= nlev; ++l)
        k_mg_rap<<<(unsigned)((c.mg[l].N + 127) / 128), 128, 0, c.stream>>>(c.mg[l - 1], c.mg[l]);
    e = cudaGetLastError();
    const MgLevel& Lc = c.mg[nlev];
    std::vector<float> coef((size_t)27 * Lc.N), dinv(Lc.N), inv;
    if (e == cudaSuccess) e = scopy(c.stream, coef.data(), Lc.coef, sizeof(float) * coef.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = scopy(c.stream, dinv.data(), Lc.dinv, sizeof(float) * dinv.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !coarsest_inverse(Lc, coef, dinv, inv)) { free_mg(c); return cudaSuccess; }
    if (e == cudaSuccess) e = scopy(c.stream, c.mg_cinv, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_mg(c); return e; }
    c.mg_single = single;
    return cudaSuccess;
}

// the kernel arguments of the context's multigrid solve
MgArgs make_mg_args(Ctx& c) {
    MgArgs a;
    a.f.m = c.mesh; a.f.o = c.obj; a.f.ntype = c.ntype; a.f.coef = c.patch_coef; a.f.coeff = c.patch_coeff;
    a.f.invdiag = c.invdiag; a.f.invdiagf = c.invdiagf;
    a.kind = c.rowkind;
    a.b = c.b; a.u = c.u; a.g = c.gdir; a.phi = c.phi;
    a.r = c.rf; a.p = c.pf; a.q = c.qf; a.x = c.uf;
    a.z = c.zf; a.x0 = c.zf2;
    a.r0 = c.mg_r0;
    a.nlev = c.mg_nlev;
    for (int l = 0; l < MG_MAX_LEVELS; ++l) a.lev[l] = c.mg[l];
    a.cinv = c.mg_cinv;
    a.cinv_ld = (int)((c.mg[c.mg_nlev].N + 3) & ~3);
    a.val = c.coop_partial;
    a.arrivals = c.bar64;
    a.hold = (const int*)(c.scal + 45);
    a.S = (PcgState*)c.scal;
    a.it_total = (long long*)(c.scal + 40);
    a.outer_total = (long long*)(c.scal + 41);
    a.err = c.err_word;
    return a;
}
// a batched multigrid solve: the system of c on one cluster of C CTAs (1..16)
cudaError_t launch_pcg_mg_cluster(Ctx& c, int C, cudaStream_t st) {
    void* kern = (void*)k_pcg_mg_cluster;
    cudaError_t e = cudaSuccess;
    if (C > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(MG_CL_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    MgArgs a = make_mg_args(c);
    void* args[] = {(void*)&a, (void*)&C};
    return cudaLaunchKernelExC(&cfg, kern, args);
}

cudaError_t launch_pcg_mg(Ctx& c, cudaStream_t st) {
    MgArgs a = make_mg_args(c);
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_mg, MG_THREADS, 0);
    if (per < 1) return cudaErrorInvalidConfiguration;
    long long G = nsm;                    // one block per SM
    if (G > MG_THREADS) G = MG_THREADS;   // an exchange reads one block partial per thread
    void* args[] = {&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(MG_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (void*)k_pcg_mg, args);
}

}  // namespace pf
