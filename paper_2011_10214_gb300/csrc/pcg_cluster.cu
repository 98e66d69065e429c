// Batched field solves on thread-block clusters.
//
// Each instance of a batch is solved by one cluster of C CTAs (C = 1, 2, 4, 8
// or 16, by the instance's size); instances never wait on one another, so the
// only synchronisation is the cluster's own hardware barrier.  The method is
// the Jacobi PCG of the single-instance solver (Sec. 2.5; MIXED: FP32 inner
// solves inside FP64 refinement), with everything an iteration touches kept on
// chip:
//
//  - CTA k owns the contiguous nodes [k M, (k+1) M) of its instance; r, p, q,
//    the correction x and the packed node coordinates of its nodes live in its
//    shared memory;
//  - z lives in the centre of a per-CTA window [k M - H, (k+1) M + H) (H = one
//    z-plane, one row and one node: every stencil neighbour); before each
//    matrix product a CTA copies the H nodes on either side from the centres of
//    its neighbouring CTAs through distributed shared memory (M >= H, so they
//    are always the adjacent ranks);
//  - a reduction is a block sum, the partial in one of two shared slots by
//    exchange parity, a cluster barrier (release/acquire), and the C partials
//    read back in rank order through distributed shared memory, so every CTA
//    of the cluster holds the same totals and takes the same decisions.
//
// The refinement residual b - A u (FP64, u in global memory) is the only step
// that reads global vectors inside the loop.
#include <cooperative_groups.h>
#include <math.h>

#include <type_traits>

#include "field_common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace pf {

constexpr int CL_THREADS = 1024;
constexpr int CL_MAX_OUTER = 12;   // MIXED: refinement steps at most
constexpr int CL_TY_LOAD = 16383;  // a patch index of 14 bits at most is kept in the row kind

// nodes per CTA at most: the working set of one CTA must fit in shared memory
constexpr int cl_max_nodes(bool mixed) { return mixed ? 8192 : 4096; }

struct ClusterShared {
    double sh[4 * 32];
    double bc[4];
    double slot[2][4];    // this CTA's partials, by exchange parity
};

// shared-memory layout of one CTA (T = working precision): r, p, q, x [M] T,
// window [M + 2H] T, pk [M] unsigned, kind [M] unsigned short -- narrower
// arrays after wider ones, so each starts aligned for any M
template <typename T>
static __host__ __device__ __forceinline__ size_t cl_smem_bytes(long long M, long long H) {
    return (size_t)M * (4 * sizeof(T) + sizeof(unsigned) + sizeof(unsigned short)) + (size_t)(M + 2 * H) * sizeof(T);
}

// reduction across the cluster: every CTA gets the same NV totals
template <typename A, int NV>
static __device__ __forceinline__ void cl_reduce(cg::cluster_group& cl, int C, int& e, A (&v)[NV], A (&tot)[NV],
                                                 ClusterShared& cs) {
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
            if (lane < C) {
                const A* rs = cl.map_shared_rank(slot, lane);
                x = rs[q];
            }
            // fixed tree over the ranks: the same sum in every CTA
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) ((A*)cs.bc)[q] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = ((A*)cs.bc)[q];
    ++e;
}

static __device__ __forceinline__ unsigned cl_pack(int i, int j, int k) {
    return (unsigned)i | ((unsigned)j << 11) | ((unsigned)k << 22);
}

static_assert(sizeof(BatchItem) <= 4096, "the solve arguments travel as a kernel parameter");

template <bool MIXED>
__global__ void __launch_bounds__(CL_THREADS, 1) k_pcg_cluster(const BatchItem a, int C) {
    using T = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char cl_raw[];
    __shared__ ClusterShared cs;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const FieldArgs& f = a.f;
    const Mesh& m = f.m;
    const long long N = m.nnodes;
    const long long M = (N + C - 1) / C;
    const long long H = (long long)m.NX * m.NY + m.NX + 1;
    const long long b0 = (long long)rank * M;
    const long long b1 = b0 + M < N ? b0 + M : N;
    const int nown = b1 > b0 ? (int)(b1 - b0) : 0;
    T* r = (T*)cl_raw;
    T* p = r + M;
    T* q = p + M;
    T* x = q + M;
    T* win = x + M;                 // node n at win[H + n - b0]
    unsigned* pk = (unsigned*)(win + M + 2 * H);
    unsigned short* kind = (unsigned short*)(pk + M);
    const int NXw = m.NX, NXYw = m.NX * m.NY;
    const T hT = (T)m.h, epsP = (T)f.o.eps_plus, epsM = (T)f.o.eps_minus;
    const T* coef = MIXED ? (const T*)f.coeff : (const T*)f.coef;
    const T* dinv = MIXED ? (const T*)f.invdiagf : (const T*)f.invdiag;
    const double tol2 = a.tol2;
    const int maxit = a.maxit;
    auto ldw = [&](long long n) { return win[H + n - b0]; };
    auto ldu = [&](long long n) { return __ldcg(a.u + n); };
    auto row = [&](int li, auto ld, const auto* cf) {
        const unsigned u = pk[li];
        using R = typename std::remove_cv<typename std::remove_pointer<decltype(cf)>::type>::type;
        return apply_row_ld<R>(f, b0 + li, (int)(u & 2047u), (int)((u >> 11) & 2047u), (int)(u >> 22), ld, cf);
    };
    // an interface (patch) row keeps its patch index in the kind bits that a
    // patch row leaves unused (0-7 and 10-15), so that its product reads the
    // coefficients without first loading ntype; CL_TY_LOAD: index too large
    auto patch_row = [&](int li, unsigned kd, auto ld, const auto* cf) {
        const unsigned u = pk[li];
        const int i = (int)(u & 2047u), j = (int)((u >> 11) & 2047u), k = (int)(u >> 22);
        const int t = (int)((kd & 0xFFu) | ((kd >> 10) << 8));
        const int ty = t == CL_TY_LOAD ? f.ntype[b0 + li] : t;
        using R = typename std::remove_cv<typename std::remove_pointer<decltype(cf)>::type>::type;
        return apply_row_ty<R>(f, b0 + li, i, j, k, ty, ld, cf);
    };
    for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
        int i, j, k;
        node_ijk(m, b0 + li, i, j, k);
        pk[li] = cl_pack(i, j, k);
        unsigned kd = row_kind(f, b0 + li, i, j, k);
        if (kd & RK_GENERAL) {
            int ty = f.ntype[b0 + li];
            if (ty > CL_TY_LOAD) ty = CL_TY_LOAD;
            kd |= (unsigned)(ty & 0xFF) | ((unsigned)(ty >> 8) << 10);
        }
        kind[li] = (unsigned short)kd;
    }
    // window halves outside the instance's nodes stay zero (never read with a
    // non-zero coefficient, but inside the buffer)
    for (long long w = threadIdx.x; w < M + 2 * H; w += CL_THREADS) win[w] = (T)0;
    __syncthreads();
    // the neighbours' window centres through distributed shared memory
    const T* prevw = rank > 0 ? cl.map_shared_rank(win, rank - 1) : nullptr;
    const T* nextw = rank + 1 < C ? cl.map_shared_rank(win, rank + 1) : nullptr;
    const long long next_own = (rank + 1 < C) ? ((b1 + M < N ? b1 + M : N) - b1) : 0;
    const int nnext = (int)(next_own < H ? (next_own > 0 ? next_own : 0) : H);

    int e = 0, it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    bool conv = false;
    for (;;) {
        // true residual of u in FP64; z = D^-1 r into the window centre, p = z, x = 0
        double v3[3] = {0.0, 0.0, 0.0};
        for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
            const long long n = b0 + li;
            const double bn = a.b[n];
            // (MIXED: three or more of these per solve; interior rows in closed form)
            double rn = 0.0;
            if (f.ntype[n] != -3) {
                if constexpr (MIXED) {
                    const unsigned u = pk[li];
                    rn = bn - apply_row64(f, n, (int)(u & 2047u), (int)((u >> 11) & 2047u), (int)(u >> 22), ldu,
                                          f.coef);
                } else {
                    rn = bn - row(li, ldu, f.coef);
                }
            }
            const T rt = (T)rn, zt = dinv[n] * rt;
            r[li] = rt;
            win[H + li] = zt;
            p[li] = zt;
            x[li] = (T)0;
            v3[0] += bn * bn;
            v3[1] += rn * rn;
            v3[2] += (double)rt * (double)zt;
        }
        double t3[3];
        cl_reduce<double, 3>(cl, C, e, v3, t3, cs);
        if (outer == 0) bb = t3[0];
        rr = t3[1];
        T rz = (T)t3[2];
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        if (conv || it >= maxit || (MIXED && outer >= CL_MAX_OUTER)) break;
        const T rr_stop = (T)(MIXED ? fmax(a.margin2 * tol2 * bb, a.inner_red2 * rr) : tol2 * bb);
        ++outer;
        T beta = (T)0, rr_in = (T)rr;
        bool first = true;
        for (;;) {
            // halo of z from the neighbouring CTAs (their centres were last
            // written before the reduction this CTA has just passed)
            if (prevw)
                for (int w = threadIdx.x; w < (int)H; w += CL_THREADS) win[w] = prevw[M + w];
            if (nextw)
                for (int w = threadIdx.x; w < nnext; w += CL_THREADS) win[H + nown + w] = nextw[H + w];
            __syncthreads();
            T v1[1] = {(T)0};
            for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
                const unsigned kd = kind[li];
                const T* wc = win + ((int)H + li);
                T az;
                if (kd & RK_DIRICHLET) az = (T)0;
                else if (kd & RK_GENERAL) az = patch_row(li, kd, ldw, coef);
                else az = regular_row_masked<T>(wc, NXw, NXYw, kd, hT, h_over6<T>(m), h_over12<T>(m), epsP, epsM);
                const T zl = wc[0];
                T pl, ql;
                if (first) {
                    pl = zl;
                    ql = az;
                } else {
                    pl = zl + beta * p[li];
                    ql = az + beta * q[li];
                }
                p[li] = pl;
                q[li] = ql;
                v1[0] += pl * ql;
            }
            first = false;
            T pq[1];
            cl_reduce<T, 1>(cl, C, e, v1, pq, cs);
            const T al = rz / pq[0];
            T v2[2] = {(T)0, (T)0};
            for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
                const long long n = b0 + li;
                x[li] = x[li] + al * p[li];
                const T rl = r[li] - al * q[li];
                const T zl = dinv[n] * rl;
                r[li] = rl;
                win[H + li] = zl;
                v2[0] += rl * rl;
                v2[1] += rl * zl;
            }
            T t2[2];
            cl_reduce<T, 2>(cl, C, e, v2, t2, cs);
            beta = t2[1] / rz;
            rz = t2[1];
            rr_in = t2[0];
            ++it;
            if (rr_in <= rr_stop || it >= maxit) break;
        }
        for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
            const long long n = b0 + li;
            a.u[n] = a.u[n] + (double)x[li];
        }
        if (!MIXED) {
            rr = (double)rr_in;
            conv = rr <= tol2 * bb;
            break;
        }
        // the next residual reads the neighbours' new u from global memory
        __threadfence();
        cl.sync();
    }
    for (int li = threadIdx.x; li < nown; li += CL_THREADS) {
        const long long n = b0 + li;
        a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    }
    if (rank == 0 && threadIdx.x == 0) {
        PcgState* S = a.S;
        S->bb = bb; S->rr = rr; S->it = it; S->outer_it = outer;
        S->converged = conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += MIXED ? outer : 0;
    }
    // no CTA may leave while a neighbour can still read its shared memory
    cl.sync();
}

// cluster size for an instance of N nodes (H = halo): the smallest C with at
// most cta_nodes nodes per CTA, else the largest C that fits; 0 if none fits
// (then the single-instance persistent solver takes the instance)
int cluster_size_for(long long N, long long H, bool mixed, long long cta_nodes) {
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long cap = cl_max_nodes(mixed);
    int best = 0;
    for (int C = 1; C <= 16; C *= 2) {
        const long long M = (N + C - 1) / C;
        if (C > 1 && M < H) break;            // the halo would reach past the adjacent CTA
        const size_t bytes = mixed ? cl_smem_bytes<float>(M, H) : cl_smem_bytes<double>(M, H);
        if (M > cap || bytes + sizeof(ClusterShared) + 1024 > (size_t)smem_max) continue;
        best = C;
        if (M <= cta_nodes) break;
    }
    return best;
}

// one instance's solve on one cluster of C CTAs (the arguments by value, in the
// kernel's parameter space); smem = its per-CTA working set
cudaError_t launch_pcg_cluster(const BatchItem& item, int C, size_t smem, bool mixed, cudaStream_t st) {
    void* kern = mixed ? (void*)k_pcg_cluster<true> : (void*)k_pcg_cluster<false>;
    // the function's limit is the device's whole opt-in budget, the same for
    // every member (a per-launch value would leave the limit at the last
    // member's size, below what earlier members' graph nodes launch with)
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const int limit = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > (long long)limit) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
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
    BatchItem a = item;
    void* args[] = {(void*)&a, (void*)&C};
    return cudaLaunchKernelExC(&cfg, kern, args);
}

size_t cluster_smem_for(long long N, long long H, int C, bool mixed) {
    const long long M = (N + C - 1) / C;
    return mixed ? cl_smem_bytes<float>(M, H) : cl_smem_bytes<double>(M, H);
}

}  // namespace pf
