// Persistent cooperative PCG (Sec. 2.5: the matrix solve is a PCG iteration
// stopped on the relative residual; Jacobi preconditioner is this build's
// reading).  One launch runs the whole solve: every block keeps iterating,
// separated by grid-wide barriers, so the loop pays no kernel launches.  The
// PCG vectors of a 64^3 mesh (a few MB) stay in L2.
//
//  FP64 mode : textbook Jacobi PCG in FP64.
//  MIXED mode: FP64 iterative refinement around an FP32 Jacobi PCG; residuals
//              of the refinement and every dot product are FP64, the inner
//              vectors and the inner operator are FP32.
//
// Reductions are deterministic: each block writes its partial, and after the
// barrier every block sums all partials in the same order, so all blocks take
// the same decisions and two runs give identical results.  Barrier waits are
// bounded (about a second); a timeout raises an error bit and ends the solve.
#include <math.h>

#include <type_traits>

#include "field_common.cuh"
#include "internal.h"

namespace pf {

constexpr double COOP_INNER_TOL = 1e-4;   // MIXED: least relative reduction per refinement step
constexpr int COOP_MAX_OUTER = 12;
constexpr int COOP_THREADS = 512;

struct CoopArgs {
    FieldArgs f;
    const double* b;
    double* u;
    double* r;        // FP64 mode vectors
    double* z;
    double* p;
    double* q;
    float* rf;        // MIXED inner vectors (df: the correction)
    float* zf;
    float* pf;
    float* qf;
    float* df;
    const double* g;  // Dirichlet values
    double* phi;
    double* partial;  // [8][gridDim.x]
    unsigned* bar_count;
    unsigned* bar_gen;
    PcgState* S;
    long long* it_total;
    long long* outer_total;
    int* err;
};

// grid barrier for a cooperative launch; false after a timeout (all blocks
// then leave the solve)
static __device__ __forceinline__ bool grid_barrier(const CoopArgs& a, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = a.bar_gen;
        unsigned g0 = *gen;
        __threadfence();
        unsigned arrived = atomicAdd(a.bar_count, 1u);
        bool ok = true;
        if (arrived == gridDim.x - 1) {
            *a.bar_count = 0u;
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > (1ll << 31)) { ok = false; atomicOr(a.err, ERR_BARRIER_TIMEOUT); break; }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// block sum of NV doubles written to partial[slot + q][blockIdx.x]
template <int NV>
static __device__ __forceinline__ void put_partial(const CoopArgs& a, double (&v)[NV], int slot, double* sh) {
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) a.partial[(long long)(slot + q) * gridDim.x + blockIdx.x] = v[q];
}

// every block: the grid totals of partial[slot..slot+NV) in a fixed order
template <int NV>
static __device__ __forceinline__ void get_total(const CoopArgs& a, int slot, double (&tot)[NV], double* sh,
                                                 double* bc) {
    double s[NV];
    for (int q = 0; q < NV; ++q) {
        s[q] = 0.0;
        for (unsigned bl = threadIdx.x; bl < gridDim.x; bl += blockDim.x)
            s[q] += __ldcg(a.partial + (long long)(slot + q) * gridDim.x + bl);
    }
    block_sum<NV>(s, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) bc[q] = s[q];
    __syncthreads();
    for (int q = 0; q < NV; ++q) tot[q] = bc[q];
    __syncthreads();
}

// Jacobi PCG with the direction product carried by recurrence: after the
// residual update every block writes z = D^-1 r; then p = z + beta p and
// q = A z + beta q (= A p) need only that one barrier, so an iteration costs
// two grid barriers (one per reduction).
template <bool MIXED>
__global__ void __launch_bounds__(COOP_THREADS, 1) k_pcg_coop(CoopArgs a) {
    using T = typename std::conditional<MIXED, float, double>::type;
    __shared__ double sh[3 * 32];
    __shared__ double bc[4];
    __shared__ int s_ok;
    const FieldArgs& f = a.f;
    const Mesh& m = f.m;
    const long long N = m.nnodes;
    const long long TT = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T* r = MIXED ? (T*)a.rf : (T*)a.r;
    T* z = MIXED ? (T*)a.zf : (T*)a.z;
    T* p = MIXED ? (T*)a.pf : (T*)a.p;
    T* q = MIXED ? (T*)a.qf : (T*)a.q;
    const T* dinv = MIXED ? (const T*)f.invdiagf : (const T*)f.invdiag;
    const T* coef = MIXED ? (const T*)f.coeff : (const T*)f.coef;
    PcgState* S = a.S;
    const double tol2 = S->tol2;
    const int maxit = S->maxit;
    int it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    bool conv = false, alive = true;

    for (;;) {   // refinement loop (a single pass in FP64 mode)
        // r = b - A u (FP64; u read through L2), z = D^-1 r, p = z
        double v[3] = {0, 0, 0};
        for (long long n = t0; n < N; n += TT) {
            int i, j, k;
            node_ijk(m, n, i, j, k);
            double bn = a.b[n];
            double rn = (f.ntype[n] == -3) ? 0.0 : bn - apply_row<double, true>(f, n, i, j, k, a.u, f.coef);
            T rt = (T)rn, zt = dinv[n] * rt;
            r[n] = rt; z[n] = zt; p[n] = zt;
            if (MIXED) a.df[n] = 0.0f;
            v[0] += bn * bn;
            v[1] += rn * rn;
            v[2] += (double)rt * (double)zt;
        }
        put_partial<3>(a, v, 0, sh);
        if (!(alive = grid_barrier(a, &s_ok))) break;
        double tot[3];
        get_total<3>(a, 0, tot, sh, bc);
        if (outer == 0) bb = tot[0];
        rr = tot[1];
        double rz = tot[2];
        // inner target: the final tolerance, or a 1e-4 reduction of this residual
        const double rr_stop = MIXED ? fmax(0.25 * tol2 * bb, COOP_INNER_TOL * COOP_INNER_TOL * tot[1]) : tol2 * bb;
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        if (conv || it >= maxit || (MIXED && outer >= COOP_MAX_OUTER)) break;
        ++outer;
        // q = A p (p = z here)
        T wt = (T)0;
        for (long long n = t0; n < N; n += TT) {
            int i, j, k;
            node_ijk(m, n, i, j, k);
            T y = apply_row<T, true>(f, n, i, j, k, z, coef);
            q[n] = y;
            wt += p[n] * y;
        }
        double w[1] = {(double)wt};
        put_partial<1>(a, w, 3, sh);
        if (!(alive = grid_barrier(a, &s_ok))) break;
        double pq[1];
        get_total<1>(a, 3, pq, sh, bc);
        double alpha = rz / pq[0];
        for (;;) {
            // u += alpha p, r -= alpha q, z = D^-1 r
            // per-thread partials in the working precision (a thread owns a few
            // nodes), widened once; block and grid sums are FP64
            T s0 = (T)0, s1 = (T)0;
            const T al = (T)alpha;
            for (long long n = t0; n < N; n += TT) {
                T rn = r[n] - al * q[n];
                if (MIXED) a.df[n] = a.df[n] + (float)al * (float)p[n];
                else a.u[n] = a.u[n] + alpha * (double)p[n];
                T zn = dinv[n] * rn;
                r[n] = rn; z[n] = zn;
                s0 += rn * rn;
                s1 += rn * zn;
            }
            double x2[2] = {(double)s0, (double)s1};
            put_partial<2>(a, x2, 4, sh);
            if (!(alive = grid_barrier(a, &s_ok))) break;
            double t2[2];
            get_total<2>(a, 4, t2, sh, bc);
            const double beta = t2[1] / rz;
            rz = t2[1];
            rr = t2[0];
            ++it;
            if (!MIXED) conv = rr <= tol2 * bb;
            if (rr <= rr_stop || it >= maxit) break;
            // p = z + beta p, q = A z + beta q (z of neighbours through L2)
            T s2 = (T)0;
            const T bt = (T)beta;
            for (long long n = t0; n < N; n += TT) {
                int i, j, k;
                node_ijk(m, n, i, j, k);
                T pn = z[n] + bt * p[n];
                T qn = apply_row<T, true>(f, n, i, j, k, z, coef) + bt * q[n];
                p[n] = pn; q[n] = qn;
                s2 += pn * qn;
            }
            double w2[1] = {(double)s2};
            put_partial<1>(a, w2, 3, sh);
            if (!(alive = grid_barrier(a, &s_ok))) break;
            double pq2[1];
            get_total<1>(a, 3, pq2, sh, bc);
            alpha = rz / pq2[0];
        }
        if (!alive || !MIXED) break;
        // refinement: u += d, then a barrier before the next residual reads u
        for (long long n = t0; n < N; n += TT) a.u[n] = a.u[n] + (double)a.df[n];
        if (!(alive = grid_barrier(a, &s_ok))) break;
    }
    for (long long n = t0; n < N; n += TT) a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->bb = bb;
        S->rr = rr;
        S->it = it;
        S->outer_it = outer;
        S->converged = alive && conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += MIXED ? outer : 0;
    }
}

static int coop_grid(Ctx& c, bool mixed) {
    int dev = c.device, nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_coop<true>, COOP_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_coop<false>, COOP_THREADS, 0);
    long long maxb = (long long)nsm * (per > 0 ? per : 1);
    long long need = (c.mesh.nnodes + COOP_THREADS - 1) / COOP_THREADS;
    long long g = need < maxb ? need : maxb;
    if (g > 2048) g = 2048;   // partial buffer holds 8 x 2048 doubles
    return (int)(g > 0 ? g : 1);
}

// the PCG state must already hold tol2 and maxit; writes phi
cudaError_t launch_pcg_coop(Ctx& c, cudaStream_t st) {
    bool mixed = c.precision == PIFEPIC_MIXED;
    CoopArgs a;
    a.f.m = c.mesh; a.f.o = c.obj; a.f.ntype = c.ntype; a.f.coef = c.patch_coef; a.f.coeff = c.patch_coeff;
    a.f.invdiag = c.invdiag; a.f.invdiagf = c.invdiagf;
    a.b = c.b; a.u = c.u; a.r = c.r; a.z = c.z; a.p = c.p; a.q = c.q;
    a.rf = c.rf; a.zf = c.zf; a.pf = c.pf; a.qf = c.qf; a.df = c.uf;
    a.g = c.gdir; a.phi = c.phi;
    a.partial = c.coop_partial;
    a.bar_count = c.red_ticket + 1;
    a.bar_gen = c.red_ticket + 2;
    a.S = (PcgState*)c.scal;
    a.it_total = (long long*)(c.scal + 40);
    a.outer_total = (long long*)(c.scal + 41);
    a.err = c.err_word;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(coop_grid(c, mixed));
    cfg.blockDim = dim3(COOP_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mixed) return cudaLaunchKernelEx(&cfg, k_pcg_coop<true>, a);
    return cudaLaunchKernelEx(&cfg, k_pcg_coop<false>, a);
}

}  // namespace pf
