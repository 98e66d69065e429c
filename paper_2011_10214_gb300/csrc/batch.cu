// Batched IFE-PIC steps: many independent instances advanced by ONE CUDA graph
// launch per step.  Each instance's particle phases (push, movers, injection,
// rebin) and right-hand side are independent branches of the graph, so small
// instances overlap on the device; the field solves run on thread-block
// clusters, one cluster per instance (pcg_cluster.cu), with a one-CTA-per-
// instance kernel for instances too large for a cluster; the node fields
// follow as branches again.  The paper runs one problem per job (Sec. 3,
// Sec. 5); batching and serving many charging problems is this build's addition
// on top of the same per-instance method.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "field_common.cuh"
#include "internal.h"

namespace pf {

cudaError_t launch_solve_prefix(Ctx& c, cudaStream_t st);
cudaError_t launch_solve_suffix(Ctx& c, cudaStream_t st);
int solve_graph_fixed_kernels(const Ctx& c);
void snapshot_counters(pifepic_ctx* ctx, unsigned long long* before, long long* it0, long long* ot0, long long* l0);
pifepic_status finish_stats(pifepic_ctx* ctx, const unsigned long long* before, long long it0, long long ot0,
                            long long nsteps, long long kernels, pifepic_stats* st);


constexpr double BATCH_INNER_TOL = 1e-4;
constexpr int BATCH_MAX_OUTER = 12;

// block-wide sums of NV doubles, the result broadcast to every thread
template <int NV>
static __device__ __forceinline__ void bsum(double (&v)[NV], double* sh, double* bc) {
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) bc[q] = v[q];
    __syncthreads();
    for (int q = 0; q < NV; ++q) v[q] = bc[q];
    __syncthreads();
}

// The same Jacobi PCG (and MIXED refinement) as the persistent kernel, run by
// one CTA on one instance.
template <bool MIXED, int THREADS>
__global__ void __launch_bounds__(THREADS) k_pcg_batch(const BatchItem* items) {
    using T = typename std::conditional<MIXED, float, double>::type;
    __shared__ double sh[3 * 32];
    __shared__ double bc[4];
    const BatchItem& a = items[blockIdx.x];
    const FieldArgs& f = a.f;
    const Mesh& m = f.m;
    const long long N = m.nnodes;
    T* r = MIXED ? (T*)a.rf : (T*)a.r;
    T* z = MIXED ? (T*)a.zf : (T*)a.z;
    T* p = MIXED ? (T*)a.pf : (T*)a.p;
    T* q = MIXED ? (T*)a.qf : (T*)a.q;
    const T* dinv = MIXED ? (const T*)f.invdiagf : (const T*)f.invdiag;
    const T* coef = MIXED ? (const T*)f.coeff : (const T*)f.coef;
    const double tol2 = a.tol2;
    const int maxit = a.maxit;
    int it = 0, outer = 0;
    double bb = 0.0, rr = 0.0;
    bool conv = false;
    for (;;) {
        double v[3] = {0, 0, 0};
        for (long long n = threadIdx.x; n < N; n += THREADS) {
            int i, j, k;
            node_ijk(m, n, i, j, k);
            double bn = a.b[n];
            double rn = (f.ntype[n] == -3) ? 0.0 : bn - apply_row<double>(f, n, i, j, k, a.u, f.coef);
            T rt = (T)rn, zt = dinv[n] * rt;
            r[n] = rt; z[n] = zt; p[n] = zt;
            if (MIXED) a.df[n] = 0.0f;
            v[0] += bn * bn;
            v[1] += rn * rn;
            v[2] += (double)rt * (double)zt;
        }
        bsum<3>(v, sh, bc);
        if (outer == 0) bb = v[0];
        rr = v[1];
        double rz = v[2];
        const double rr_stop = MIXED ? fmax(0.25 * tol2 * bb, BATCH_INNER_TOL * BATCH_INNER_TOL * v[1]) : tol2 * bb;
        conv = (bb == 0.0) || (rr <= tol2 * bb);
        if (conv || it >= maxit || (MIXED && outer >= BATCH_MAX_OUTER)) break;
        ++outer;
        T wt = (T)0;
        for (long long n = threadIdx.x; n < N; n += THREADS) {
            int i, j, k;
            node_ijk(m, n, i, j, k);
            T y = apply_row<T>(f, n, i, j, k, z, coef);
            q[n] = y;
            wt += p[n] * y;
        }
        double w[1] = {(double)wt};
        bsum<1>(w, sh, bc);
        double alpha = rz / w[0];
        for (;;) {
            T s0 = (T)0, s1 = (T)0;
            const T al = (T)alpha;
            for (long long n = threadIdx.x; n < N; n += THREADS) {
                T rn = r[n] - al * q[n];
                if (MIXED) a.df[n] = a.df[n] + (float)al * (float)p[n];
                else a.u[n] = a.u[n] + alpha * (double)p[n];
                T zn = dinv[n] * rn;
                r[n] = rn; z[n] = zn;
                s0 += rn * rn;
                s1 += rn * zn;
            }
            double x2[2] = {(double)s0, (double)s1};
            bsum<2>(x2, sh, bc);
            const double beta = x2[1] / rz;
            rz = x2[1];
            rr = x2[0];
            ++it;
            if (!MIXED) conv = rr <= tol2 * bb;
            if (rr <= rr_stop || it >= maxit) break;
            T s2 = (T)0;
            const T bt = (T)beta;
            for (long long n = threadIdx.x; n < N; n += THREADS) {
                int i, j, k;
                node_ijk(m, n, i, j, k);
                T pn = z[n] + bt * p[n];
                T qn = apply_row<T>(f, n, i, j, k, z, coef) + bt * q[n];
                p[n] = pn; q[n] = qn;
                s2 += pn * qn;
            }
            double w2[1] = {(double)s2};
            bsum<1>(w2, sh, bc);
            alpha = rz / w2[0];
        }
        if (!MIXED) break;
        for (long long n = threadIdx.x; n < N; n += THREADS) a.u[n] = a.u[n] + (double)a.df[n];
        __syncthreads();
    }
    for (long long n = threadIdx.x; n < N; n += THREADS) a.phi[n] = (bb == 0.0) ? a.g[n] : a.u[n] + a.g[n];
    if (threadIdx.x == 0) {
        PcgState* S = a.S;
        S->bb = bb; S->rr = rr; S->it = it; S->outer_it = outer;
        S->converged = conv;
        S->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        *a.it_total += it;
        *a.outer_total += MIXED ? outer : 0;
    }
}

int cluster_size_for(long long N, long long H, bool mixed);                      // pcg_cluster.cu
size_t cluster_smem_for(long long N, long long H, int C, bool mixed);
cudaError_t launch_pcg_cluster(const BatchItem* items, int count, int C, size_t smem, bool mixed, cudaStream_t st);
cudaError_t launch_push(Ctx& c);
cudaError_t launch_movers(Ctx& c);
cudaError_t launch_inject(Ctx& c);
cudaError_t launch_rebin(Ctx& c);
cudaError_t launch_push_mixed(Ctx& c);
cudaError_t launch_movers_mixed(Ctx& c);
cudaError_t launch_inject_mixed(Ctx& c);
cudaError_t launch_rebin_mixed(Ctx& c);

static BatchItem make_item(Ctx& c) {
    BatchItem a;
    a.f.m = c.mesh; a.f.o = c.obj; a.f.ntype = c.ntype; a.f.coef = c.patch_coef; a.f.coeff = c.patch_coeff;
    a.f.invdiag = c.invdiag; a.f.invdiagf = c.invdiagf;
    a.b = c.b; a.u = c.u; a.r = c.r; a.z = c.z; a.p = c.p; a.q = c.q;
    a.rf = c.rf; a.zf = c.zf; a.pf = c.pf; a.qf = c.qf; a.df = c.uf;
    a.g = c.gdir; a.phi = c.phi;
    a.S = (PcgState*)c.scal;
    a.it_total = (long long*)(c.scal + 40);
    a.outer_total = (long long*)(c.scal + 41);
    a.tol2 = c.tol * c.tol;
    a.maxit = c.maxit;
    return a;
}

// capture fn(c) for one context on a capture stream into a new graph
template <class F>
static cudaError_t capture(Ctx& c, cudaStream_t cs, F fn, cudaGraph_t* out) {
    cudaStream_t keep = c.stream;
    c.stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = fn(c);
        e = cudaStreamEndCapture(cs, out);
        if (e == cudaSuccess) e = e2;
    }
    c.stream = keep;
    return e;
}

template <bool MIXED>
static cudaError_t launch_batch_pcg(const BatchItem* items, int n, int threads, cudaStream_t st) {
    if (threads == 256) k_pcg_batch<MIXED, 256><<<n, 256, 0, st>>>(items);
    else if (threads == 512) k_pcg_batch<MIXED, 512><<<n, 512, 0, st>>>(items);
    else k_pcg_batch<MIXED, 1024><<<n, 1024, 0, st>>>(items);
    return cudaGetLastError();
}

}  // namespace pf

using namespace pf;

struct pifepic_batch {
    std::vector<pifepic_ctx*> ctx;
    cudaStream_t stream = nullptr;
    BatchItem* items = nullptr;
    int items_cap = 0;
    int threads = 512;
    bool dirty = true;
    std::vector<long long> kernels;   // kernels per step of each instance (its share of the batch graph)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
};

static pifepic_status batch_fail(pifepic_batch* b, pifepic_status st, const std::string& m) {
    b->err = m;
    return st;
}

static long long node_halo(const Mesh& m) { return (long long)m.NX * m.NY + m.NX + 1; }

// The batch step as one graph: per instance a chain of its particle phases,
// right-hand side, field solve (one cluster launch; instances too large for a
// cluster share one launch of the one-CTA-per-instance kernel) and node field,
// so every instance advances as soon as its own work allows.
static cudaError_t build_batch_graph(pifepic_batch* b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    int n = (int)b->ctx.size();
    if (n == 0) { b->dirty = false; return cudaSuccess; }
    bool mixed = b->ctx[0]->c.precision == PIFEPIC_MIXED;
    if (n > b->items_cap) {
        cudaFree(b->items);
        cudaError_t e = cudaMalloc(&b->items, sizeof(BatchItem) * n);
        if (e != cudaSuccess) return e;
        b->items_cap = n;
    }
    // solve groups: cluster size per instance (0: the one-CTA kernel), items in group order
    std::vector<int> csize(n, -1);
    for (int i = 0; i < n; ++i) {
        const Ctx& c = b->ctx[i]->c;
        if (!c.external_E) csize[i] = cluster_size_for(c.mesh.nnodes, node_halo(c.mesh), mixed);
    }
    const int groups[6] = {16, 8, 4, 2, 1, 0};
    std::vector<int> order;
    std::vector<BatchItem> h;
    for (int g : groups)
        for (int i = 0; i < n; ++i)
            if (csize[i] == g) { order.push_back(i); h.push_back(make_item(b->ctx[i]->c)); }
    cudaError_t e = cudaSuccess;
    if (!h.empty()) {
        e = cudaMemcpyAsync(b->items, h.data(), sizeof(BatchItem) * h.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return e;
    }
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g;
    e = cudaGraphCreate(&g, 0);
    std::vector<cudaGraphNode_t> pre(n), post(n), solve_of(n, nullptr);
    b->kernels.assign(n, 0);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Ctx& c = b->ctx[i]->c;
        cudaGraph_t sub = nullptr;
        long long l0 = c.launches;
        e = capture(c, cs, [mixed](Ctx& cc) -> cudaError_t {
            cudaError_t r = mixed ? launch_push_mixed(cc) : launch_push(cc);
            if (r == cudaSuccess) r = mixed ? launch_movers_mixed(cc) : launch_movers(cc);
            if (r == cudaSuccess) r = mixed ? launch_inject_mixed(cc) : launch_inject(cc);
            if (r == cudaSuccess) r = mixed ? launch_rebin_mixed(cc) : launch_rebin(cc);
            if (r == cudaSuccess && !cc.external_E) r = launch_solve_prefix(cc, cc.stream);
            return r;
        }, &sub);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&pre[i], g, nullptr, 0, sub);
        if (sub) cudaGraphDestroy(sub);
        // captured particle kernels, the solve prefix and suffix, and its share of one solve launch
        b->kernels[i] = (c.launches - l0) + (c.external_E ? 0 : (solve_graph_fixed_kernels(c) - 1));
        c.launches = l0;
    }
    // one solve launch per instance, waiting only for that instance's branch
    // (instances too large for a cluster share the one-CTA-per-instance kernel)
    size_t off = 0;
    std::vector<int> fallback;
    for (int gsz : groups) {
        for (int i : order) {
            if (csize[i] != gsz) continue;
            const BatchItem* items = b->items + off;
            ++off;
            if (gsz == 0) { fallback.push_back(i); continue; }
            if (e != cudaSuccess) break;
            const Ctx& c = b->ctx[i]->c;
            const size_t smem = cluster_smem_for(c.mesh.nnodes, node_halo(c.mesh), gsz, mixed);
            cudaGraph_t sub = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = launch_pcg_cluster(items, 1, gsz, smem, mixed, cs);
                e = cudaStreamEndCapture(cs, &sub);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&solve_of[i], g, &pre[i], 1, sub);
            if (sub) cudaGraphDestroy(sub);
        }
    }
    if (e == cudaSuccess && !fallback.empty()) {
        const BatchItem* items = b->items + (off - fallback.size());
        std::vector<cudaGraphNode_t> deps;
        for (int i : fallback) deps.push_back(pre[i]);
        cudaGraph_t sub = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = mixed ? launch_batch_pcg<true>(items, (int)fallback.size(), b->threads, cs)
                                   : launch_batch_pcg<false>(items, (int)fallback.size(), b->threads, cs);
            e = cudaStreamEndCapture(cs, &sub);
            if (e == cudaSuccess) e = e2;
        }
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&node, g, deps.data(), deps.size(), sub);
        if (sub) cudaGraphDestroy(sub);
        for (int i : fallback) solve_of[i] = node;
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Ctx& c = b->ctx[i]->c;
        if (c.external_E) continue;
        cudaGraph_t s2 = nullptr;
        e = capture(c, cs, [](Ctx& cc) -> cudaError_t { return launch_solve_suffix(cc, cc.stream); }, &s2);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&post[i], g, &solve_of[i], 1, s2);
        if (s2) cudaGraphDestroy(s2);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e == cudaSuccess) { b->graph = g; b->dirty = false; }
    else cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

extern "C" {

pifepic_status pifepic_batch_create(pifepic_ctx** ctxs, int n, void* stream, pifepic_batch** out) {
    if (!out || n < 0 || (n > 0 && !ctxs)) return PIFEPIC_EINVAL;
    pifepic_batch* b = new (std::nothrow) pifepic_batch();
    if (!b) return PIFEPIC_ENOMEM;
    b->stream = (cudaStream_t)stream;
    *out = b;
    for (int i = 0; i < n; ++i) {
        pifepic_status st = pifepic_batch_add(b, ctxs[i]);
        if (st) return st;
    }
    return PIFEPIC_OK;
}

pifepic_status pifepic_batch_add(pifepic_batch* b, pifepic_ctx* ctx) {
    if (!b || !ctx) return PIFEPIC_EINVAL;
    if (!ctx->c.have_object) return batch_fail(b, PIFEPIC_ESTATE, "context has no object set up");
    if (!b->ctx.empty() && b->ctx[0]->c.precision != ctx->c.precision)
        return batch_fail(b, PIFEPIC_EINVAL, "all contexts of a batch share one precision");
    if (std::find(b->ctx.begin(), b->ctx.end(), ctx) != b->ctx.end())
        return batch_fail(b, PIFEPIC_EINVAL, "context already in the batch");
    b->ctx.push_back(ctx);
    b->dirty = true;
    return PIFEPIC_OK;
}

pifepic_status pifepic_batch_remove(pifepic_batch* b, pifepic_ctx* ctx) {
    if (!b || !ctx) return PIFEPIC_EINVAL;
    auto it = std::find(b->ctx.begin(), b->ctx.end(), ctx);
    if (it == b->ctx.end()) return batch_fail(b, PIFEPIC_EINVAL, "context not in the batch");
    b->ctx.erase(it);
    b->dirty = true;
    return PIFEPIC_OK;
}

pifepic_status pifepic_batch_set_threads(pifepic_batch* b, int threads) {
    if (!b || (threads != 256 && threads != 512 && threads != 1024)) return PIFEPIC_EINVAL;
    if (threads != b->threads) { b->threads = threads; b->dirty = true; }
    return PIFEPIC_OK;
}

pifepic_status pifepic_batch_step(pifepic_batch* b, int nsteps, pifepic_stats* stats) {
    if (!b || nsteps < 0) return PIFEPIC_EINVAL;
    if (b->ctx.empty()) return PIFEPIC_OK;
    // the instances' own streams must be idle before the batch stream takes over
    for (auto* x : b->ctx) {
        cudaError_t e = cudaStreamSynchronize(x->c.stream);
        if (e != cudaSuccess) return batch_fail(b, PIFEPIC_ECUDA, cudaGetErrorString(e));
    }
    if (b->dirty) {
        cudaError_t e = build_batch_graph(b);
        if (e != cudaSuccess) return batch_fail(b, PIFEPIC_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    int n = (int)b->ctx.size();
    std::vector<unsigned long long> before(stats ? (size_t)n * MAX_SPECIES * NCTR : 0);
    std::vector<long long> it0(n), ot0(n), l0(n);
    if (stats)
        for (int i = 0; i < n; ++i)
            snapshot_counters(b->ctx[i], before.data() + (size_t)i * MAX_SPECIES * NCTR, &it0[i], &ot0[i], &l0[i]);
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return batch_fail(b, PIFEPIC_ECUDA, cudaGetErrorString(e));
        for (auto* x : b->ctx) x->c.step_no += 1;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, PIFEPIC_ECUDA, cudaGetErrorString(e));
    if (stats) {
        for (int i = 0; i < n; ++i) {
            pifepic_status st = finish_stats(b->ctx[i], before.data() + (size_t)i * MAX_SPECIES * NCTR, it0[i], ot0[i],
                                             nsteps, b->kernels[i] * (long long)nsteps, &stats[i]);
            if (st) return batch_fail(b, st, pifepic_last_error(b->ctx[i]));
        }
    }
    return PIFEPIC_OK;
}

const char* pifepic_batch_last_error(const pifepic_batch* b) { return b ? b->err.c_str() : "null batch"; }

void pifepic_batch_destroy(pifepic_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->items);
    delete b;
}

}  // extern "C"
