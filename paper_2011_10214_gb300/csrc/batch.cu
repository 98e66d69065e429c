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
#include <string.h>

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


int cluster_size_for(long long N, long long H, bool mixed, long long cta_nodes);   // pcg_cluster.cu
cudaError_t build_pcg_graph(Ctx& c);                                                // field.cu
cudaError_t launch_pcg_mg_cluster(Ctx& c, int C, cudaStream_t st);                 // pcg_mg.cu
size_t cluster_smem_for(long long N, long long H, int C, bool mixed);
cudaError_t launch_pcg_cluster(const BatchItem& item, int C, size_t smem, bool mixed, cudaStream_t st);
cudaError_t launch_pcg_coop(Ctx& c, cudaStream_t st);                               // pcg_coop.cu
cudaError_t launch_push(Ctx& c);
cudaError_t launch_movers(Ctx& c);
cudaError_t launch_inject(Ctx& c);
cudaError_t launch_rebin(Ctx& c);
cudaError_t launch_push_mixed(Ctx& c);
cudaError_t launch_movers_mixed(Ctx& c);
cudaError_t launch_inject_mixed(Ctx& c);
cudaError_t launch_rebin_mixed(Ctx& c);

constexpr double CL_INNER_RED = 1e-6;   // the batched Jacobi clusters' inner reduction (at most)

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
    // the clusters' classic (two-exchange) loop reaches the tolerance in one
    // refinement step with inner solves that reduce the residual 1e-6-fold
    // (the context's reduction, 1e-4 by default, suits its own pipelined loop):
    // one FP64 residual pass fewer per solve
    const double red = c.inner_red < CL_INNER_RED ? c.inner_red : CL_INNER_RED;
    a.inner_red2 = red * red;
    a.margin2 = c.inner_margin * c.inner_margin;
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

}  // namespace pf

using namespace pf;

struct pifepic_batch {
    std::vector<pifepic_ctx*> ctx;
    cudaStream_t stream = nullptr;
    int cta_nodes = 8192;
    int precond = PIFEPIC_PRECOND_AUTO;   // MIXED members: MULTIGRID = multigrid clusters, else Jacobi clusters
    bool dirty = true;
    std::vector<long long> kernels;   // kernels per step of each instance (its share of the batch graph)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
};

static pifepic_status batch_fail(pifepic_batch* b, pifepic_status st, const std::string& m) {
    b->err = m;
    log_error(m.c_str());
    return st;
}

static long long node_halo(const Mesh& m) { return (long long)m.NX * m.NY + m.NX + 1; }

// The batch step as one graph: per instance a chain of its particle phases,
// right-hand side, field solve (one cluster launch; an instance too large for
// a cluster uses the single-instance persistent solver) and node field, so
// every instance advances as soon as its own work allows.
static cudaError_t build_batch_graph(pifepic_batch* b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    int n = (int)b->ctx.size();
    if (n == 0) { b->dirty = false; return cudaSuccess; }
    bool mixed = b->ctx[0]->c.precision == PIFEPIC_MIXED;
    // the solve of each instance: csize = its Jacobi cluster size (0: too large
    // for a cluster, the single-instance persistent solver); members solved by
    // the multigrid cluster kernel (MIXED, with a hierarchy) get csize -2 and
    // their cluster size in mg_c
    std::vector<int> csize(n, -1), mg_c(n, 0);
    std::vector<int> mg_members;
    for (int i = 0; i < n; ++i) {
        Ctx& c = b->ctx[i]->c;
        if (c.external_E) continue;
        if (mixed && b->precond == PIFEPIC_PRECOND_MULTIGRID && c.mg_nlev == 0 && !c.mg_wanted) {
            // the hierarchy on first use; the member's own solve graph is
            // re-planned with it (its plan's buffers are replaced)
            c.mg_wanted = true;
            cudaError_t e = build_pcg_graph(c);
            if (e != cudaSuccess) return e;
        }
        if (mixed && b->precond == PIFEPIC_PRECOND_MULTIGRID && c.mg_nlev > 0) {
            long long C = (c.mesh.nnodes + b->cta_nodes - 1) / b->cta_nodes;
            mg_c[i] = (int)std::max(1ll, std::min(16ll, C));
            csize[i] = -2;
            mg_members.push_back(i);
            continue;
        }
        csize[i] = cluster_size_for(c.mesh.nnodes, node_halo(c.mesh), mixed, b->cta_nodes);
    }
    const int groups[6] = {16, 8, 4, 2, 1, 0};
    std::vector<int> order;
    for (int g : groups)
        for (int i = 0; i < n; ++i)
            if (csize[i] == g) order.push_back(i);
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
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
    std::vector<int> fallback;
    for (int gsz : groups) {
        for (int i : order) {
            if (csize[i] != gsz) continue;
            if (gsz == 0) { fallback.push_back(i); continue; }
            if (e != cudaSuccess) break;
            Ctx& c = b->ctx[i]->c;
            const size_t smem = cluster_smem_for(c.mesh.nnodes, node_halo(c.mesh), gsz, mixed);
            cudaGraph_t sub = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = launch_pcg_cluster(make_item(c), gsz, smem, mixed, cs);
                e = cudaStreamEndCapture(cs, &sub);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&solve_of[i], g, &pre[i], 1, sub);
            if (sub) cudaGraphDestroy(sub);
        }
    }
    // multigrid members: one cluster launch each
    for (size_t k = 0; k < mg_members.size() && e == cudaSuccess; ++k) {
        const int i = mg_members[k];
        cudaGraph_t sub = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = launch_pcg_mg_cluster(b->ctx[i]->c, mg_c[i], cs);
            e = cudaStreamEndCapture(cs, &sub);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&solve_of[i], g, &pre[i], 1, sub);
        if (sub) cudaGraphDestroy(sub);
    }
    // instances too large for a cluster: the single-instance persistent solver
    // (one cooperative launch over the device), one after another -- two
    // cooperative grids spinning on halves of the device could wait on each other
    cudaGraphNode_t last_big = nullptr;
    for (int i : fallback) {
        if (e != cudaSuccess) break;
        Ctx& c = b->ctx[i]->c;
        cudaGraph_t sub = nullptr;
        e = capture(c, cs, [](Ctx& cc) -> cudaError_t { return launch_pcg_coop(cc, cc.stream); }, &sub);
        cudaGraphNode_t deps[2] = {pre[i], last_big};
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&solve_of[i], g, deps, last_big ? 2 : 1, sub);
        if (sub) cudaGraphDestroy(sub);
        last_big = solve_of[i];
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

pifepic_status pifepic_batch_set_cta_nodes(pifepic_batch* b, int cta_nodes) {
    if (!b || cta_nodes < 2048 || cta_nodes > 65536 || (cta_nodes & (cta_nodes - 1))) return PIFEPIC_EINVAL;
    if (cta_nodes != b->cta_nodes) { b->cta_nodes = cta_nodes; b->dirty = true; }
    return PIFEPIC_OK;
}

pifepic_status pifepic_batch_set_preconditioner(pifepic_batch* b, int kind) {
    if (!b) return PIFEPIC_EINVAL;
    if (kind != PIFEPIC_PRECOND_AUTO && kind != PIFEPIC_PRECOND_JACOBI && kind != PIFEPIC_PRECOND_MULTIGRID)
        return batch_fail(b, PIFEPIC_EINVAL, "unknown preconditioner");
    if (kind != b->precond) { b->precond = kind; b->dirty = true; }
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
    delete b;
}

}  // extern "C"
