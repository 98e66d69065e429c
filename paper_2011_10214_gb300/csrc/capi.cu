// libpifepic C ABI: context lifecycle, set-up, the PIC step and read-back.
// Host code here only orders kernel launches, owns device memory and converts
// descriptors; every step of the particle cycle and the field solve runs in
// the kernels of setup.cu, particles.cu, particles_mixed.cu and field.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <new>
#include <unordered_map>

#include <cmath>

#include "internal.h"

namespace pf {

// ---- the library's device memory: a process-wide count and an optional cap ----
static std::mutex g_mem_mu;
static std::unordered_map<void*, size_t> g_mem_blocks;
static size_t g_mem_used = 0;
static size_t g_mem_limit = 0;   // 0: no cap

cudaError_t lib_malloc_bytes(void** p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (g_mem_limit && g_mem_used + bytes > g_mem_limit) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_blocks[*p] = bytes;
    g_mem_used += bytes;
    return cudaSuccess;
}

cudaError_t lib_free(void* p) {
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        auto it = g_mem_blocks.find(p);
        if (it != g_mem_blocks.end()) {
            g_mem_used -= it->second;
            g_mem_blocks.erase(it);
        }
    }
    return cudaFree(p);
}

// the tet tables are the same for every context: uploaded once per device
static std::atomic<int> g_tables_ready[64];

cudaError_t set_field_tables(const TetTables& t);
cudaError_t set_particle_tables(const TetTables& t);
cudaError_t set_mixed_tables(const TetTables& t);
cudaError_t launch_solve_external(Ctx& c, const double* Fdev, int* iters, double* relres);
int solve_graph_fixed_kernels(const Ctx& c);
cudaError_t alloc_parrf(PArrF& a, long long n, bool id);
void free_parrf(PArrF& a);
pifepic_status solve_field_noalloc(Ctx& c, const double* F, const double* q, double* phi, int* iters,
                                   double* relres);
void free_mg(Ctx& c);                         // pcg_mg.cu
cudaError_t build_pcg_graph(Ctx& c);          // field.cu

// 5-tet split tables, computed from the definition (reading of Sec. 3.1.1)
static TetTables make_tables() {
    TetTables t;
    memset(&t, 0, sizeof(t));
    for (int p = 0; p < 2; ++p) {
        int even[4], odd[4], ne = 0, no = 0;
        for (int l = 0; l < 8; ++l) {
            int s = (l & 1) + ((l >> 1) & 1) + ((l >> 2) & 1);
            if ((s & 1) == p) even[ne++] = l; else odd[no++] = l;
        }
        for (int v = 0; v < 4; ++v) t.vert[p][0][v] = even[v];
        for (int q = 0; q < 4; ++q) {
            int o = odd[q];
            t.vert[p][1 + q][0] = o; t.vert[p][1 + q][1] = o ^ 1; t.vert[p][1 + q][2] = o ^ 2; t.vert[p][1 + q][3] = o ^ 4;
        }
        for (int tt = 0; tt < 5; ++tt) {
            // P1 gradients (h = 1): invert [1 x y z] rows of the 4 vertices
            double M[4][4], I[4][4];
            for (int v = 0; v < 4; ++v) {
                int l = t.vert[p][tt][v];
                M[v][0] = 1; M[v][1] = l & 1; M[v][2] = (l >> 1) & 1; M[v][3] = (l >> 2) & 1;
                for (int q = 0; q < 4; ++q) I[v][q] = v == q;
            }
            for (int cc = 0; cc < 4; ++cc) {
                int piv = cc;
                for (int r = cc + 1; r < 4; ++r) if (fabs(M[r][cc]) > fabs(M[piv][cc])) piv = r;
                for (int q = 0; q < 4; ++q) { std::swap(M[cc][q], M[piv][q]); std::swap(I[cc][q], I[piv][q]); }
                double d = M[cc][cc];
                for (int q = 0; q < 4; ++q) { M[cc][q] /= d; I[cc][q] /= d; }
                for (int r = 0; r < 4; ++r) {
                    if (r == cc) continue;
                    double f = M[r][cc];
                    for (int q = 0; q < 4; ++q) { M[r][q] -= f * M[cc][q]; I[r][q] -= f * I[cc][q]; }
                }
            }
            // column v of the inverse holds basis v's coefficients (a, gx, gy, gz)
            for (int v = 0; v < 4; ++v)
                for (int d = 0; d < 3; ++d) t.grad[p][tt][v][d] = I[1 + d][v];
        }
    }
    t.vol[0] = 1.0 / 3.0;
    for (int q = 1; q < 5; ++q) t.vol[q] = 1.0 / 6.0;
    const int off[19][3] = {{0, 0, 0},  {-1, 0, 0},  {1, 0, 0},  {0, -1, 0}, {0, 1, 0},  {0, 0, -1}, {0, 0, 1},
                            {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                            {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};
    for (int q = 0; q < 27; ++q) t.slot[q] = -1;
    for (int s = 0; s < 19; ++s) {
        for (int d = 0; d < 3; ++d) t.off[s][d] = off[s][d];
        t.slot[(off[s][2] + 1) * 9 + (off[s][1] + 1) * 3 + (off[s][0] + 1)] = s;
    }
    return t;
}

__global__ void k_pack_E(long long n, const double* E3, double4* E, float4* Ef) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 e = make_double4(E3[3 * i], E3[3 * i + 1], E3[3 * i + 2], 0.0);
    E[i] = e;
    Ef[i] = make_float4((float)e.x, (float)e.y, (float)e.z, 0.0f);
}
__global__ void k_unpack_E(long long n, const double4* E, double* E3) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 e = E[i];
    E3[3 * i] = e.x; E3[3 * i + 1] = e.y; E3[3 * i + 2] = e.z;
}
__global__ void k_unpack_Ef(long long n, const float4* E, float* E3) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 e = E[i];
    E3[3 * i] = e.x; E3[3 * i + 1] = e.y; E3[3 * i + 2] = e.z;
}
// entries that are not finite
__global__ void k_count_nonfinite(long long n, const double* a, unsigned long long* bad) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool b = i < n && !isfinite(a[i]);
    const unsigned m = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(bad, (unsigned long long)__popc(m));
}
// particles outside the box [0, n) in cell units, or with a velocity that is not finite
__global__ void k_count_bad_particles(long long n, const double* x, const double* y, const double* z,
                                      const double* vx, const double* vy, const double* vz, double nx, double ny,
                                      double nz, unsigned long long* bad) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool b = false;
    if (i < n) {
        const double px = x[i], py = y[i], pz = z[i];
        const bool in = px >= 0.0 && px < nx && py >= 0.0 && py < ny && pz >= 0.0 && pz < nz;
        b = !in || !isfinite(vx[i]) || !isfinite(vy[i]) || !isfinite(vz[i]);
    }
    const unsigned m = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(bad, (unsigned long long)__popc(m));
}
__global__ void k_max_id(long long n, const long long* id, unsigned long long* out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, (unsigned long long)id[i]);
}
__global__ void k_seq_id(long long n, long long base, long long* id) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) id[i] = base + i;
}

// the optional log sink (pifepic_set_log_callback)
static std::atomic<pifepic_log_fn> g_log_fn{nullptr};
static std::atomic<void*> g_log_user{nullptr};
void log_error(const char* message) {
    const pifepic_log_fn fn = g_log_fn.load(std::memory_order_acquire);
    if (fn) fn(message, g_log_user.load(std::memory_order_relaxed));
}

}  // namespace pf

using namespace pf;


#define FAIL(code, ...)                                                              \
    do {                                                                             \
        char _b[512];                                                                \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                                       \
        ctx->c.err = _b;                                                             \
        log_error(_b);                                                               \
        return code;                                                                 \
    } while (0)
#define CUDA_OK(x)                                                                            \
    do {                                                                                      \
        cudaError_t _e = (x);                                                                 \
        if (_e != cudaSuccess) FAIL(PIFEPIC_ECUDA, "%s: %s", #x, cudaGetErrorString(_e));     \
    } while (0)
#define ALLOC(ptr, bytes)                                                                        \
    do {                                                                                         \
        cudaError_t _e = lib_malloc((void**)&(ptr), (bytes) > 0 ? (size_t)(bytes) : (size_t)16); \
        if (_e != cudaSuccess) FAIL(PIFEPIC_ENOMEM, "lib_malloc(%lld bytes) failed: %s",         \
                                    (long long)(bytes), cudaGetErrorString(_e));                 \
    } while (0)
#define NEED(ptr) do { if (!(ptr)) return PIFEPIC_EINVAL; } while (0)

static unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// input checks on the device (counter in a scalar slot of the context, read back)
static unsigned long long* bad_counter(Ctx& c) { return (unsigned long long*)(c.scal + 46); }
static cudaError_t count_nonfinite(Ctx& c, long long n, const double* a, unsigned long long* bad) {
    *bad = 0;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bad_counter(c), 0, sizeof(unsigned long long), c.stream);
    if (e != cudaSuccess) return e;
    k_count_nonfinite<<<nb256(n), 256, 0, c.stream>>>(n, a, bad_counter(c));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return scopy(c.stream, bad, bad_counter(c), sizeof(unsigned long long), cudaMemcpyDeviceToHost);
}

// the six FP64 arrays (and ids) in one allocation: one cudaMalloc and one
// cudaFree per buffer instead of seven (both cost a fraction of a millisecond)
static PArr alloc_parr_raw(long long n, bool id, cudaError_t* err) {
    PArr a{};
    const size_t m = (size_t)(n > 0 ? n : 1);
    char* b = nullptr;
    *err = lib_malloc(&b, sizeof(double) * m * (id ? 7 : 6));
    if (*err != cudaSuccess) return a;
    a.base = b;
    double** arr[6] = {&a.x, &a.y, &a.z, &a.vx, &a.vy, &a.vz};
    for (int d = 0; d < 6; ++d) *arr[d] = (double*)(b + sizeof(double) * m * d);
    if (id) a.id = (long long*)(b + sizeof(double) * m * 6);
    return a;
}
static void free_parr(PArr& a) {
    if (a.base) {
        lib_free(a.base);
    } else {
        lib_free(a.x); lib_free(a.y); lib_free(a.z); lib_free(a.vx); lib_free(a.vy); lib_free(a.vz); lib_free(a.id);
    }
    a = PArr{};
}

extern "C" {

// particle bins of edge^3 PIC cells
static void set_bin_grid(Ctx& c, int edge) {
    const Mesh& pm = c.pmesh;
    c.bin_edge = edge;
    c.nbx = (pm.nx + edge - 1) / edge; c.nby = (pm.ny + edge - 1) / edge; c.nbz = (pm.nz + edge - 1) / edge;
    c.nblocks = c.nbx * c.nby * c.nbz;
}

pifepic_status pifepic_create(const pifepic_mesh_desc* mesh, const pifepic_solver_desc* solver, void* stream,
                              pifepic_ctx** out) {
    if (!mesh || !solver || !out) return PIFEPIC_EINVAL;
    *out = nullptr;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->h > 0.0) || !(solver->dt > 0.0))
        return PIFEPIC_EINVAL;
    const int rf = mesh->ife_refine > 1 ? mesh->ife_refine : 1;
    if (rf != 1 && rf != 2 && rf != 4 && rf != 8) return PIFEPIC_EINVAL;
    if ((long long)mesh->nx * rf > 2047 || (long long)mesh->ny * rf > 2047 || (long long)mesh->nz * rf > 1023)
        return PIFEPIC_EINVAL;
    if (solver->precision != PIFEPIC_FP64 && solver->precision != PIFEPIC_MIXED) return PIFEPIC_EINVAL;
    pifepic_ctx* ctx = new (std::nothrow) pifepic_ctx();
    if (!ctx) return PIFEPIC_ENOMEM;
    *out = ctx;
    Ctx& c = ctx->c;
    c.stream = (cudaStream_t)stream;
    CUDA_OK(cudaGetDevice(&c.device));
    {
        // pifepic_step's side stream (the waiting list's push and the injection
        // beside the push) at the highest priority: its few blocks are scheduled
        // as the push's blocks retire, instead of after the whole push
        int lo = 0, hi = 0;
        CUDA_OK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CUDA_OK(cudaStreamCreateWithPriority(&c.side, cudaStreamNonBlocking, hi));
        CUDA_OK(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
        CUDA_OK(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
    }
    // the PIC mesh, and the IFE mesh: the PIC mesh with each cell split rf^3 times
    auto make_mesh = [](int nx, int ny, int nz, double h) {
        Mesh q{};
        q.nx = nx; q.ny = ny; q.nz = nz;
        q.NX = nx + 1; q.NY = ny + 1; q.NZ = nz + 1;
        q.nnodes = (long long)q.NX * q.NY * q.NZ;
        q.ncells = (long long)nx * ny * nz;
        q.h = h;
        q.h6 = h / 6.0; q.h12 = h / 12.0;
        q.h6f = (float)h / 6.0f; q.h12f = (float)h / 12.0f;
        return q;
    };
    c.refine = rf;
    c.pmesh = make_mesh(mesh->nx, mesh->ny, mesh->nz, mesh->h);
    c.mesh = make_mesh(mesh->nx * rf, mesh->ny * rf, mesh->nz * rf, mesh->h / rf);
    Mesh& m = c.mesh;
    for (int d = 0; d < 3; ++d) c.origin[d] = mesh->origin[d];
    c.dt = solver->dt;
    c.dth = solver->dt / mesh->h;
    c.precision = solver->precision;
    c.tol = solver->pcg_tol > 0 ? solver->pcg_tol : 1e-6;
    c.maxit = solver->pcg_max_iter > 0 ? solver->pcg_max_iter : 150;
    c.track = solver->track_ids ? 1 : 0;
    const Mesh& pm = c.pmesh;
    set_bin_grid(c, BLK);
    for (int f = 0; f < 6; ++f) { c.bc[f].kind = PIFEPIC_BC_DIRICHLET; c.bc[f].value = 0.0; }
    long long N = m.nnodes, C = m.ncells;
    ALLOC(c.Lnode, sizeof(double) * N);
    ALLOC(c.ntype, sizeof(int) * N);
    ALLOC(c.gdir, sizeof(double) * N);
    ALLOC(c.lift, sizeof(double) * N);
    ALLOC(c.invdiag, sizeof(double) * N);
    ALLOC(c.invdiagf, sizeof(float) * N);
    ALLOC(c.phi, sizeof(double) * N);
    ALLOC(c.u, sizeof(double) * N);
    ALLOC(c.phi_prev, sizeof(double) * N);
    CUDA_OK(szero(c.stream, c.phi_prev, sizeof(double) * N));
    ALLOC(c.b, sizeof(double) * N);
    ALLOC(c.r, sizeof(double) * N);
    ALLOC(c.p, sizeof(double) * N);
    ALLOC(c.q, sizeof(double) * N);
    // z / zf: the persistent PCG reads them in 16-byte vectors, up to 16 entries
    // past N, and the global-memory PCG's branch-free stencil reads (and
    // multiplies by zero) the neighbours of a boundary node up to one plane,
    // one row and one node outside [0, N); both therefore sit inside a zeroed
    // guard of that reach on each side (16-entry multiples keep the alignment)
    {
        c.zguard = ((long long)c.mesh.NX * c.mesh.NY + c.mesh.NX + 1 + 15) / 16 * 16;
        const long long zlen = (N + 2 * c.zguard + 16 + 15) / 16 * 16;   // one guarded copy
        double* zb = nullptr;
        float* zfb = nullptr;
        // two copies each (the PCG alternates them by iteration parity)
        ALLOC(zb, sizeof(double) * 2 * zlen);
        c.z = zb + c.zguard;
        c.z2 = c.z + zlen;
        ALLOC(zfb, sizeof(float) * 2 * zlen);
        c.zf = zfb + c.zguard;
        c.zf2 = c.zf + zlen;
        CUDA_OK(szero(c.stream, zb, sizeof(double) * 2 * zlen));
        CUDA_OK(szero(c.stream, zfb, sizeof(float) * 2 * zlen));
    }
    ALLOC(c.rf, sizeof(float) * N);
    ALLOC(c.pf, sizeof(float) * N);
    ALLOC(c.qf, sizeof(float) * N);
    ALLOC(c.uf, sizeof(float) * N);
    ALLOC(c.E, sizeof(double4) * N);
    ALLOC(c.Ef, sizeof(float4) * N);
    if (rf > 1) {
        ALLOC(c.Ep, sizeof(double4) * c.pmesh.nnodes);
        ALLOC(c.Efp, sizeof(float4) * c.pmesh.nnodes);
        CUDA_OK(szero(c.stream, c.Ep, sizeof(double4) * c.pmesh.nnodes));
        CUDA_OK(szero(c.stream, c.Efp, sizeof(float4) * c.pmesh.nnodes));
    } else {
        c.Ep = c.E;
        c.Efp = c.Ef;
    }
    ALLOC(c.Wall, sizeof(unsigned long long) * MAX_SPECIES * N);
    ALLOC(c.ctrall, sizeof(unsigned long long) * MAX_SPECIES * NCTR);
    ALLOC(c.imask, C);
    ALLOC(c.ibase, sizeof(int) * C);
    ALLOC(c.cell_acc, sizeof(int) * C);
    ALLOC(c.red, sizeof(double) * 4 * (N / 128 + 1024));
    ALLOC(c.coop_partial, sizeof(double) * 8 * 2048);
    ALLOC(c.scal, sizeof(double) * 64);
    ALLOC(c.red_ticket, sizeof(unsigned) * 4);
    ALLOC(c.bar64, sizeof(unsigned long long) * BAR64_WORDS);
    ALLOC(c.err_word, sizeof(int));
    ALLOC(c.stat_dev, sizeof(StatPack));
    if (cudaMallocHost(&c.stat_host, sizeof(StatPack)) != cudaSuccess) {
        cudaGetLastError();
        c.stat_host = nullptr;
        FAIL(PIFEPIC_ENOMEM, "pinned statistics buffer");
    }
    ALLOC(c.next_id, sizeof(long long) * MAX_SPECIES);
    ALLOC(c.inj_count, sizeof(int) * MAX_SPECIES * 6);
    ALLOC(c.inj_base, sizeof(long long) * MAX_SPECIES * 6);
    ALLOC(c.inj_carry, sizeof(double) * MAX_SPECIES * 6);
    ALLOC(c.inj_dev, sizeof(InjectDev) * MAX_SPECIES * 6);
    CUDA_OK(szero(c.stream, c.phi, sizeof(double) * N));
    CUDA_OK(szero(c.stream, c.E, sizeof(double4) * N));
    CUDA_OK(szero(c.stream, c.Ef, sizeof(float4) * N));
    CUDA_OK(szero(c.stream, c.Wall, sizeof(unsigned long long) * MAX_SPECIES * N));
    CUDA_OK(szero(c.stream, c.ctrall, sizeof(unsigned long long) * MAX_SPECIES * NCTR));
    CUDA_OK(szero(c.stream, c.scal, sizeof(double) * 64));
    CUDA_OK(szero(c.stream, c.red_ticket, sizeof(unsigned) * 4));
    CUDA_OK(szero(c.stream, c.bar64, sizeof(unsigned long long) * BAR64_WORDS));
    CUDA_OK(szero(c.stream, c.err_word, sizeof(int)));
    CUDA_OK(szero(c.stream, c.next_id, sizeof(long long) * MAX_SPECIES));
    CUDA_OK(szero(c.stream, c.inj_carry, sizeof(double) * MAX_SPECIES * 6));
    // constant tables (unit-cube tets, independent of the mesh): once per device,
    // so that a context created while others run does not rewrite them
    if (c.device < 0 || c.device >= 64 || !g_tables_ready[c.device].load(std::memory_order_acquire)) {
        TetTables t = make_tables();
        CUDA_OK(set_tet_tables(t));
        CUDA_OK(set_field_tables(t));
        CUDA_OK(set_particle_tables(t));
        if (c.device >= 0 && c.device < 64) g_tables_ready[c.device].store(1, std::memory_order_release);
    }
    for (int e = 0; e < 16; ++e) CUDA_OK(cudaEventCreate(&c.ev[e]));
    c.ev_ok = true;
    return PIFEPIC_OK;
}

void pifepic_destroy(pifepic_ctx* ctx) {
    if (!ctx) return;
    Ctx& c = ctx->c;
    if (c.stream) cudaStreamSynchronize(c.stream); else cudaDeviceSynchronize();
    if (c.side) cudaStreamSynchronize(c.side);
    void* ptrs[] = {c.Lnode, c.ne_row, c.ne_coef, c.ne_qoff, c.ne_q, c.ne_qc, c.ntype, c.gdir, c.lift, c.invdiag, c.invdiagf, c.phi, c.phi_prev, c.u, c.b, c.r, c.p, c.q,
                    c.z ? (void*)(c.z - c.zguard) : nullptr, c.zf ? (void*)(c.zf - c.zguard) : nullptr,
                    c.rf, c.pf, c.qf, c.uf, c.E, c.Ef, c.Wall, c.surfall, c.ctrall, c.imask, c.ibase, c.cell_acc,
                    c.it_cell, c.it_t, c.it_data, c.it_acc, c.qT, c.cut_cell, c.cut_area, c.qcut, c.patch_node,
                    c.patch_coef, c.patch_coeff, c.red, c.coop_partial, c.rowkind, c.pcg_x, c.ph_tets, c.ph_Q, c.ph_carry, c.ph_cnt, c.ph_base, c.ph_tiles, c.ph_total, c.scal, c.red_ticket, c.bar64, c.err_word, c.stat_dev, c.inj_dev, c.inj_count,
                    c.inj_base, c.inj_carry, c.next_id};
    for (void* p : ptrs) lib_free(p);
    if (c.stat_host) cudaFreeHost(c.stat_host);
    if (c.refine > 1) { lib_free(c.Ep); lib_free(c.Efp); }
    free_mg(c);
    for (auto& s : c.sp) {
        free_parr(s.bins); free_parr(s.mov[0]); free_parr(s.mov[1]);
        lib_free(s.bstart); lib_free(s.bcap); lib_free(s.bcount); lib_free(s.bstay); lib_free(s.mov_n);
        free_parrf(s.binsF);
        for (int q = 0; q < 2; ++q) free_parrf(s.movF[q]);
    }
    if (c.pcg_exec) cudaGraphExecDestroy(c.pcg_exec);
    if (c.pcg_graph) cudaGraphDestroy(c.pcg_graph);
    if (c.ev_ok) for (int e = 0; e < 16; ++e) cudaEventDestroy(c.ev[e]);
    for (cudaEvent_t e : c.step_ev) cudaEventDestroy(e);
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    if (c.side) cudaStreamDestroy(c.side);
    if (c.spill_host) cudaFreeHost(c.spill_host);
    delete ctx;
}

const char* pifepic_last_error(const pifepic_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }


void pifepic_set_log_callback(pifepic_log_fn fn, void* user) {
    g_log_user.store(user, std::memory_order_relaxed);
    g_log_fn.store(fn, std::memory_order_release);
}

static pifepic_status encode_tmaps(pifepic_ctx* ctx) {
    Ctx& c = ctx->c;
    typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    CUDA_OK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) FAIL(PIFEPIC_ECUDA, "cuTensorMapEncodeTiled not available");
    EncodeFn enc = (EncodeFn)fn;
    const Mesh& m = c.pmesh;   // the push reads the node field at the PIC nodes
    cuuint64_t dims[4] = {4, (cuuint64_t)m.NX, (cuuint64_t)m.NY, (cuuint64_t)m.NZ};
    const cuuint32_t tl = (cuuint32_t)c.bin_edge + 1;   // a bin's node tile
    cuuint32_t box[4] = {4, tl, tl, tl};
    cuuint32_t es[4] = {1, 1, 1, 1};
    cuuint64_t sd[3] = {32, (cuuint64_t)m.NX * 32, (cuuint64_t)m.NX * m.NY * 32};
    CUresult r = enc(&c.tmapE, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, c.Ep, dims, sd, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) FAIL(PIFEPIC_ECUDA, "cuTensorMapEncodeTiled(E) failed: %d", (int)r);
    cuuint64_t sf[3] = {16, (cuuint64_t)m.NX * 16, (cuuint64_t)m.NX * m.NY * 16};
    r = enc(&c.tmapEf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c.Efp, dims, sf, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) FAIL(PIFEPIC_ECUDA, "cuTensorMapEncodeTiled(Ef) failed: %d", (int)r);
    c.tmap_ok = true;
    return PIFEPIC_OK;
}

static pifepic_status do_setup(pifepic_ctx* ctx) {
    Ctx& c = ctx->c;
    // free a previous interface set-up
    void* old[] = {c.it_cell, c.it_t, c.it_data, c.it_acc, c.qT, c.cut_cell, c.cut_area, c.qcut,
                   c.patch_node, c.patch_coef, c.patch_coeff, c.surfall};
    for (void* p : old) lib_free(p);
    c.it_cell = c.it_t = c.it_acc = c.cut_cell = nullptr;
    c.it_data = c.qT = c.cut_area = c.qcut = c.patch_coef = nullptr;
    c.patch_node = nullptr; c.patch_coeff = nullptr; c.surfall = nullptr;
    cudaError_t se = launch_setup(c);
    if (c.bed_outside) FAIL(PIFEPIC_EINVAL, "the bedrock must lie inside the object (a bedrock node has L >= 0)");
    CUDA_OK(se);
    CUDA_OK(launch_node_rows(c));
    ALLOC(c.surfall, sizeof(unsigned long long) * MAX_SPECIES * (c.ncut > 0 ? c.ncut : 1));
    CUDA_OK(szero(c.stream, c.surfall, sizeof(unsigned long long) * MAX_SPECIES * (c.ncut > 0 ? c.ncut : 1)));
    for (size_t s = 0; s < c.sp.size(); ++s) c.sp[s].surf = c.surfall + s * (c.ncut > 0 ? c.ncut : 1);
    CUDA_OK(launch_field_lift(c));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(build_pcg_graph(c));
    pifepic_status st = encode_tmaps(ctx);
    if (st) return st;
    c.have_object = true;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_object(pifepic_ctx* ctx, const pifepic_object_desc* o) {
    NEED(ctx); NEED(o);
    Ctx& c = ctx->c;
    if (!c.sp.empty()) FAIL(PIFEPIC_ESTATE, "set_object must precede add_species");
    if (!(o->eps_in > 0) || !(o->eps_out > 0)) FAIL(PIFEPIC_EINVAL, "permittivities must be positive");
    Object ob{};
    ob.eps_minus = o->eps_in;
    ob.eps_plus = o->eps_out;
    double h = c.pmesh.h;   // the object lives in PIC cell units (the set-up scales IFE nodes by 1/refine)
    const double* q = o->params;
    switch (o->kind) {
    case PIFEPIC_OBJ_NONE: ob.kind = 0; ob.eps_minus = ob.eps_plus = o->eps_out; break;
    case PIFEPIC_OBJ_SPHERE: {
        if (!(q[3] > 0)) FAIL(PIFEPIC_EINVAL, "sphere radius must be positive");
        ob.kind = 1;
        ob.a0 = (q[0] - c.origin[0]) / h; ob.a1 = (q[1] - c.origin[1]) / h; ob.a2 = (q[2] - c.origin[2]) / h;
        double r = q[3] / h;
        ob.a3 = r * r;
        break;
    }
    case PIFEPIC_OBJ_CAP_CRATER: {
        if (!(q[3] > 0) || !(q[4] > 0)) FAIL(PIFEPIC_EINVAL, "crater rim radius and depth must be positive");
        ob.kind = 2;
        double zg = (q[0] - c.origin[2]) / h, xc = (q[1] - c.origin[0]) / h, yc = (q[2] - c.origin[1]) / h;
        double a = q[3] / h, D = q[4] / h;
        double Rs = (a * a + D * D) / (2.0 * D);
        ob.a0 = zg; ob.a1 = xc; ob.a2 = yc; ob.a3 = a * a; ob.a4 = Rs * Rs; ob.a5 = (zg - D) + Rs;
        break;
    }
    case PIFEPIC_OBJ_PLANE:
        ob.kind = 3; ob.a0 = q[0]; ob.a1 = q[1]; ob.a2 = q[2]; ob.a3 = q[3];
        break;
    case PIFEPIC_OBJ_RIM_CRATER: {
        double zg = (q[0] - c.origin[2]) / h, xc = (q[1] - c.origin[0]) / h, yc = (q[2] - c.origin[1]) / h;
        double ri = q[3] / h, rt = q[4] / h, ro = q[5] / h, H = q[6] / h, D = q[7] / h;
        if (!(ri >= 0.0 && ri < rt && rt < ro) || !(H >= 0.0) || !(D >= 0.0))
            FAIL(PIFEPIC_EINVAL, "rim crater needs 0 <= r_inner < r_top < r_outer, height >= 0, depth >= 0");
        ob.kind = 4;
        ob.a0 = xc; ob.a1 = yc; ob.a2 = ri; ob.a3 = rt; ob.a4 = ro;
        ob.a5 = zg - D; ob.a6 = zg + H; ob.a7 = D + H; ob.a8 = H; ob.a9 = rt - ri; ob.a10 = ro - rt; ob.a11 = zg;
        break;
    }
    default: FAIL(PIFEPIC_EINVAL, "unknown object kind %d", o->kind);
    }
    if (c.bed_on && ob.kind != 0) {
        ob.bed = 1;
        ob.zb = (c.bed_z - c.origin[2]) / c.mesh.h;   // the set-up's IFE cell units
        ob.eps_bed = c.bed_eps;
    }
    c.obj = ob;
    return do_setup(ctx);
}

pifepic_status pifepic_set_bedrock(pifepic_ctx* ctx, double z_bed, double eps_bed) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (c.have_object) FAIL(PIFEPIC_ESTATE, "set_bedrock must precede set_object");
    if (!(eps_bed > 0.0) || !std::isfinite(z_bed)) FAIL(PIFEPIC_EINVAL, "eps_bed must be positive and z_bed finite");
    c.bed_on = true;
    c.bed_z = z_bed;
    c.bed_eps = eps_bed;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_refinement(pifepic_ctx* ctx, double reduction, double margin) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (!(reduction > 0.0 && reduction < 1.0) || !(margin > 0.0 && margin <= 1.0))
        FAIL(PIFEPIC_EINVAL, "refinement needs 0 < reduction < 1 and 0 < margin <= 1");
    c.inner_red = reduction;
    c.inner_margin = margin;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_preconditioner(pifepic_ctx* ctx, int kind) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (kind != PIFEPIC_PRECOND_AUTO && kind != PIFEPIC_PRECOND_JACOBI && kind != PIFEPIC_PRECOND_MULTIGRID)
        FAIL(PIFEPIC_EINVAL, "unknown preconditioner %d", kind);
    c.precond = kind;
    if (c.have_object) {   // re-plan the solve (and its graph) for the new preconditioner
        cudaError_t e = build_pcg_graph(c);
        if (e == cudaErrorMemoryAllocation) FAIL(PIFEPIC_ENOMEM, "preconditioner set-up: out of memory");
        CUDA_OK(e);
    }
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_field_bc(pifepic_ctx* ctx, const pifepic_face_bc bc[6]) {
    NEED(ctx); NEED(bc);
    Ctx& c = ctx->c;
    for (int f = 0; f < 6; ++f)
        if (bc[f].kind != PIFEPIC_BC_DIRICHLET && bc[f].kind != PIFEPIC_BC_NEUMANN)
            FAIL(PIFEPIC_EINVAL, "face %d: unknown boundary kind", f);
    for (int f = 0; f < 6; ++f) c.bc[f] = bc[f];
    if (c.have_object) {
        if (!c.sp.empty()) FAIL(PIFEPIC_ESTATE, "field boundaries must be set before species are added");
        return do_setup(ctx);
    }
    return PIFEPIC_OK;
}

static pifepic_status upload_species_params(pifepic_ctx* ctx) {
    Ctx& c = ctx->c;
    double co[MAX_SPECIES] = {0};
    for (size_t s = 0; s < c.sp.size(); ++s) co[s] = c.sp[s].q * c.sp[s].w;
    int ns = (int)c.sp.size();
    CUDA_OK(scopy(c.stream, c.scal + 16, co, sizeof(co), cudaMemcpyHostToDevice));
    CUDA_OK(scopy(c.stream, (int*)(c.scal + 24), &ns, sizeof(int), cudaMemcpyHostToDevice));
    return PIFEPIC_OK;
}

static pifepic_status ensure_movers(pifepic_ctx* ctx, int s, long long need) {
    Ctx& c = ctx->c;
    Species& q = c.sp[s];
    if (need <= q.mcap) return PIFEPIC_OK;
    CUDA_OK(cudaStreamSynchronize(c.stream));
    long long keep = 0;
    if (q.mov_n) {
        unsigned long long n0 = 0;
        CUDA_OK(scopy(c.stream, &n0, q.mov_n, sizeof(n0), cudaMemcpyDeviceToHost));
        keep = (long long)n0;
    }
    cudaError_t e;
    if (c.precision == PIFEPIC_MIXED) {
        PArrF f0{}, f1{};
        e = alloc_parrf(f0, need, c.track != 0);
        if (e == cudaSuccess) e = alloc_parrf(f1, need, c.track != 0);
        if (e != cudaSuccess) FAIL(PIFEPIC_ENOMEM, "mover list allocation failed");
        if (keep > 0) {
            CUDA_OK(scopy(c.stream, f0.cell, q.movF[0].cell, sizeof(int) * keep, cudaMemcpyDeviceToDevice));
            float* src[6] = {q.movF[0].fx, q.movF[0].fy, q.movF[0].fz, q.movF[0].vx, q.movF[0].vy, q.movF[0].vz};
            float* dst[6] = {f0.fx, f0.fy, f0.fz, f0.vx, f0.vy, f0.vz};
            for (int d = 0; d < 6; ++d)
                CUDA_OK(scopy(c.stream, dst[d], src[d], sizeof(float) * keep, cudaMemcpyDeviceToDevice));
            if (c.track) CUDA_OK(scopy(c.stream, f0.id, q.movF[0].id, sizeof(long long) * keep, cudaMemcpyDeviceToDevice));
        }
        PArrF old0 = q.movF[0], old1 = q.movF[1];
        q.movF[0] = f0; q.movF[1] = f1;
        free_parrf(old0); free_parrf(old1);
        q.mcap = need;
        return PIFEPIC_OK;
    }
    PArr a0 = alloc_parr_raw(need, c.track != 0, &e);
    if (e != cudaSuccess) { free_parr(a0); FAIL(PIFEPIC_ENOMEM, "mover list allocation failed"); }
    PArr a1 = alloc_parr_raw(need, c.track != 0, &e);
    if (e != cudaSuccess) { free_parr(a0); free_parr(a1); FAIL(PIFEPIC_ENOMEM, "mover list allocation failed"); }
    if (keep > 0) {   // carry the waiting list over
        double* src[6] = {q.mov[0].x, q.mov[0].y, q.mov[0].z, q.mov[0].vx, q.mov[0].vy, q.mov[0].vz};
        double* dst[6] = {a0.x, a0.y, a0.z, a0.vx, a0.vy, a0.vz};
        for (int d = 0; d < 6; ++d) CUDA_OK(scopy(c.stream, dst[d], src[d], sizeof(double) * keep, cudaMemcpyDeviceToDevice));
        if (c.track) CUDA_OK(scopy(c.stream, a0.id, q.mov[0].id, sizeof(long long) * keep, cudaMemcpyDeviceToDevice));
    }
    free_parr(q.mov[0]); free_parr(q.mov[1]);
    q.mov[0] = a0; q.mov[1] = a1;
    q.mcap = need;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_bin_edge(pifepic_ctx* ctx, int edge) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (edge != 4 && edge != 8) FAIL(PIFEPIC_EINVAL, "the bin edge is 4 or 8 cells");
    if (edge != 4 && c.precision != PIFEPIC_MIXED) FAIL(PIFEPIC_EINVAL, "FP64 contexts bin by 4 cells");
    if (!c.sp.empty()) FAIL(PIFEPIC_ESTATE, "set_bin_edge must precede add_species");
    if (edge == c.bin_edge) return PIFEPIC_OK;
    set_bin_grid(c, edge);
    if (c.tmap_ok) return encode_tmaps(ctx);   // the node tile's box follows the bin edge
    return PIFEPIC_OK;
}

int pifepic_get_bin_edge(const pifepic_ctx* ctx) { return ctx ? ctx->c.bin_edge : 0; }

int pifepic_get_solver(const pifepic_ctx* ctx) {
    if (!ctx) return 0;
    const Ctx& c = ctx->c;
    if (c.precision == PIFEPIC_MIXED && c.mg_single && c.mg_nlev > 0) return PIFEPIC_SOLVER_MULTIGRID;
    return c.pcg_npt > 0 ? PIFEPIC_SOLVER_REGISTERS : PIFEPIC_SOLVER_GLOBAL;
}

pifepic_status pifepic_add_species(pifepic_ctx* ctx, double qq, double mm, double w, int* id) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (!c.have_object) FAIL(PIFEPIC_ESTATE, "set_object must precede add_species");
    if ((int)c.sp.size() >= MAX_SPECIES) FAIL(PIFEPIC_EINVAL, "at most %d species", MAX_SPECIES);
    if (!(mm > 0) || !(w > 0)) FAIL(PIFEPIC_EINVAL, "mass and weight must be positive");
    Species s;
    s.q = qq; s.m = mm; s.w = w;
    s.k = (qq / mm) * c.dt;
    int idx = (int)c.sp.size();
    c.sp.push_back(s);
    Species& q = c.sp.back();
    q.W = c.Wall + (long long)idx * c.mesh.nnodes;
    q.surf = c.surfall + (long long)idx * (c.ncut > 0 ? c.ncut : 1);
    q.ctr = c.ctrall + idx * NCTR;
    ALLOC(q.mov_n, 2 * sizeof(unsigned long long));
    CUDA_OK(szero(c.stream, q.mov_n, 2 * sizeof(unsigned long long)));
    pifepic_status st = ensure_movers(ctx, idx, 1 << 16);
    if (st) return st;
    // empty bins
    PArr none{};
    CUDA_OK(c.precision == PIFEPIC_MIXED ? launch_build_bins_mixed(c, idx, none, 0, true)
                                         : launch_build_bins(c, idx, none, 0, true));
    st = upload_species_params(ctx);
    if (st) return st;
    if (id) *id = idx;
    return PIFEPIC_OK;
}

static long long count_particles(Ctx& c, int s);

// flatten species s (bins + waiting list) into a fresh flat array with room for extra
static pifepic_status flatten(pifepic_ctx* ctx, int s, long long extra, PArr* flat, unsigned long long** nflat,
                              long long* nexist) {
    Ctx& c = ctx->c;
    long long n0 = count_particles(c, s);
    if (n0 < 0) FAIL(PIFEPIC_ECUDA, "count failed");
    cudaError_t e;
    *flat = alloc_parr_raw(n0 + extra, true, &e);
    if (e != cudaSuccess) { free_parr(*flat); FAIL(PIFEPIC_ENOMEM, "flat particle buffer allocation failed"); }
    if (lib_malloc(nflat, sizeof(unsigned long long)) != cudaSuccess) {
        free_parr(*flat);
        FAIL(PIFEPIC_ENOMEM, "flat particle counter allocation failed");
    }
    CUDA_OK(szero(c.stream, *nflat, sizeof(unsigned long long)));
    if (!c.track) {   // without ids the flat copy still carries an id array: fill it later
    }
    CUDA_OK(c.precision == PIFEPIC_MIXED ? launch_flatten_mixed_to_f64(c, s, *flat, *nflat)
                                         : launch_flatten(c, s, *flat, *nflat));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    *nexist = n0;
    return PIFEPIC_OK;
}

static long long count_particles(Ctx& c, int s) {
    Species& q = c.sp[s];
    std::vector<int> cnt(c.nblocks);
    if (scopy(c.stream, cnt.data(), q.bcount, sizeof(int) * c.nblocks, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    long long n = 0;
    for (int v : cnt) n += v;
    unsigned long long w = 0;
    if (scopy(c.stream, &w, q.mov_n, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return n + (long long)w;
}

static pifepic_status rebuild(pifepic_ctx* ctx, int s, PArr flat, long long n) {
    Ctx& c = ctx->c;
    long long need = std::max<long long>(1 << 16, n / 8 + 4096);
    for (auto& d : c.inj) if (d.species == s) need += 4ll * (d.maxcnt + 1);
    if (s == c.ph_species) need += 4ll * (long long)c.ph_rate + 4096;
    pifepic_status st = ensure_movers(ctx, s, need);
    if (st) return st;
    CUDA_OK(c.precision == PIFEPIC_MIXED ? launch_build_bins_mixed(c, s, flat, n, true)
                                         : launch_build_bins(c, s, flat, n, true));
    return PIFEPIC_OK;
}

// a species that grows during the run (photoelectrons start empty): when its
// spill list passes a quarter of the mover capacity, rebuild its bins from the
// current particles (capacity count * 1.25 + 64 per bin)
static pifepic_status regrow_if_spilling(pifepic_ctx* ctx, int s) {
    Ctx& c = ctx->c;
    Species& q = c.sp[s];
    unsigned long long w = 0;
    CUDA_OK(scopy(c.stream, &w, q.mov_n, sizeof(w), cudaMemcpyDeviceToHost));
    if ((long long)w * 4 <= q.mcap) return PIFEPIC_OK;
    PArr flat; unsigned long long* nflat = nullptr; long long n0 = 0;
    pifepic_status st = flatten(ctx, s, 0, &flat, &nflat, &n0);
    if (st) return st;
    unsigned long long nt = 0;
    CUDA_OK(scopy(c.stream, &nt, nflat, sizeof(nt), cudaMemcpyDeviceToHost));
    st = rebuild(ctx, s, flat, (long long)nt);
    free_parr(flat); lib_free(nflat);
    return st;
}

pifepic_status pifepic_load_maxwellian(pifepic_ctx* ctx, int s, int ppc, double vth, const double drift[3],
                                       uint64_t seed) {
    NEED(ctx); NEED(drift);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    if (ppc < 0 || !(vth >= 0)) FAIL(PIFEPIC_EINVAL, "ppc and vth must be non-negative");
    PArr flat; unsigned long long* nflat = nullptr; long long n0 = 0;
    long long add = c.pmesh.ncells * (long long)ppc;
    pifepic_status st = flatten(ctx, s, add, &flat, &nflat, &n0);
    if (st) return st;
    CUDA_OK(launch_load_maxwellian(c, s, ppc, vth, drift, seed, flat, nflat, n0 + add));
    unsigned long long nt = 0;
    CUDA_OK(scopy(c.stream, &nt, nflat, sizeof(nt), cudaMemcpyDeviceToHost));
    st = rebuild(ctx, s, flat, (long long)nt);
    free_parr(flat); lib_free(nflat);
    if (st) return st;
    Species& q = c.sp[s];
    q.next_id = std::max<long long>(q.next_id, c.pmesh.ncells * (long long)ppc);
    CUDA_OK(scopy(c.stream, c.next_id + s, &q.next_id, sizeof(long long), cudaMemcpyHostToDevice));
    return PIFEPIC_OK;
}

pifepic_status pifepic_load_particles(pifepic_ctx* ctx, int s, size_t n, const double* x, const double* y,
                                      const double* z, const double* vx, const double* vy, const double* vz,
                                      const int64_t* ids, int mem_kind) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    if (n > 0 && (!x || !y || !z || !vx || !vy || !vz)) FAIL(PIFEPIC_EINVAL, "null particle array");
    PArr flat; unsigned long long* nflat = nullptr; long long n0 = 0;
    pifepic_status st = flatten(ctx, s, (long long)n, &flat, &nflat, &n0);
    if (st) return st;
    unsigned long long cur = 0;
    CUDA_OK(scopy(c.stream, &cur, nflat, sizeof(cur), cudaMemcpyDeviceToHost));
    cudaMemcpyKind k = mem_kind == PIFEPIC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* src[6] = {x, y, z, vx, vy, vz};
    double* dst[6] = {flat.x, flat.y, flat.z, flat.vx, flat.vy, flat.vz};
    Species& q = c.sp[s];
    if (n > 0) {
        for (int d = 0; d < 6; ++d) CUDA_OK(scopy(c.stream, dst[d] + cur, src[d], sizeof(double) * n, k));
        // every new particle must lie inside the box with finite state; otherwise
        // nothing is appended
        CUDA_OK(cudaMemsetAsync(bad_counter(c), 0, sizeof(unsigned long long), c.stream));
        k_count_bad_particles<<<nb256((long long)n), 256, 0, c.stream>>>(
            (long long)n, flat.x + cur, flat.y + cur, flat.z + cur, flat.vx + cur, flat.vy + cur, flat.vz + cur,
            (double)c.pmesh.nx, (double)c.pmesh.ny, (double)c.pmesh.nz, bad_counter(c));
        CUDA_OK(cudaGetLastError());
        unsigned long long bad = 0;
        CUDA_OK(scopy(c.stream, &bad, bad_counter(c), sizeof(bad), cudaMemcpyDeviceToHost));
        if (bad) {
            st = rebuild(ctx, s, flat, (long long)cur);
            free_parr(flat); lib_free(nflat);
            if (st) return st;
            FAIL(PIFEPIC_EINVAL, "load_particles: %llu of %zu particles outside the box or not finite", bad, n);
        }
        long long newmax = q.next_id + (long long)n - 1;
        if (ids) {
            CUDA_OK(scopy(c.stream, flat.id + cur, ids, sizeof(long long) * n, k));
            unsigned long long* mx = nullptr;
            ALLOC(mx, sizeof(unsigned long long));
            CUDA_OK(szero(c.stream, mx, sizeof(unsigned long long)));
            k_max_id<<<nb256((long long)n), 256, 0, c.stream>>>((long long)n, (const long long*)flat.id + cur, mx);
            unsigned long long hm = 0;
            CUDA_OK(scopy(c.stream, &hm, mx, sizeof(hm), cudaMemcpyDeviceToHost));
            lib_free(mx);
            newmax = (long long)hm;
        } else {
            k_seq_id<<<nb256((long long)n), 256, 0, c.stream>>>((long long)n, q.next_id, flat.id + cur);
        }
        CUDA_OK(cudaGetLastError());
        q.next_id = std::max<long long>(q.next_id, newmax + 1);
        CUDA_OK(scopy(c.stream, c.next_id + s, &q.next_id, sizeof(long long), cudaMemcpyHostToDevice));
    }
    st = rebuild(ctx, s, flat, (long long)cur + (long long)n);
    free_parr(flat); lib_free(nflat);
    return st;
}

static double flux_density(double n, double vth, double vdn) {
    double s = vdn / vth;
    return n * vth * (exp(-0.5 * s * s) / sqrt(2.0 * M_PI) + 0.5 * s * (1.0 + erf(s / sqrt(2.0))));
}

pifepic_status pifepic_set_particle_bc(pifepic_ctx* ctx, int s, const int face_kind[6]) {
    NEED(ctx); NEED(face_kind);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    int mask = 0;
    for (int f = 0; f < 6; ++f) {
        const int k = face_kind[f];
        if (k != PIFEPIC_PBC_ABSORB && k != PIFEPIC_PBC_INJECT && k != PIFEPIC_PBC_REFLECT)
            FAIL(PIFEPIC_EINVAL, "bad particle boundary kind %d on face %d", k, f);
        if (k == PIFEPIC_PBC_REFLECT) mask |= 1 << f;
    }
    if (c.sp[s].inject && (c.sp[s].face_mask & mask))
        FAIL(PIFEPIC_EINVAL, "species %d injects on a face marked REFLECT", s);
    c.sp[s].reflect = mask;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_injection(pifepic_ctx* ctx, int s, int face_mask, double density, double vth,
                                     const double drift[3], uint64_t seed) {
    NEED(ctx); NEED(drift);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    if (!(vth > 0) || density < 0) FAIL(PIFEPIC_EINVAL, "injection needs vth > 0 and density >= 0");
    if (face_mask & ~63) FAIL(PIFEPIC_EINVAL, "face_mask 0x%x has bits beyond the six faces", face_mask);
    if (face_mask & c.sp[s].reflect) FAIL(PIFEPIC_EINVAL, "face_mask 0x%x includes a reflecting face", face_mask);
    Species& q = c.sp[s];
    q.inject = face_mask != 0;
    q.face_mask = face_mask; q.density = density; q.vth = vth;
    for (int d = 0; d < 3; ++d) q.drift[d] = drift[d];
    q.seed = seed;
    const Mesh& m = c.pmesh;
    double nax[3] = {(double)m.nx, (double)m.ny, (double)m.nz};
    for (int f = 0; f < 6; ++f) {
        int ax = f >> 1;
        int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        double area = (nax[t1] * m.h) * (nax[t2] * m.h);
        double sgn = (f & 1) ? -1.0 : 1.0;
        q.rate[f] = ((face_mask >> f) & 1) ? flux_density(density, vth, sgn * drift[ax]) * area * c.dt / q.w : 0.0;
        q.maxcnt[f] = ((face_mask >> f) & 1) ? (int)ceil(q.rate[f]) + 1 : 0;
    }
    // rebuild the stream list in (species, face) order; keep carries of unchanged streams
    std::vector<double> oldcarry(MAX_SPECIES * 6, 0.0), hc(c.inj.size());
    if (!c.inj.empty()) {
        CUDA_OK(scopy(c.stream, hc.data(), c.inj_carry, sizeof(double) * c.inj.size(), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < c.inj.size(); ++i) oldcarry[c.inj[i].species * 6 + c.inj[i].face] = hc[i];
    }
    for (int f = 0; f < 6; ++f) oldcarry[s * 6 + f] = 0.0;
    c.inj.clear();
    std::vector<double> carry;
    for (int ss = 0; ss < (int)c.sp.size(); ++ss) {
        Species& p = c.sp[ss];
        if (!p.inject) continue;
        for (int f = 0; f < 6; ++f) {
            if (!((p.face_mask >> f) & 1)) continue;
            InjectDev d{};
            d.species = ss; d.face = f; d.maxcnt = p.maxcnt[f]; d.vth = p.vth;
            for (int k = 0; k < 3; ++k) d.drift[k] = p.drift[k];
            d.rate = p.rate[f]; d.seed = p.seed;
            c.inj.push_back(d);
            carry.push_back(oldcarry[ss * 6 + f]);
        }
    }
    if (!c.inj.empty()) {
        CUDA_OK(scopy(c.stream, c.inj_dev, c.inj.data(), sizeof(InjectDev) * c.inj.size(), cudaMemcpyHostToDevice));
        CUDA_OK(scopy(c.stream, c.inj_carry, carry.data(), sizeof(double) * carry.size(), cudaMemcpyHostToDevice));
    }
    long long n = count_particles(c, s);
    long long need = std::max<long long>(1 << 16, n / 8 + 4096);
    for (auto& d : c.inj) if (d.species == s) need += 4ll * (d.maxcnt + 1);
    if (s == c.ph_species) need += 4ll * (long long)c.ph_rate + 4096;
    return ensure_movers(ctx, s, need);
}

pifepic_status pifepic_set_photoemission(pifepic_ctx* ctx, int s, const double sun_dir[3], double density,
                                         double vth, uint64_t seed) {
    NEED(ctx); NEED(sun_dir);
    Ctx& c = ctx->c;
    if (!c.have_object) FAIL(PIFEPIC_ESTATE, "set_object first");
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    if (!(density >= 0.0) || !(vth > 0.0)) FAIL(PIFEPIC_EINVAL, "density must be >= 0 and vth > 0");
    const double sl = (sun_dir[0] * sun_dir[0] + sun_dir[1] * sun_dir[1]) + sun_dir[2] * sun_dir[2];
    if (!(sl > 0.0)) FAIL(PIFEPIC_EINVAL, "sun direction must be non-zero");
    c.ph_species = s;
    c.ph_seed = seed;
    CUDA_OK(launch_photo_setup(c, sun_dir, density, vth, c.sp[s].w));
    int64_t q = 0;
    pifepic_status st = pifepic_get_photoemission(ctx, &q, nullptr);
    if (st) return st;
    c.ph_rate = (double)q / (double)(1ll << PHOTO_RATE_BITS);
    // the mover list takes each step's emissions before the rebin
    return ensure_movers(ctx, s, std::max<long long>(1 << 16, 4ll * (long long)c.ph_rate + 4096));
}

pifepic_status pifepic_get_photoemission(pifepic_ctx* ctx, int64_t* rate_fixed, int64_t* emitting_tets) {
    NEED(ctx);
    Ctx& c = ctx->c;
    std::vector<long long> Q((size_t)c.ph_ne);
    if (c.ph_ne > 0) CUDA_OK(scopy(c.stream, Q.data(), c.ph_Q, sizeof(long long) * c.ph_ne, cudaMemcpyDeviceToHost));
    long long sum = 0;
    for (long long v : Q) sum += v;
    if (rate_fixed) *rate_fixed = sum;
    if (emitting_tets) *emitting_tets = c.ph_ne;
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_injection_rate(pifepic_ctx* ctx, int s, double rate[6]) {
    NEED(ctx); NEED(rate);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    for (int f = 0; f < 6; ++f) rate[f] = c.sp[s].rate[f];
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_external_E(pifepic_ctx* ctx, const double* E, int mem_kind) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (!E) { c.external_E = false; return PIFEPIC_OK; }
    long long N = c.mesh.nnodes;
    double* tmp = nullptr;
    ALLOC(tmp, sizeof(double) * 3 * N);
    CUDA_OK(scopy(c.stream, tmp, E, sizeof(double) * 3 * N,
                       mem_kind == PIFEPIC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    unsigned long long bad = 0;
    CUDA_OK(count_nonfinite(c, 3 * N, tmp, &bad));
    if (bad) {
        lib_free(tmp);
        FAIL(PIFEPIC_EINVAL, "set_external_E: %llu field values not finite", bad);
    }
    k_pack_E<<<nb256(N), 256, 0, c.stream>>>(N, tmp, c.E, c.Ef);
    CUDA_OK(cudaGetLastError());
    CUDA_OK(launch_E_to_pic(c, c.stream, true));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    lib_free(tmp);
    c.external_E = true;
    return PIFEPIC_OK;
}

static pifepic_status fill_stats(pifepic_ctx* ctx, const unsigned long long* before, pifepic_stats* st,
                                 const float* phase_ms, long long it0, long long l0, long long nsolves,
                                 long long ot0);

}  // extern "C"

namespace pf {
// counters before a batched call, and the statistics after it (batch.cu)
void snapshot_counters(pifepic_ctx* ctx, unsigned long long* before, long long* it0, long long* ot0, long long* l0) {
    StatPack pk;
    if (gather_stats(ctx->c, &pk, false) != cudaSuccess) memset(&pk, 0, sizeof(pk));
    memcpy(before, pk.ctr, sizeof(pk.ctr));
    *it0 = pk.it_total;
    *ot0 = pk.outer_total;
    *l0 = ctx->c.launches;
}
pifepic_status finish_stats(pifepic_ctx* ctx, const unsigned long long* before, long long it0, long long ot0,
                            long long nsteps, long long kernels, pifepic_stats* st) {
    long long l0 = ctx->c.launches - kernels;
    return fill_stats(ctx, before, st, nullptr, it0, l0, 0, ot0);
}
}  // namespace pf

extern "C" {

static pifepic_status fill_stats(pifepic_ctx* ctx, const unsigned long long* before, pifepic_stats* st,
                                 const float* phase_ms, long long it0, long long l0, long long nsolves,
                                 long long ot0) {
    Ctx& c = ctx->c;
    StatPack pk;
    cudaError_t e = gather_stats(c, &pk, c.have_object);
    if (e != cudaSuccess) FAIL(PIFEPIC_ECUDA, "statistics: %s", cudaGetErrorString(e));
    const unsigned long long* now = pk.ctr;
    pifepic_stats s;
    memset(&s, 0, sizeof(s));
    s.steps = c.step_no;
    for (size_t q = 0; q < c.sp.size(); ++q) {
        const unsigned long long* a = now + q * NCTR;
        const unsigned long long* b = before + q * NCTR;
        s.pushed[q] = (int64_t)(a[C_PUSHED] - b[C_PUSHED]);
        s.injected[q] = (int64_t)(a[C_INJECTED] - b[C_INJECTED]);
        s.absorbed[q] = (int64_t)(a[C_ABSORBED] - b[C_ABSORBED]);
        s.collected[q] = (int64_t)(a[C_COLLECTED] - b[C_COLLECTED]);
        s.lost_charge[q] = (int64_t)(a[C_LOST] - b[C_LOST]);
        s.inj_rejected[q] = (int64_t)(a[C_REJECTED] - b[C_REJECTED]);
        s.spilled[q] = (int64_t)a[C_SPILLED];
        s.dropped[q] = (int64_t)(a[C_DROPPED] - b[C_DROPPED]);
        s.count[q] = pk.count[q];
    }
    s.pcg_iters_total = pk.it_total - it0;
    // host-launched kernels + the solve graph's kernels (the PCG is one persistent launch)
    s.kernel_launches = (c.launches - l0) + nsolves * solve_graph_fixed_kernels(c);
    s.pcg_outer_total = pk.outer_total - ot0;
    s.pcg_iters = c.last_iters;
    s.pcg_relres = c.last_relres;
    s.pcg_converged = c.last_conv;
    s.surface_charge = pk.surface_charge;
    s.surface_potential = pk.surface_potential;
    if (phase_ms) for (int k = 0; k < 8; ++k) s.phase_ms[k] = phase_ms[k];
    const int herr = pk.err;
    c.stats = s;
    if (st) *st = s;
    if (herr & ERR_TMA_TIMEOUT) {
        szero(c.stream, c.err_word, sizeof(int));
        cudaStreamSynchronize(c.stream);
        FAIL(PIFEPIC_ETIMEOUT, "a node-field tile load timed out");
    }
    if (herr & ERR_CHUNK_TIMEOUT) {
        szero(c.stream, c.err_word, sizeof(int));
        cudaStreamSynchronize(c.stream);
        FAIL(PIFEPIC_ETIMEOUT, "a bin's compaction order wait timed out (its particles were dropped)");
    }
    if (herr & ERR_BARRIER_TIMEOUT) {
        // the barrier counters are left mid-count: clear them and the flag so
        // that a later solve starts from a clean state
        szero(c.stream, c.red_ticket, sizeof(unsigned) * 4);
        szero(c.stream, c.bar64, sizeof(unsigned long long) * BAR64_WORDS);
        szero(c.stream, c.err_word, sizeof(int));
        szero(c.stream, c.scal + 45, sizeof(int));     // the exchange test hook, if it was set
        cudaStreamSynchronize(c.stream);
        FAIL(PIFEPIC_ETIMEOUT, "a grid barrier of the PCG solve timed out");
    }
    for (size_t q = 0; q < c.sp.size(); ++q)
        if (s.dropped[q]) FAIL(PIFEPIC_ENOMEM, "species %zu: %lld particles dropped (mover list full)", q,
                               (long long)s.dropped[q]);
    return PIFEPIC_OK;
}

static cudaError_t run_solve(Ctx& c) {
    return launch_pcg(c);   // (the solve graph holds the precision's kernels)
}

// AUTO (MIXED): once a warm-started Jacobi solve of the context (any but its
// first, which starts from zero) has ended at the iteration cap without
// converging, its later solves run the multigrid cycle (the solve is
// re-planned once; a mesh too small for a hierarchy keeps Jacobi)
static pifepic_status escalate_if_capped(pifepic_ctx* ctx) {
    Ctx& c = ctx->c;
    if (c.precision != PIFEPIC_MIXED || c.precond != PIFEPIC_PRECOND_AUTO || c.mg_single || c.mg_escalated)
        return PIFEPIC_OK;
    if (c.solves_done < 2 || c.last_conv || c.last_iters < c.maxit) return PIFEPIC_OK;
    c.mg_escalated = true;
    CUDA_OK(build_pcg_graph(c));
    return PIFEPIC_OK;
}

pifepic_status pifepic_solve(pifepic_ctx* ctx, pifepic_stats* st) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (!c.have_object) FAIL(PIFEPIC_ESTATE, "set_object first");
    unsigned long long before[MAX_SPECIES * NCTR];
    long long it0, l0, ot0;
    snapshot_counters(ctx, before, &it0, &ot0, &l0);
    if (c.precision == PIFEPIC_MIXED) CUDA_OK(launch_deposit_all_mixed(c));
    else CUDA_OK(launch_deposit_all(c));
    if (!c.external_E) CUDA_OK(run_solve(c));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    pifepic_status r = fill_stats(ctx, before, st, nullptr, it0, l0, c.external_E ? 0 : 1, ot0);
    if (r || c.external_E) return r;
    c.solves_done += 1;
    return escalate_if_capped(ctx);
}

pifepic_status pifepic_leapfrog_init(pifepic_ctx* ctx) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (c.precision == PIFEPIC_MIXED) CUDA_OK(launch_half_kick_mixed(c));
    else CUDA_OK(launch_half_kick(c));
    CUDA_OK(cudaStreamSynchronize(c.stream));
    return PIFEPIC_OK;
}

pifepic_status pifepic_step(pifepic_ctx* ctx, int nsteps, pifepic_stats* st) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (!c.have_object) FAIL(PIFEPIC_ESTATE, "set_object first");
    if (nsteps < 0) FAIL(PIFEPIC_EINVAL, "nsteps < 0");
    unsigned long long before[MAX_SPECIES * NCTR];
    long long it0, l0, ot0;
    snapshot_counters(ctx, before, &it0, &ot0, &l0);
    float ph[8] = {0};
    bool mixed = c.precision == PIFEPIC_MIXED;
    // The host does not wait for each step: every step records its six phase
    // events into one of STEP_RING sets, and a set is read (after its last
    // event) only when it is reused and at the end, so the host keeps the
    // stream fed.  A photoemitting species' waiting list is watched with a
    // lag of one step: each step copies its length to pinned memory before
    // its last event, and the host reads step it-1's copy while step it is
    // queued; only a list past a quarter of its capacity stops the stream for
    // a rebuild (the lists are sized for more than one step of growth).
    constexpr int STEP_RING = 64;
    if (c.step_ev.empty()) {
        c.step_ev.resize(6 * STEP_RING);
        for (auto& e : c.step_ev) CUDA_OK(cudaEventCreate(&e));
    }
    if (!c.spill_host && cudaMallocHost(&c.spill_host, sizeof(unsigned long long) * STEP_RING) != cudaSuccess) {
        cudaGetLastError();
        c.spill_host = nullptr;
        FAIL(PIFEPIC_ENOMEM, "pinned step buffer");
    }
    const bool each = c.ph_species >= 0;
    auto check_spill = [&](int slot) -> pifepic_status {
        const Species& q = c.sp[c.ph_species];
        if ((long long)c.spill_host[slot] * 4 <= q.mcap) return PIFEPIC_OK;
        CUDA_OK(cudaStreamSynchronize(c.stream));
        return regrow_if_spilling(ctx, c.ph_species);
    };
    std::vector<char> unread(STEP_RING, 0);
    auto read_set = [&](int slot) -> cudaError_t {
        cudaEvent_t* ev = &c.step_ev[6 * slot];
        cudaError_t e = cudaEventSynchronize(ev[5]);
        if (e != cudaSuccess) return e;
        const int map[5] = {0, 1, 2, 3, 5};   // push, movers, inject, rebin, solve(+rhs+E)
        for (int k = 0; k < 5; ++k) {
            float t;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (e != cudaSuccess) return e;
            ph[map[k]] += t;
        }
        unread[slot] = 0;
        return cudaSuccess;
    };
    for (int it = 0; it < nsteps; ++it) {
        const int slot = it % STEP_RING;
        if (unread[slot]) CUDA_OK(read_set(slot));
        cudaEvent_t* ev = &c.step_ev[6 * slot];
        CUDA_OK(cudaEventRecord(ev[0], c.stream));
        CUDA_OK(mixed ? launch_push_prep_mixed(c) : launch_push_prep(c));
        // the waiting list's push and the injection only append to the step's
        // mover list and add to the surface accumulators (atomics), so they run
        // on the side stream beside the bins' push; the rebin waits for both
        CUDA_OK(cudaEventRecord(c.ev_fork, c.stream));
        CUDA_OK(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
        {
            cudaStream_t keep = c.stream;
            c.stream = c.side;
            cudaError_t e1 = mixed ? launch_movers_mixed(c) : launch_movers(c);
            if (e1 == cudaSuccess) e1 = mixed ? launch_inject_mixed(c) : launch_inject(c);
            c.stream = keep;
            // the join is recorded and awaited whatever happened, so that no
            // side-stream work outlives the main stream's view of the step
            cudaError_t e2 = cudaEventRecord(c.ev_join, c.side);
            cudaError_t e3 = e1 == cudaSuccess && e2 == cudaSuccess
                                 ? (mixed ? launch_push_bins_mixed(c) : launch_push_bins(c)) : cudaSuccess;
            cudaError_t e4 = cudaEventRecord(ev[1], c.stream);
            cudaError_t e5 = e2 == cudaSuccess ? cudaStreamWaitEvent(c.stream, c.ev_join, 0) : cudaStreamSynchronize(c.side);
            CUDA_OK(e1);
            CUDA_OK(e2);
            CUDA_OK(e3);
            CUDA_OK(e4);
            CUDA_OK(e5);
        }
        CUDA_OK(cudaEventRecord(ev[2], c.stream));   // (the side stream's time beyond the push)
        CUDA_OK(cudaEventRecord(ev[3], c.stream));
        CUDA_OK(mixed ? launch_rebin_mixed(c) : launch_rebin(c));
        CUDA_OK(cudaEventRecord(ev[4], c.stream));
        if (!c.external_E) CUDA_OK(run_solve(c));
        if (each)
            CUDA_OK(cudaMemcpyAsync(c.spill_host + slot, c.sp[c.ph_species].mov_n, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, c.stream));
        CUDA_OK(cudaEventRecord(ev[5], c.stream));
        c.step_no += 1;
        unread[slot] = 1;
        if (each && it > 0) {   // the previous step, while this one runs
            const int prev = (it - 1) % STEP_RING;
            if (unread[prev]) CUDA_OK(read_set(prev));
            pifepic_status g = check_spill(prev);
            if (g) return g;
        }
    }
    for (int k = 0; k < STEP_RING; ++k) {   // the sets not read yet, oldest first
        const int slot = (nsteps + k) % STEP_RING;
        if (unread[slot]) CUDA_OK(read_set(slot));
    }
    if (each && nsteps > 0) {
        pifepic_status g = check_spill((nsteps - 1) % STEP_RING);
        if (g) return g;
    }
    pifepic_status r = fill_stats(ctx, before, st, ph, it0, l0, c.external_E ? 0 : nsteps, ot0);
    if (r || c.external_E || nsteps == 0) return r;
    c.solves_done += nsteps;
    return escalate_if_capped(ctx);
}

pifepic_status pifepic_get_sizes(pifepic_ctx* ctx, int64_t* nn, int64_t* nc, int64_t* nit, int64_t* ncut) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (nn) *nn = c.mesh.nnodes;
    if (nc) *nc = c.mesh.ncells;
    if (nit) *nit = c.nit;
    if (ncut) *ncut = c.ncut;
    return PIFEPIC_OK;
}

static cudaMemcpyKind out_kind(int mem_kind) {
    return mem_kind == PIFEPIC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

pifepic_status pifepic_get_potential(pifepic_ctx* ctx, double* phi, int mem_kind) {
    NEED(ctx); NEED(phi);
    Ctx& c = ctx->c;
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(scopy(c.stream, phi, c.phi, sizeof(double) * c.mesh.nnodes, out_kind(mem_kind)));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_node_E(pifepic_ctx* ctx, double* E, int mem_kind) {
    NEED(ctx); NEED(E);
    Ctx& c = ctx->c;
    long long N = c.mesh.nnodes;
    // MIXED steps keep only the FP32 node field; the FP64 one is made here from phi
    if (c.precision == PIFEPIC_MIXED && !c.external_E && c.have_object) CUDA_OK(launch_node_E64(c));
    double* tmp = nullptr;
    ALLOC(tmp, sizeof(double) * 3 * N);
    k_unpack_E<<<nb256(N), 256, 0, c.stream>>>(N, c.E, tmp);
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(scopy(c.stream, E, tmp, sizeof(double) * 3 * N, out_kind(mem_kind)));
    lib_free(tmp);
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_node_E_f32(pifepic_ctx* ctx, float* E, int mem_kind) {
    NEED(ctx); NEED(E);
    Ctx& c = ctx->c;
    long long N = c.mesh.nnodes;
    float* tmp = nullptr;
    ALLOC(tmp, sizeof(float) * 3 * N);
    k_unpack_Ef<<<nb256(N), 256, 0, c.stream>>>(N, c.Ef, tmp);
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(scopy(c.stream, E, tmp, sizeof(float) * 3 * N, out_kind(mem_kind)));
    lib_free(tmp);
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_node_charge(pifepic_ctx* ctx, int s, int64_t* W, int mem_kind) {
    NEED(ctx); NEED(W);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    CUDA_OK(cudaStreamSynchronize(c.stream));
    CUDA_OK(scopy(c.stream, W, c.sp[s].W, sizeof(int64_t) * c.mesh.nnodes, out_kind(mem_kind)));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_surface_charge(pifepic_ctx* ctx, int s, int64_t* cnt, int mem_kind) {
    NEED(ctx); NEED(cnt);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    CUDA_OK(cudaStreamSynchronize(c.stream));
    if (c.ncut > 0) CUDA_OK(scopy(c.stream, cnt, c.sp[s].surf, sizeof(int64_t) * c.ncut, out_kind(mem_kind)));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_cut_cells(pifepic_ctx* ctx, int32_t* cells, double* area) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (c.ncut == 0) return PIFEPIC_OK;
    if (cells) CUDA_OK(scopy(c.stream, cells, c.cut_cell, sizeof(int32_t) * c.ncut, cudaMemcpyDeviceToHost));
    if (area) CUDA_OK(scopy(c.stream, area, c.cut_area, sizeof(double) * c.ncut, cudaMemcpyDeviceToHost));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_cell_target(pifepic_ctx* ctx, int32_t* target) {
    NEED(ctx); NEED(target);
    Ctx& c = ctx->c;
    CUDA_OK(scopy(c.stream, target, c.cell_acc, sizeof(int32_t) * c.mesh.ncells, cudaMemcpyDeviceToHost));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_interface(pifepic_ctx* ctx, int32_t* cell, int32_t* tet, double* vp, double* vm,
                                     double* area, double* K, double* cvec) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (c.nit == 0) return PIFEPIC_OK;
    if (cell) CUDA_OK(scopy(c.stream, cell, c.it_cell, sizeof(int32_t) * c.nit, cudaMemcpyDeviceToHost));
    if (tet) CUDA_OK(scopy(c.stream, tet, c.it_t, sizeof(int32_t) * c.nit, cudaMemcpyDeviceToHost));
    std::vector<double> rec((size_t)c.nit * IT_STRIDE);
    CUDA_OK(scopy(c.stream, rec.data(), c.it_data, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost));
    for (long long T = 0; T < c.nit; ++T) {
        const double* r = rec.data() + T * IT_STRIDE;
        if (vp) vp[T] = r[IT_VOLP];
        if (vm) vm[T] = r[IT_VOLM];
        if (area) area[T] = r[IT_AREA];
        if (K) for (int q = 0; q < 16; ++q) K[T * 16 + q] = r[IT_K + q];
        if (cvec) for (int q = 0; q < 4; ++q) cvec[T * 4 + q] = r[IT_C + q];
    }
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_particle_count(pifepic_ctx* ctx, int s, int64_t* n) {
    NEED(ctx); NEED(n);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    CUDA_OK(cudaStreamSynchronize(c.stream));
    *n = count_particles(c, s);
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_particles(pifepic_ctx* ctx, int s, int64_t cap, double* x, double* y, double* z,
                                     double* vx, double* vy, double* vz, int64_t* ids, int64_t* n, int mem_kind) {
    NEED(ctx); NEED(n);
    Ctx& c = ctx->c;
    if (s < 0 || s >= (int)c.sp.size()) FAIL(PIFEPIC_EINVAL, "bad species %d", s);
    if (ids && !c.track) FAIL(PIFEPIC_EINVAL, "ids requested but the context does not track ids");
    CUDA_OK(cudaStreamSynchronize(c.stream));
    PArr flat; unsigned long long* nflat = nullptr; long long n0 = 0;
    pifepic_status st;
    if (c.precision == PIFEPIC_MIXED) {
        long long cnt = count_particles(c, s);
        cudaError_t e;
        flat = alloc_parr_raw(cnt, true, &e);
        if (e != cudaSuccess) { free_parr(flat); FAIL(PIFEPIC_ENOMEM, "flat buffer"); }
        ALLOC(nflat, sizeof(unsigned long long));
        CUDA_OK(szero(c.stream, nflat, sizeof(unsigned long long)));
        CUDA_OK(launch_flatten_mixed_to_f64(c, s, flat, nflat));
        CUDA_OK(cudaStreamSynchronize(c.stream));
        n0 = cnt;
    } else {
        st = flatten(ctx, s, 0, &flat, &nflat, &n0);
        if (st) return st;
    }
    long long m = std::min<long long>(n0, cap);
    cudaMemcpyKind k = out_kind(mem_kind);
    double* dst[6] = {x, y, z, vx, vy, vz};
    double* src[6] = {flat.x, flat.y, flat.z, flat.vx, flat.vy, flat.vz};
    for (int d = 0; d < 6; ++d)
        if (dst[d] && m > 0) CUDA_OK(scopy(c.stream, dst[d], src[d], sizeof(double) * m, k));
    if (ids && m > 0) CUDA_OK(scopy(c.stream, ids, flat.id, sizeof(int64_t) * m, k));
    *n = m;
    free_parr(flat); lib_free(nflat);
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_stats(pifepic_ctx* ctx, pifepic_stats* st) {
    NEED(ctx); NEED(st);
    *st = ctx->c.stats;
    return PIFEPIC_OK;
}

pifepic_status pifepic_solve_field(pifepic_ctx* ctx, const double* F, const double* q, int mem_kind, int* iters,
                                   double* relres) {
    NEED(ctx); NEED(F);
    Ctx& c = ctx->c;
    if (!c.have_object) FAIL(PIFEPIC_ESTATE, "set_object first");
    long long N = c.mesh.nnodes;
    double* Fd = nullptr;
    ALLOC(Fd, sizeof(double) * N);
    cudaMemcpyKind k = mem_kind == PIFEPIC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_OK(scopy(c.stream, Fd, F, sizeof(double) * N, k));
    if (c.nit > 0) {
        if (q) CUDA_OK(scopy(c.stream, c.qT, q, sizeof(double) * c.nit, k));
        else CUDA_OK(szero(c.stream, c.qT, sizeof(double) * c.nit));
    }
    unsigned long long badF = 0, badq = 0;
    CUDA_OK(count_nonfinite(c, N, Fd, &badF));
    if (c.nit > 0 && q) CUDA_OK(count_nonfinite(c, c.nit, c.qT, &badq));
    if (badF || badq) {
        if (c.nit > 0) szero(c.stream, c.qT, sizeof(double) * c.nit);
        lib_free(Fd);
        FAIL(PIFEPIC_EINVAL, "solve_field: %llu load and %llu flux-jump values not finite", badF, badq);
    }
    cudaError_t e = launch_solve_external(c, Fd, iters, relres);
    lib_free(Fd);
    if (e != cudaSuccess) FAIL(PIFEPIC_ECUDA, "field solve: %s", cudaGetErrorString(e));
    return PIFEPIC_OK;
}

pifepic_status pifepic_get_memory_use(size_t* bytes) {
    if (!bytes) return PIFEPIC_EINVAL;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    *bytes = g_mem_used;
    return PIFEPIC_OK;
}

pifepic_status pifepic_set_memory_limit(size_t bytes) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_limit = bytes;
    return PIFEPIC_OK;
}

pifepic_status pifepic_test_hold_exchange(pifepic_ctx* ctx, int extra) {
    NEED(ctx);
    Ctx& c = ctx->c;
    if (extra < 0 || extra > 1) FAIL(PIFEPIC_EINVAL, "test_hold_exchange: extra must be 0 or 1, not %d", extra);
    CUDA_OK(scopy(c.stream, (int*)(c.scal + 45), &extra, sizeof(int), cudaMemcpyHostToDevice));
    return PIFEPIC_OK;
}

pifepic_status pifepic_solve_field_noalloc(pifepic_ctx* ctx, const double* F, const double* q, double* phi,
                                           int* iters, double* relres) {
    NEED(ctx); NEED(F); NEED(phi);
    if (!ctx->c.have_object) FAIL(PIFEPIC_ESTATE, "set_object first");
    return solve_field_noalloc(ctx->c, F, q, phi, iters, relres);
}

}  // extern "C"
