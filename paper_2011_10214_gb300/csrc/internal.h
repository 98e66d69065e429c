// Internal state of a libpifepic context and the host-side launchers of each
// kernel group.  Not part of the public ABI (include/pifepic.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "pifepic.h"

namespace pf {

// ---- device memory of the library ------------------------------------------
// Every device allocation of the library goes through lib_malloc / lib_free,
// which keep a process-wide count of the bytes held and refuse an allocation
// that would take the count past the limit set by pifepic_set_memory_limit.
cudaError_t lib_malloc_bytes(void** p, size_t bytes);
cudaError_t lib_free(void* p);
template <typename T>
static inline cudaError_t lib_malloc(T** p, size_t bytes) { return lib_malloc_bytes((void**)p, bytes); }

// ---- multigrid levels of the MIXED field solve (pcg_mg.cu) -----------------
constexpr int MG_MAX_LEVELS = 8;
struct MgLevel {                  // a coarse level (27-point Galerkin rows)
    int nx = 0, ny = 0, nz = 0;   // cells
    int NX = 0, NY = 0, NZ = 0;   // nodes
    long long N = 0;
    float* coef = nullptr;        // [27][N]: coefficient plane q of offset (q%3-1, q/3%3-1, q/9-1)
    float* dinv = nullptr;        // [N] inverse diagonal, 0 where the row is empty (Dirichlet support)
    float *b = nullptr, *x = nullptr, *res = nullptr, *y = nullptr;   // cycle vectors [N]
};

// ---- particle arrays (SoA) -------------------------------------------------
struct PArr {            // FP64 mode: xi in cell units, physical velocity
    double *x, *y, *z, *vx, *vy, *vz;
    long long* id;
    void* base;          // the one allocation holding all arrays (null: allocated one by one)
};
struct PArrF {           // MIXED mode: packed cell (i | j<<11 | k<<22), FP32 offset and velocity
    int* cell;
    float *fx, *fy, *fz, *vx, *vy, *vz;
    long long* id;
    void* base;          // as PArr::base
};

// per-species parameters and pointers handed to kernels by value
struct SpeciesDev {
    double k;                       // (q/m) dt
    double khalf;                   // k / 2
    PArr bins;                      // bin storage
    PArrF binsF;
    const long long* bstart;        // [nblocks] first slot of each bin
    const int* bcap;                // [nblocks] capacity
    int* bcount;                    // [nblocks] live particles
    int* bstay;                     // [nblocks] MIXED: the bin's stayers after the push (its arrivals follow)
    PArr mov_in, mov_out;           // mover lists (previous-step spill, this step)
    PArrF movF_in, movF_out;
    unsigned long long* mov_in_n;   // counters (device)
    unsigned long long* mov_out_n;
    long long mcap;
    unsigned long long* W;          // [nnodes] fixed-point charge
    unsigned long long* surf;       // [ncut] collected macro-particles
    unsigned long long* ctr;        // [NCTR] counters
    int reflect;                    // reflecting particle faces, bit f = face f
};

struct InjectDev {                  // one (species, face) injection stream
    int species, face, maxcnt;
    double vth, drift[3];
    double rate;                    // expected particles per step
    unsigned long long seed;
};

// one emitting interface tet of photoelectron emission (Sec. 5.2.2)
struct PhotoDev {
    double n[3], t1[3], t2[3];      // surface normal (into the plasma) and tangent basis
    double P[2][3][3];              // Gamma_h triangles, global cell units
    double area0, A;                // first triangle's area and the total (cell units)
    int ntri, acc;                  // triangles; cut-cell accumulator of the tet's cell
};
constexpr int PHOTO_RATE_BITS = 20;  // per-tet rates and carries in units of 2^-20 particles
constexpr int BAR64_WORDS = 160;     // PCG exchange words per context (Ctx::bar64): 10 lines of 16

struct Launch {                     // what every particle kernel needs
    Mesh mesh;
    Object obj;
    double dth;                     // dt / h
    int nbx, nby, nbz, nblocks;
    int bsh;                        // bin edge = 2^bsh cells (4 or 8)
    int nspecies;
    int track;
    const int* cell_acc;            // [ncells] surface accumulator of a hit cell
    const double4* E;               // node field
    const float4* Ef;               // node field, FP32 copy
    int* err;                       // device error word
    Mesh fmesh;                     // field (IFE) mesh: mesh refined refine times
    int refine;                     // 1: the meshes coincide
    double rf;                      // refine as a double (a power of two: exact scaling)
    SpeciesDev sp[MAX_SPECIES];
};

struct Species {
    double q, m, w, k;
    long long cap = 0;              // bin slots
    long long mcap = 0;             // mover list capacity
    PArr bins{}, mov[2]{};
    PArrF binsF{}, movF[2]{};
    long long* bstart = nullptr;
    int* bcap = nullptr;
    int* bcount = nullptr;
    int* bstay = nullptr;
    unsigned long long* mov_n = nullptr;   // [2]
    unsigned long long* W = nullptr;
    unsigned long long* surf = nullptr;
    unsigned long long* ctr = nullptr;
    int cur = 0;                    // which mover buffer is "in"
    bool inject = false;
    int face_mask = 0;
    int reflect = 0;                // reflecting particle faces, bit f = face f
    double density = 0, vth = 0, drift[3] = {0, 0, 0};
    unsigned long long seed = 0;
    double rate[6] = {0, 0, 0, 0, 0, 0};
    int maxcnt[6] = {0, 0, 0, 0, 0, 0};
    long long next_id = 0;
};

// the values a call's statistics need, gathered on the device into one block
// (one copy and one synchronisation per read)
struct StatPack {
    unsigned long long ctr[MAX_SPECIES * NCTR];   // the species' event counters
    long long count[MAX_SPECIES];                 // particles in bins + waiting list
    long long it_total, outer_total;              // PCG iteration counters
    double relres, surface_charge, surface_potential;
    int it, converged, err, pad;
};

struct Ctx {
    std::string err;
    cudaStream_t stream = nullptr;
    int device = 0;
    Mesh mesh{};                    // the field (IFE) mesh
    Mesh pmesh{};                   // the particle (PIC) mesh; mesh is it refined refine times
    int refine = 1;
    double origin[3] = {0, 0, 0};
    double dt = 0, dth = 0;
    int precision = PIFEPIC_FP64;
    double tol = 1e-6;
    int maxit = 150;
    double inner_red = 1e-4;      // MIXED: inner solves stop at max(margin tol |b|, red |r0|)
    double inner_margin = 0.5;
    int track = 0;
    int nbx = 0, nby = 0, nbz = 0, nblocks = 0;
    int bin_edge = BLK;           // particle bins of bin_edge^3 PIC cells (MIXED: 4 or 8; FP64: 4)

    Object obj{};
    bool have_object = false;
    pifepic_face_bc bc[6];
    bool external_E = false;

    // node arrays
    double* Lnode = nullptr;
    int* ntype = nullptr;          // >=0 patch row, -1 plus, -2 minus, -3 Dirichlet
    double* gdir = nullptr;        // Dirichlet values (0 on free nodes)
    double* lift = nullptr;        // (A g) restricted to free nodes
    double* invdiag = nullptr;
    double* phi = nullptr;
    double* u = nullptr;           // unknown (phi - g)
    double* phi_prev = nullptr;    // potential before the last solve (start extrapolation)
    double* b = nullptr;           // right-hand side
    double *r = nullptr, *p = nullptr, *q = nullptr;
    double* z = nullptr;           // inside a zeroed guard (zguard)
    float* zf = nullptr;           // inside a zeroed guard (zguard)
    double* z2 = nullptr;          // second guarded copies in the same allocations
    float* zf2 = nullptr;
    float *rf = nullptr, *pf = nullptr, *qf = nullptr, *uf = nullptr, *invdiagf = nullptr;
    double4* E = nullptr;          // node field (x, y, z, 0)
    float4* Ef = nullptr;          // FP32 copy for the MIXED push
    double4* Ep = nullptr;         // node field at the PIC nodes (E itself when refine == 1)
    float4* Efp = nullptr;         // its FP32 copy (Ef itself when refine == 1)
    unsigned long long* Wall = nullptr;     // [MAX_SPECIES][nnodes] fixed-point charge
    unsigned long long* surfall = nullptr;  // [MAX_SPECIES][ncut] collected particles
    unsigned long long* ctrall = nullptr;   // [MAX_SPECIES][NCTR]
    // cells
    unsigned char* imask = nullptr;
    int* ibase = nullptr;
    int* cell_acc = nullptr;
    // interface tets
    long long nit = 0;
    int* it_cell = nullptr;
    int* it_t = nullptr;
    double* it_data = nullptr;     // IT_STRIDE doubles per tet
    // node rows (launch_node_rows): a node that is not interior-regular has row
    // ne_row[n] >= 0 (else -1): its node field is sum over the 27 neighbours of
    // ne_coef[(3 nb + d) R + row] phi_nb plus sum over its interface tets of the
    // FP32 coefficients in ne_q times q_T; ne_qc holds each such tet's FP64
    // unit-jump load at the node (the right-hand side's flux-jump term)
    int* ne_row = nullptr;         // [nnodes]
    long long ne_nrows = 0;        // R
    float* ne_coef = nullptr;      // [81][R]
    int* ne_qoff = nullptr;        // [R + 1]: the row's interface tets, ne_q[ne_qoff[row] .. ne_qoff[row + 1])
    int4* ne_q = nullptr;          // {T, 3 FP32 coefficients as bits}
    double* ne_qc = nullptr;       // FP64 unit-jump load of tet T at the node
    int* it_acc = nullptr;
    double* qT = nullptr;
    // cut cells
    long long ncut = 0;
    int* cut_cell = nullptr;
    double* cut_area = nullptr;
    double* qcut = nullptr;
    // patch rows
    long long npatch = 0;
    long long* patch_node = nullptr;
    double* patch_coef = nullptr;  // [npatch][19]
    float* patch_coeff = nullptr;
    // reductions / PCG scalars
    double* red = nullptr;         // partial sums
    double* coop_partial = nullptr; // [8][2048] block partials of the persistent PCG
    double* scal = nullptr;        // PCG scalars
    unsigned int* red_ticket = nullptr;
    // PCG exchange words: [0] the arrival counter (a multiple of the grid between
    // launches); [16], [32], [48] the fixed-point reduction words (one 128-byte
    // line each)
    unsigned long long* bar64 = nullptr;
    long long zguard = 0;           // zeroed entries before z / zf (and after, plus 16)
    // layered object (pifepic_set_bedrock), copied into obj by set_object
    bool bed_on = false;
    double bed_z = 0.0, bed_eps = 1.0;
    bool bed_outside = false;       // set-up found a bedrock node outside the object
    // register-resident PCG launch plan (pcg_coop.cu): nodes per thread (0: the
    // global-memory kernel; -1: not planned yet), blocks, nodes per block, z window
    int pcg_npt = -1;
    bool pcg_rows = false;            // operator rows staged in shared memory
    int precond = PIFEPIC_PRECOND_AUTO;   // MIXED single-context solves: Jacobi or multigrid
    int mg_nlev = 0;                  // multigrid coarse levels (0: none)
    bool mg_single = false;           // the context's own MIXED solve uses the multigrid cycle
    MgLevel mg[MG_MAX_LEVELS];        // mg[1..mg_nlev]
    float* mg_r0 = nullptr;           // fine residual after pre-smoothing
    float* mg_cinv = nullptr;         // dense inverse of the coarsest operator
    bool mg_wanted = false;           // a batch solves this context with multigrid: keep a hierarchy
    bool mg_escalated = false;        // AUTO: a Jacobi solve ended at the cap unconverged; multigrid since
    long long solves_done = 0;        // field solves of pifepic_solve and pifepic_step so far
    cudaStream_t side = nullptr;      // movers and injection beside the push (pifepic_step)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    unsigned short* rowkind = nullptr;  // global-memory PCG (larger meshes): row kinds, [N]
    double* pcg_x = nullptr;            // and its FP64 correction vector, [N]
    int pcg_G = 1;
    long long pcg_M = 0;
    size_t pcg_smem = 0;
    int* err_word = nullptr;
    StatPack* stat_dev = nullptr;   // gather_stats: device block and its pinned host copy
    StatPack* stat_host = nullptr;
    // graphs
    cudaGraphExec_t pcg_exec = nullptr;
    cudaGraph_t pcg_graph = nullptr;
    // photoelectron emission: emitting tets in interface-tet order
    int ph_species = -1;
    long long ph_ne = 0;
    PhotoDev* ph_tets = nullptr;
    long long* ph_Q = nullptr;        // fixed-point rate per step
    long long* ph_carry = nullptr;
    int* ph_cnt = nullptr;            // this step's count per tet
    long long* ph_base = nullptr;     // exclusive scan of ph_cnt
    long long* ph_tiles = nullptr;    // scan tile sums
    long long* ph_total = nullptr;    // this step's emissions
    double ph_vth = 0.0;
    double ph_rate = 0.0;             // expected emissions per step (sizes the mover list)
    unsigned long long ph_seed = 0;
    // particles
    std::vector<Species> sp;
    std::vector<InjectDev> inj;
    InjectDev* inj_dev = nullptr;
    int* inj_count = nullptr;       // [MAX_SPECIES*6]
    long long* inj_base = nullptr;  // id base per (species, face)
    double* inj_carry = nullptr;    // [MAX_SPECIES*6]
    long long* next_id = nullptr;   // [MAX_SPECIES]
    long long step_no = 0;
    long long launches = 0;         // kernels launched by host code (graphs counted separately)
    // TMA descriptors of the node field
    CUtensorMap tmapE;
    CUtensorMap tmapEf;
    bool tmap_ok = false;
    // timers
    cudaEvent_t ev[16];
    std::vector<cudaEvent_t> step_ev;   // phase events of up to STEP_RING steps in flight (created on first step)
    unsigned long long* spill_host = nullptr;   // pinned: a photoemitting species' waiting-list length per step
    bool ev_ok = false;
    pifepic_stats stats{};
    int last_iters = 0;
    double last_relres = 0;
    int last_conv = 1;
};

// Stream-ordered copies and fills on the context's stream.  The caller's
// stream may be non-blocking with respect to the legacy default stream (as
// PyTorch streams are), so the library never uses the synchronous
// cudaMemcpy / cudaMemset, which run on the legacy stream.
inline cudaError_t scopy(cudaStream_t st, void* dst, const void* src, size_t n, cudaMemcpyKind k) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, n, k, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}
inline cudaError_t szero(cudaStream_t st, void* p, size_t n) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p, 0, n, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

// interface-tet record layout (doubles)
enum {
    IT_VOLP = 0, IT_VOLM = 1, IT_AREA = 2,
    IT_K = 3,            // 16
    IT_C = 19,           // 4  unit-jump load
    IT_GP = 23,          // 15 (5 x 3)
    IT_GM = 38,          // 15
    IT_S = 53,           // 4  int_Gamma psi_i
    IT_SJ = 57,          // 1  int_Gamma phi_J (unit q)
    IT_KIND = 58,        // 1  0: the object's surface; 1: the bedrock plane (no charge, no area)
    IT_STRIDE = 59
};

// ---- launchers ---------------------------------------------------------------
cudaError_t set_tet_tables(const TetTables& t);
cudaError_t launch_setup(Ctx& c);                      // S0 (setup.cu)
void log_error(const char* message);                   // capi.cu: to the log callback, if set
cudaError_t launch_node_rows(Ctx& c);                  // setup.cu: ne_row, ne_coef, ne_qoff, ne_q, ne_qc
cudaError_t launch_photo_setup(Ctx& c, const double* sun, double density, double vth, double w);  // setup.cu
cudaError_t launch_photo(Ctx& c);                      // particles.cu: one step of emission (FP64)
cudaError_t launch_photo_mixed(Ctx& c);                // particles_mixed.cu
cudaError_t launch_node_E64(Ctx& c);                   // field.cu: FP64 E from phi (E only)
// field.cu: the node field at the PIC nodes from the IFE nodes (refine > 1;
// both: the FP64 field too, else the FP32 copy only)
cudaError_t launch_E_to_pic(const Ctx& c, cudaStream_t st, bool both);
cudaError_t launch_field_lift(Ctx& c);
cudaError_t build_pcg_graph(Ctx& c);                   // field.cu
void plan_pcg(Ctx& c);                                 // pcg_coop.cu
cudaError_t launch_pcg(Ctx& c);
// diag: also the surface charge and mean surface potential (a few kernels)
cudaError_t gather_stats(Ctx& c, StatPack* out, bool diag);
cudaError_t launch_qtets(Ctx& c);

Launch make_launch(Ctx& c);
cudaError_t launch_load_maxwellian(Ctx& c, int s, int ppc, double vth, const double drift[3],
                                   unsigned long long seed, PArr flat, unsigned long long* nflat, long long cap);
cudaError_t launch_build_bins(Ctx& c, int s, PArr flat, long long n, bool fresh_caps);
cudaError_t launch_flatten(Ctx& c, int s, PArr flat, unsigned long long* nflat);
cudaError_t launch_deposit_all(Ctx& c);
cudaError_t launch_half_kick(Ctx& c);
cudaError_t launch_push(Ctx& c);        // launch_push_prep + launch_push_bins
cudaError_t launch_push_prep(Ctx& c);
cudaError_t launch_push_bins(Ctx& c);
cudaError_t launch_movers(Ctx& c);
cudaError_t launch_inject(Ctx& c);
cudaError_t launch_rebin(Ctx& c);

// MIXED mode
cudaError_t launch_flatten_mixed_to_f64(Ctx& c, int s, PArr flat, unsigned long long* nflat);
cudaError_t launch_build_bins_mixed(Ctx& c, int s, PArr flat, long long n, bool fresh_caps);
cudaError_t launch_push_mixed(Ctx& c);  // launch_push_prep_mixed + launch_push_bins_mixed
cudaError_t launch_push_prep_mixed(Ctx& c);
cudaError_t launch_push_bins_mixed(Ctx& c);
cudaError_t launch_movers_mixed(Ctx& c);
cudaError_t launch_inject_mixed(Ctx& c);
cudaError_t launch_rebin_mixed(Ctx& c);
cudaError_t launch_deposit_all_mixed(Ctx& c);
cudaError_t launch_half_kick_mixed(Ctx& c);

}  // namespace pf

struct pifepic_ctx {
    pf::Ctx c;
};
