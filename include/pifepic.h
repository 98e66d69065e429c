/*
 * pifepic.h -- C ABI of libpifepic, a single-GPU (sm_103a) implementation of
 * the hot path of the non-homogeneous IFE-PIC method of arXiv:2011.10214
 * (PIFE-PIC): the per-step particle cycle (gather, push, object collection
 * with surface charging, scatter) and the linear-IFE PCG field solve it drives.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a pifepic_status; 0 is success.  The library never
 *    aborts, throws or prints.  After a non-zero status,
 *    pifepic_last_error(ctx) returns a context-owned, NUL-terminated message
 *    that stays valid until the next call on the same context; the same
 *    message also goes to the log callback, if one is set
 *    (pifepic_set_log_callback).
 *  - Units are the plasma units the paper's experiments are stated in
 *    (Sec. 3.1, Sec. 5.1): lengths in Debye lengths, time in 1/omega_pe,
 *    potential in kT_e/e, density in the reference density, eps_0 = 1.
 *  - Node arrays are indexed n = i + (nx+1) * (j + (ny+1) * k); cell arrays
 *    c = i + nx * (j + ny * k).  A node vector (E) is interleaved xyz.
 *  - Pointers passed in are borrowed for the duration of the call only.
 *    mem_kind says where they live: PIFEPIC_HOST (pageable or pinned host
 *    memory) or PIFEPIC_DEVICE (device memory of the context's GPU, e.g. a
 *    torch CUDA tensor's data_ptr()).  The library owns all of its device
 *    state and frees it in pifepic_destroy.
 *  - Work is enqueued on the CUDA stream given to pifepic_create (NULL = the
 *    legacy default stream).  Calls that return data or statistics
 *    synchronise that stream before returning.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef PIFEPIC_H
#define PIFEPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIFEPIC_OK = 0,
    PIFEPIC_EINVAL = 1,     /* bad argument or descriptor                        */
    PIFEPIC_ENOMEM = 2,     /* device allocation failed / capacity exhausted     */
    PIFEPIC_ESTATE = 3,     /* call out of order (e.g. step before set_object)   */
    PIFEPIC_ECUDA = 4,      /* a CUDA runtime or driver call failed              */
    PIFEPIC_ETIMEOUT = 5,   /* a bounded device-side wait gave up                */
    PIFEPIC_ENOTCONV = 6    /* reserved: the PCG cap is recorded in the stats, not
                               returned, because the paper caps iterations        */
} pifepic_status;

enum { PIFEPIC_HOST = 0, PIFEPIC_DEVICE = 1 };

/* Arithmetic of the particle cycle and the PCG (BASIS: the paper states no
 * precision).  FP64: everything in double.  MIXED: push in FP32 with an int32
 * packed cell index plus FP32 in-cell offset, PCG in FP32 inside an FP64
 * iterative refinement whose residuals and dot products are FP64. */
enum { PIFEPIC_FP64 = 0, PIFEPIC_MIXED = 1 };

/* Uniform Cartesian PIC mesh of nx*ny*nz cubic cells of edge h, each cut into
 * 5 tetrahedra; the IFE mesh equals the PIC mesh (Sec. 3.1.1). */
typedef struct {
    int nx, ny, nz;
    double h;
    double origin[3];
    /* Hybrid grid (Sec. 2.2: PIC and IFE meshes may differ in resolution):
     * the IFE mesh is this PIC mesh with every cell split r x r x r, r = 1
     * (0 reads as 1), 2, 4 or 8.  Particles move, gather and are binned on the
     * PIC mesh; they deposit on the IFE mesh (trilinear weights of the IFE
     * cell), the field is solved there, and the PIC nodes (IFE nodes) read the
     * node field.  Node and cell arrays of the API (potential, node field,
     * charges, cut cells, external field) are on the IFE mesh; particle
     * positions and the PLANE object's parameters are in PIC cell units. */
    int ife_refine;
} pifepic_mesh_desc;

/* Time step and field-solver controls.  pcg_tol is the relative-residual
 * tolerance ||r|| <= tol ||b|| and pcg_max_iter the iteration cap (the paper
 * uses 1e-6 with caps of 60 and 150, Sec. 3.2, Sec. 4, Sec. 5.2.2).  In MIXED
 * mode pcg_max_iter caps the FP32 inner iterations summed over refinements.
 * track_ids = 1 carries an int64 id with every particle (parity tests). */
typedef struct {
    double dt;
    int precision;
    double pcg_tol;
    int pcg_max_iter;
    int track_ids;
} pifepic_solver_desc;

/* Immersed object (Sec. 2.1: the interface Gamma splits the box into Omega^-
 * (object, eps_in) and Omega^+ (plasma, eps_out)), as an analytic level set
 * L >= 0 in the plasma:
 *   SPHERE:     params = {cx, cy, cz, R}                    (Sec. 3.1.1)
 *   CAP_CRATER: params = {z_ground, xc, yc, rim_radius, depth}; planar ground
 *               with a spherical-cap crater             (reading of Sec. 5.2.1)
 *   PLANE:      params = {n_x, n_y, n_z, d0} in cell units: L = n.xi - d0
 *   RIM_CRATER: params = {z_ground, xc, yc, r_inner, r_top, r_outer, height,
 *               depth}: planar ground with a raised-rim crater (Sec. 5.2.1
 *               names the crater by its inner-rim, top-rim and outer-rim radii
 *               and its top height; the profile is this library's reading): a
 *               flat floor at depth below the ground inside r_inner, an inner
 *               wall rising to the rim top (height above the ground) at r_top
 *               and an outer flank falling to the ground at r_outer, both
 *               ramps the cubic smoothstep t^2 (3 - 2t) of the radius.  EINVAL
 *               unless 0 <= r_inner < r_top < r_outer, height, depth >= 0.
 *   NONE:       no object. */
enum {
    PIFEPIC_OBJ_NONE = 0,
    PIFEPIC_OBJ_SPHERE = 1,
    PIFEPIC_OBJ_CAP_CRATER = 2,
    PIFEPIC_OBJ_PLANE = 3,
    PIFEPIC_OBJ_RIM_CRATER = 4
};
typedef struct {
    int kind;
    double params[8];
    double eps_in, eps_out;
} pifepic_object_desc;

/* Field boundary of one face (Eqs. 2.2-2.3): Dirichlet phi = value, or zero
 * Neumann.  Faces are ordered x-, x+, y-, y+, z-, z+. */
enum { PIFEPIC_BC_DIRICHLET = 0, PIFEPIC_BC_NEUMANN = 1 };
typedef struct {
    int kind;
    double value;
} pifepic_face_bc;

/* Statistics of the last call (one entry per species where indexed). */
#define PIFEPIC_MAX_SPECIES 8
typedef struct {
    int64_t steps;                             /* PIC steps taken so far        */
    int64_t pushed[PIFEPIC_MAX_SPECIES];       /* particle-steps in this call   */
    int64_t count[PIFEPIC_MAX_SPECIES];        /* particles alive now           */
    int64_t injected[PIFEPIC_MAX_SPECIES];     /* entered through open faces    */
    int64_t absorbed[PIFEPIC_MAX_SPECIES];     /* left through absorbing faces  */
    int64_t collected[PIFEPIC_MAX_SPECIES];    /* hit the object                */
    int64_t lost_charge[PIFEPIC_MAX_SPECIES];  /* hits with no cut cell nearby  */
    int64_t inj_rejected[PIFEPIC_MAX_SPECIES]; /* injection starts in the object*/
    int64_t spilled[PIFEPIC_MAX_SPECIES];      /* waiting in the overflow list  */
    int64_t dropped[PIFEPIC_MAX_SPECIES];      /* lost: all buffers full (error)*/
    int64_t pcg_iters_total;                   /* PCG iterations in this call   */
    int64_t kernel_launches;                   /* kernels launched in this call */
    int pcg_iters;                             /* last solve                    */
    int pcg_converged;
    double pcg_relres;
    double surface_charge;                     /* total charge on the object    */
    double surface_potential;                  /* area-mean phi on Gamma_h      */
    double phase_ms[8];                        /* GPU time per phase, this call:
                                                  push, movers, inject, rebin,
                                                  rhs, pcg, node_E, other.  In
                                                  pifepic_step the waiting
                                                  list's push and the injection
                                                  run beside the bins' push: the
                                                  push phase covers them, the
                                                  movers phase holds what
                                                  outlasts it, inject is 0      */
    int64_t pcg_outer_total;                   /* MIXED refinement steps in this
                                                  call (FP64 residuals - 1 per
                                                  solve)                         */
} pifepic_stats;

typedef struct pifepic_ctx pifepic_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (may
 * be NULL).  Fails with EINVAL on a degenerate mesh (n < 1 or h <= 0), with
 * ENOMEM if the mesh arrays do not fit. */
pifepic_status pifepic_create(const pifepic_mesh_desc* mesh, const pifepic_solver_desc* solver,
                              void* stream, pifepic_ctx** out);
void pifepic_destroy(pifepic_ctx* ctx);
const char* pifepic_last_error(const pifepic_ctx* ctx);

/* Optional log sink.  Every error message that pifepic_last_error or
 * pifepic_batch_last_error returns is also passed to fn, with user, on the
 * calling thread, when the error is recorded (the message is valid during the
 * call only).  NULL (the default) turns it off.  Process-wide: set it while no
 * other thread calls the library. */
typedef void (*pifepic_log_fn)(const char* message, void* user);
void pifepic_set_log_callback(pifepic_log_fn fn, void* user);

/* Object and field boundary set-up (Sec. 2.1, Sec. 3.1.2, Sec. 5.2.2): node
 * level set, tet classification, per-interface-tet linear IFE basis (a 4x4
 * FP64 solve each), stiffness patch rows, cut cells, and the node rows of the
 * node field (for every node on a face or next to an interface tet: its
 * 27 x 3 coefficients and interface-tet terms, about 330 bytes a node).  Must
 * precede particle calls.  set_field_bc may be called before or after
 * set_object. */
pifepic_status pifepic_set_object(pifepic_ctx* ctx, const pifepic_object_desc* obj);

/* A second dielectric layer of the object (Sec. 5.2.1: the lunar regolith lies
 * on bedrock of higher permittivity): below the plane z = z_bed (physical
 * height) the object has permittivity eps_bed.  Tets inside the object that
 * the plane cuts become interface tets of the plane (homogeneous flux jump, no
 * surface charge, no photoemission); a tet cut by the object's surface keeps
 * the surface alone even where the plane also crosses it.  The bedrock must
 * lie inside the object: set_object fails with EINVAL if a mesh node below
 * z_bed is outside it.  Call before pifepic_set_object.  Errors: EINVAL
 * (eps_bed <= 0, z_bed not finite), ESTATE (after set_object). */
pifepic_status pifepic_set_bedrock(pifepic_ctx* ctx, double z_bed, double eps_bed);

/* MIXED-mode refinement controls (FP64 iterative refinement around FP32
 * inner PCG solves; a reading of the PCG of Sec. 2.5 for FP32 arithmetic).
 * Each inner solve stops once its FP32 residual norm is at most
 * max(margin * pcg_tol * ||b||, reduction * ||r0||), r0 the FP64 residual it
 * started from; the refinement ends when the FP64 residual meets pcg_tol.
 * Defaults reduction = 1e-4, margin = 0.5.  A batch's Jacobi clusters use a
 * reduction of at most 1e-6 (their two-exchange loop then meets pcg_tol after
 * one refinement step).  Takes effect at the next solve; call before the
 * context joins a batch (a batch's captured step does not see a later
 * change).  No effect in FP64 mode.  Errors: EINVAL unless 0 < reduction < 1
 * and 0 < margin <= 1. */
pifepic_status pifepic_set_refinement(pifepic_ctx* ctx, double reduction, double margin);

/* Preconditioner of the MIXED inner PCG of a single context (Sec. 2.5 names
 * the PCG but no preconditioner).  JACOBI: the diagonal, as the FP64 path and
 * the oracle.  MULTIGRID: one geometric V(1,1) cycle per iteration -- coarse
 * levels at the even nodes of each axis (plus the last node of an odd axis),
 * trilinear prolongation with zero Dirichlet correction, restriction its
 * transpose, Galerkin coarse operators (27-point, built at set-up), damped
 * Jacobi smoothing (weight 0.6), the coarsest level (at most 256 nodes)
 * solved exactly by its dense inverse.  AUTO (the default): MULTIGRID for
 * meshes too large for the register-resident solver (more than 8 nodes per
 * thread of a full grid, about 620,000 nodes), where the Jacobi iteration
 * count outgrows the cap, else JACOBI -- until a warm-started solve of
 * pifepic_solve or pifepic_step (any but the context's first, which starts
 * from zero) ends at the iteration cap without converging: from then on
 * the context solves with MULTIGRID (meshes of at most 256 nodes have no
 * hierarchy and keep Jacobi).  Either solves the same system to the same
 * stopping test.  Takes effect at once (the solve is re-planned); no
 * effect in FP64 mode or on batched solves.  Errors: EINVAL (unknown kind),
 * ENOMEM. */
enum { PIFEPIC_PRECOND_AUTO = 0, PIFEPIC_PRECOND_JACOBI = 1, PIFEPIC_PRECOND_MULTIGRID = 2 };
pifepic_status pifepic_set_preconditioner(pifepic_ctx* ctx, int kind);
/* The persistent solver the context's next solve runs (after AUTO's choices):
 * 1 = Jacobi PCG with the vectors in registers (meshes of at most 8 nodes per
 * thread of a full grid), 2 = Jacobi PCG with the vectors in global memory,
 * 3 = multigrid-preconditioned PCG (MIXED); 0 for a NULL context. */
enum { PIFEPIC_SOLVER_REGISTERS = 1, PIFEPIC_SOLVER_GLOBAL = 2, PIFEPIC_SOLVER_MULTIGRID = 3 };
int pifepic_get_solver(const pifepic_ctx* ctx);
pifepic_status pifepic_set_field_bc(pifepic_ctx* ctx, const pifepic_face_bc bc[6]);

/* Particle bins (the cell blocks of Sec. 2.3's particle storage): particles
 * are stored sorted by bins of edge^3 PIC cells, and one CTA pushes one bin
 * and species through the bin's (edge+1)^3 node-field tile (TMA) and deposit
 * tile in shared memory.  edge is 4 (the default) or 8; MIXED contexts only
 * for 8.  Larger bins mean fewer bin leavers per step and fewer CTAs, and more
 * shared memory per CTA; a bin holds at most 32767 particles per species (the
 * rest waits in the mover list), so 8 suits up to about 48 particles per cell
 * and species.  A particle's push is the same arithmetic for either edge; a
 * bin's stayers deposit with weights rounded to 2^-19 of a particle and its
 * leavers with 2^-32 weights, so node charges (whose totals stay exact) differ
 * between edges within that rounding.  Call before the first
 * pifepic_add_species.  Errors: EINVAL (edge not 4 or 8, or 8 in FP64),
 * ESTATE (species exist).  pifepic_get_bin_edge returns the edge (0 for NULL). */
pifepic_status pifepic_set_bin_edge(pifepic_ctx* ctx, int edge);
int pifepic_get_bin_edge(const pifepic_ctx* ctx);

/* Species with charge q, mass m (q/m sets the push) and macro-particle
 * weight w (charge per macro-particle = q*w; w = density*h^3/ppc).  At most
 * PIFEPIC_MAX_SPECIES. */
pifepic_status pifepic_add_species(pifepic_ctx* ctx, double q, double m, double w, int* species_id);

/* Pre-load (Sec. 3.1.3): ppc particles per cell uniform in the cell,
 * velocities Maxwellian (thermal speed vth) plus drift, drawn from
 * Philox4x64-10 keyed by seed; particles inside the object are dropped. */
pifepic_status pifepic_load_maxwellian(pifepic_ctx* ctx, int species, int ppc, double vth,
                                       const double drift[3], uint64_t seed);

/* Append n explicit particles: positions in cell units xi = (x-origin)/h,
 * physical velocities, optional int64 ids (NULL: consecutive ids).  Every
 * position must lie inside the box [0, n) per axis and every value be finite
 * (checked on the device after the copy): otherwise EINVAL and nothing is
 * appended. */
pifepic_status pifepic_load_particles(pifepic_ctx* ctx, int species, size_t n, const double* x,
                                      const double* y, const double* z, const double* vx,
                                      const double* vy, const double* vz, const int64_t* ids,
                                      int mem_kind);

/* Injection at open faces every step (Sec. 3.1.3, Sec. 5.2.2): for each face
 * f with bit f of face_mask set, floor(rate + carry) particles per step with
 * rate = one-way drifting-Maxwellian flux * face area * dt / w.  Errors:
 * EINVAL (bad species, vth <= 0, density < 0, mask bits beyond the six faces
 * or on a face marked REFLECT by set_particle_bc). */
pifepic_status pifepic_set_injection(pifepic_ctx* ctx, int species, int face_mask, double density,
                                     double vth, const double drift[3], uint64_t seed);
/* Particle boundary kinds of a face (pifepic_set_particle_bc). */
enum { PIFEPIC_PBC_ABSORB = 0, PIFEPIC_PBC_INJECT = 1, PIFEPIC_PBC_REFLECT = 2 };

/* Particle boundary of the six faces for one species (Sec. 3.1.3: open faces
 * absorb the particles that leave and inject new ones; Sec. 5.2.2: particles
 * are reflected at the symmetry plane of a half-domain run).  face_kind: 6
 * ints, host, faces x-, x+, y-, y+, z-, z+ (the order of set_field_bc).
 * ABSORB (the default) and INJECT remove a particle whose new position lies
 * beyond the face; INJECT marks a face whose injection set_injection turns on.
 * REFLECT mirrors the position back into the box after every move (pushed,
 * injected and photoemitted particles alike), xi -> -xi at a minus face and
 * xi -> 2n - xi at a plus face, before the boundary and object tests, and
 * reverses the normal velocity; a mirror that lands exactly on the plus face
 * takes the largest coordinate below n.  The field boundary of the face is
 * separate (a symmetry plane is normally Neumann, set_field_bc).  Call before
 * stepping, and before the context joins a batch (a batch's captured step does
 * not see a later change).  Errors: EINVAL (bad species or kind, a REFLECT face
 * in the species' injection mask). */
pifepic_status pifepic_set_particle_bc(pifepic_ctx* ctx, int species, const int face_kind[6]);

/* The six per-face rates (expected particles per step) of a species' injection. */
pifepic_status pifepic_get_injection_rate(pifepic_ctx* ctx, int species, double rate[6]);

/* Photoelectron emission (Sec. 5.2.2: photoelectrons are generated at the
 * sunlit regions by the local sunlight index, the inner product of the sun
 * vector and the surface normal).  Species s is emitted every step from the
 * Gamma_h piece of every interface tet T with n_T . s > 0 whose centroid sees
 * the sun (a ray towards sun_dir, sampled every quarter cell, never enters the
 * object): rate J S_T A_T dt / w per step with J = density vth / sqrt(2 pi),
 * held in fixed point (2^-20 particles) with an exact per-tet carry; points
 * uniform on Gamma_h, flux-weighted half-Maxwellian normal speed, Gaussian
 * tangential speeds, a partial first step; each emitted particle takes one
 * count off its cut cell's surface accumulator (the surface charges up).
 * sun_dir: 3 doubles, host, towards the sun, any length > 0.  Call after
 * set_object and add_species; again to change it.  Errors: EINVAL (bad species,
 * density < 0, vth <= 0, zero sun_dir), ESTATE (no object). */
pifepic_status pifepic_set_photoemission(pifepic_ctx* ctx, int species, const double sun_dir[3], double density,
                                         double vth, uint64_t seed);
/* The emission set-up: rate_fixed = sum over emitting tets of the fixed-point
 * rate (units of 2^-20 particles per step), emitting_tets = their number.
 * Either pointer may be NULL. */
pifepic_status pifepic_get_photoemission(pifepic_ctx* ctx, int64_t* rate_fixed, int64_t* emitting_tets);

/* Freeze the node field to the given (nnodes x 3) array: steps then skip the
 * field solve (particle-only parity runs).  E == NULL unfreezes.  EINVAL if a
 * value is not finite (the field is then left as it was). */
pifepic_status pifepic_set_external_E(pifepic_ctx* ctx, const double* E, int mem_kind);

/* Scatter all particles, solve the IFE system, compute the node field (the
 * initial field solve, Sec. 3.2.1). */
pifepic_status pifepic_solve(pifepic_ctx* ctx, pifepic_stats* stats);

/* Leapfrog start: v <- v - (q/m)(dt/2) E(x) with the current node field. */
pifepic_status pifepic_leapfrog_init(pifepic_ctx* ctx);

/* nsteps PIC steps (Sec. 2.1 Fig. 1): push + collection + injection, rebin,
 * scatter, IFE solve, node field.  A PCG that reaches its cap is recorded in
 * stats (pcg_converged = 0), not returned as an error.  stats may be NULL. */
pifepic_status pifepic_step(pifepic_ctx* ctx, int nsteps, pifepic_stats* stats);

/* Read-back.  Arrays are caller-owned with the stated sizes. */
pifepic_status pifepic_get_sizes(pifepic_ctx* ctx, int64_t* nnodes, int64_t* ncells,
                                 int64_t* n_interface_tets, int64_t* n_cut_cells);
pifepic_status pifepic_get_potential(pifepic_ctx* ctx, double* phi, int mem_kind);        /* nnodes   */
pifepic_status pifepic_get_node_E(pifepic_ctx* ctx, double* E, int mem_kind);             /* nnodes*3 */
/* The FP32 node field the MIXED push gathers from (nnodes x 3 floats,
 * interleaved xyz, IFE-mesh nodes): in MIXED mode the field the last solve's
 * FP32 node-field kernel wrote (the node field of Sec. 2.1's gather, evaluated
 * in FP32 from the FP64 potential), in FP64 mode the FP32 rounding of the FP64
 * field.  pifepic_get_node_E returns the FP64 field instead, which MIXED mode
 * computes from phi on demand. */
pifepic_status pifepic_get_node_E_f32(pifepic_ctx* ctx, float* E, int mem_kind);          /* nnodes*3 */
pifepic_status pifepic_get_node_charge(pifepic_ctx* ctx, int species, int64_t* W, int mem_kind); /* nnodes, 2^32 per particle */
pifepic_status pifepic_get_surface_charge(pifepic_ctx* ctx, int species, int64_t* counts,
                                          int mem_kind);                                   /* n_cut_cells */
pifepic_status pifepic_get_cut_cells(pifepic_ctx* ctx, int32_t* cells, double* area);      /* n_cut_cells */
pifepic_status pifepic_get_cell_target(pifepic_ctx* ctx, int32_t* target);                  /* ncells: cut index or -1 */
/* Interface tets, ordered by (cell, local tet): cell, local tet (0..4),
 * sub-volumes, Gamma_h area, element stiffness (16, row-major) and the
 * unit-jump load vector (4). Any pointer may be NULL. */
pifepic_status pifepic_get_interface(pifepic_ctx* ctx, int32_t* cell, int32_t* tet, double* vol_plus,
                                     double* vol_minus, double* area, double* K, double* c);
pifepic_status pifepic_get_particle_count(pifepic_ctx* ctx, int species, int64_t* n);
/* Copies up to cap particles (any order); *n receives the number copied.
 * ids may be NULL (it must be NULL when track_ids is 0). */
pifepic_status pifepic_get_particles(pifepic_ctx* ctx, int species, int64_t cap, double* x, double* y,
                                     double* z, double* vx, double* vy, double* vz, int64_t* ids,
                                     int64_t* n, int mem_kind);
pifepic_status pifepic_get_stats(pifepic_ctx* ctx, pifepic_stats* stats);

/* Field solve on its own (Sec. 2.1 Eqs. 2.1-2.5, PCG level of Sec. 2.5): node
 * load F (nnodes, FP64) and flux jump q per interface tet (n_interface_tets,
 * in pifepic_get_interface order) -> phi and the node field.  Used by the
 * solver parity tests; F and q may be host or device arrays.  EINVAL if a
 * value of F or q is not finite. */
pifepic_status pifepic_solve_field(pifepic_ctx* ctx, const double* F, const double* q, int mem_kind,
                                   int* iters, double* relres);

/* Batched steps over many independent contexts (serving many charging
 * problems at once; the paper runs one problem per job, Sec. 3 and Sec. 5).
 * One CUDA graph launch per step advances every member: each member is its own
 * chain of particle phases, right-hand side, field solve and node field, and
 * the chains overlap on the device.  A member's field solve runs on one
 * thread-block cluster (1 to 16 CTAs of at most cta_nodes nodes each); a member
 * too large for a cluster uses the single-member persistent solver.  Members
 * must share one precision; their own streams are synchronised before the
 * batch stream (given at creation) takes over.  A member's results do not
 * depend on the other members.  The graph is rebuilt on the next step after
 * add / remove / set_cta_nodes.  stats (if not NULL) receives one entry per
 * member, in member order.  The batch borrows the contexts: destroy the batch
 * first. */
typedef struct pifepic_batch pifepic_batch;
pifepic_status pifepic_batch_create(pifepic_ctx** ctxs, int n, void* stream, pifepic_batch** out);
pifepic_status pifepic_batch_add(pifepic_batch* batch, pifepic_ctx* ctx);
pifepic_status pifepic_batch_remove(pifepic_batch* batch, pifepic_ctx* ctx);
/* Preferred nodes per CTA of the clustered solves (a power of two from 2048
 * to 65536; 8192 is the default): a member gets the smallest cluster that
 * keeps each CTA at or under it (Jacobi clusters: also the smallest whose
 * working set fits in shared memory).  Fewer nodes per CTA is less work per
 * iteration and more synchronisation; the serving loop's tuner picks by timing
 * steps.  EINVAL for other values. */
pifepic_status pifepic_batch_set_cta_nodes(pifepic_batch* batch, int cta_nodes);
/* Preconditioner of the batch's MIXED field solves: MULTIGRID solves every
 * member that has a multigrid hierarchy (built for the member on the first
 * step that needs it; meshes of at most 256 nodes have none and keep Jacobi)
 * by the multigrid-preconditioned PCG on one thread-block cluster of
 * ceil(nodes / cta_nodes) CTAs (1 to 16); AUTO (the default) and JACOBI keep
 * the Jacobi PCG on clusters of the member's whole working set in shared
 * memory (fewer iterations with multigrid, but each costs about eleven Jacobi
 * iterations on a cluster, and the Jacobi clusters step the batch faster).
 * FP64 batches always use Jacobi.  The graph is rebuilt on the next step.
 * EINVAL for an unknown kind. */
pifepic_status pifepic_batch_set_preconditioner(pifepic_batch* batch, int kind);
pifepic_status pifepic_batch_step(pifepic_batch* batch, int nsteps, pifepic_stats* stats);
const char* pifepic_batch_last_error(const pifepic_batch* batch);
void pifepic_batch_destroy(pifepic_batch* batch);

/* Device memory of the library, process-wide (every context and batch in the
 * process): *bytes receives the bytes it holds now.  pifepic_set_memory_limit
 * caps that total (0 = no cap, the default): an allocation that would pass
 * the cap fails as if the device were out of memory, and the call that needed
 * it returns ENOMEM (a context whose creation fails this way is freed by
 * pifepic_destroy as usual).  A serving loop can hold the library to an HBM
 * budget with it, and tests reach the out-of-memory paths without exhausting
 * the GPU.  Errors: EINVAL (bytes NULL). */
pifepic_status pifepic_get_memory_use(size_t* bytes);
pifepic_status pifepic_set_memory_limit(size_t bytes);

/* Test hook for the bounded waits of the persistent PCG (the solve of a single
 * context, not of a batch): the first grid exchange of the context's next
 * solve waits for `extra` arrivals beyond its grid, which never come, so its
 * bounded wait (about a second) gives up.  That solve's call returns ETIMEOUT;
 * the library then clears the exchange counters, the error word and the hook,
 * and the context stays usable.  extra = 0 turns the hook off.  Nothing
 * faults: every wait of the solve is bounded.  Errors: EINVAL unless
 * 0 <= extra <= 1. */
pifepic_status pifepic_test_hold_exchange(pifepic_ctx* ctx, int extra);

/* Field solve that allocates nothing.  (The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory once they are
 * running -- a serving loop whose device memory comes from a pool it does not
 * own, where a cudaMalloc can fail or stall every stream of the process, or a
 * host application that forbids allocation after start-up.
 * pifepic_solve_field allocates a staging buffer and builds a CUDA graph on
 * every call; this variant does neither.)
 *
 * Same system and stopping rule as pifepic_solve_field, on the context's
 * operator, tolerance and iteration cap; the context's own potential, node
 * field and solver state are left untouched.  It always runs the plain FP64
 * Jacobi PCG, whatever the context's precision (a MIXED context's refined
 * solve reaches the same solution at the same tolerance).  F (nnodes), q
 * (n_interface_tets; NULL means no flux jump) and phi (nnodes, output) are
 * caller-owned DEVICE arrays of the context's GPU, which must be the current
 * device (EINVAL otherwise).  The PCG work vectors live in one fixed
 * __device__ array of the library, 5.3 MB, which every GPU that loads the
 * library holds until the process exits; meshes with more than
 * PIFEPIC_NOALLOC_MAX_NODES nodes are rejected with EINVAL.  The first call
 * on a device looks up that array's address (cudaGetSymbolAddress), so make
 * it before any stream capture.  Every call shares the array and it keeps the
 * previous call's contents (each call sets what it reads before reading it):
 * calls that overlap on the GPU (other streams, other contexts on the same
 * device) race.  Each call queues 3 * pcg_max_iter + 5 kernel launches on the
 * context's stream (those after convergence return at once; on small meshes
 * the launches, not the arithmetic, set the call's time) and synchronises that
 * stream to return iters and relres. */
#define PIFEPIC_NOALLOC_MAX_NODES 131072
pifepic_status pifepic_solve_field_noalloc(pifepic_ctx* ctx, const double* F, const double* q, double* phi,
                                           int* iters, double* relres);

#ifdef __cplusplus
}
#endif
#endif /* PIFEPIC_H */
