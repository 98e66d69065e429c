// IFE field solve on the GPU: right-hand side with the flux-jump term, Jacobi
// PCG with a matrix-free operator plus 19-slot patch rows, node field.
//
// Sec. 2.1 (Eqs. 2.1-2.5): weak form a(phi, v) = (rho, v) - int_Gamma q v; the
// non-homogeneous IFE solution is phi_h = u_h + phi_J (phi_J the element-wise
// jump function) with a_h(u_h, psi_i) = F_i - int_Gamma q psi_i - a_h(phi_J,
// psi_i), i.e. F_i + sum_T q_T c_{T,i} (c the unit-jump load of interface tet
// T).  Sec. 2.5: the matrix solve is a PCG iteration stopped on the relative
// residual (Sec. 3.2, Sec. 4, Sec. 5.2.2 give tolerance 1e-6 and caps 60/150).
// Preconditioner (unstated in the paper): Jacobi.
//
// The whole solve is one CUDA graph: q_T, RHS, initial residual, then a
// conditional WHILE node whose body is one PCG iteration (spmv + p.q, update +
// r.r + r.z, direction update).  The iteration count and convergence test live
// on the device; no host round trip.  Reductions are deterministic: per-block
// partials, summed in a fixed order by the last block to finish.
#include <math.h>
#include <stdio.h>
#include <atomic>

#include "internal.h"
#include "field_common.cuh"

namespace pf {

__constant__ TetTables cTf;
// Interior-regular nodes (all eight cubes present, none holding an interface
// tet): every tet around the node lies on one side, so the node field is one
// fixed 27-point stencil per node parity P, cFold[P][3 nb + d] with
// nb = (dx + 1) + 3 (dy + 1) + 9 (dz + 1): minus the sum over the node's tets of
// vol_t grad_t (h = 1) at neighbour nb, over the sum of vol_t; E = cFold phi / h.
__constant__ float cFold[2][81];

// ---- right-hand side ----------------------------------------------------------
struct RhsArgs {
    const unsigned long long* W;     // [MAX_SPECIES][nnodes]
    const unsigned long long* surf;  // [MAX_SPECIES][ncut]
    const double* coefs;             // [MAX_SPECIES] q_s w_s (device)
    const int* nspec;                // device
    long long ncut;
};

__global__ void k_qcut(RhsArgs a, const double* area, double* qcut) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= a.ncut) return;
    double Q = 0.0;
    int ns = *a.nspec;
    for (int s = 0; s < ns; ++s) Q = Q + a.coefs[s] * (double)(long long)a.surf[(long long)s * a.ncut + c];
    qcut[c] = -(Q / area[c]);
}

__global__ void k_qtets(long long nit, const int* it_acc, const double* qcut, double* qT) {
    long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (T >= nit) return;
    int a = it_acc[T];
    qT[T] = a >= 0 ? qcut[a] : 0.0;
}

// the flux-jump terms of a node's right-hand side (the node rows of the set-up)
struct FluxRows {
    const int* row;
    const int* qoff;
    const int4* q;
    const double* qc;
};

__global__ void k_rhs(FieldArgs f, RhsArgs a, FluxRows fr, const double* qT, const double* lift, double* b,
                      const double* Fext, long long* hist) {
    const Mesh& m = f.m;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // solves so far, this one included (capped at 3): the start-vector kernel
    // that follows extrapolates only once two earlier solves exist
    if (hist && n == 0 && *hist < 3) *hist += 1;
    if (n >= m.nnodes) return;
    int ty = f.ntype[n];
    if (ty == -3) { b[n] = 0.0; return; }
    double F = 0.0;
    if (Fext) {
        F = Fext[n];
    } else {
        int ns = *a.nspec;
        for (int s = 0; s < ns; ++s)
            F = F + (a.coefs[s] * 2.3283064365386963e-10) * (double)(long long)a.W[(long long)s * m.nnodes + n];
    }
    if (ty >= 0 && qT) {   // touches interface tets: flux-jump load (none when qT is NULL)
        const int r = fr.row[n];
        if (r >= 0) {
            const int e1 = fr.qoff[r + 1];
            for (int e = fr.qoff[r]; e < e1; ++e) F += qT[fr.q[e].x] * fr.qc[e];
        }
    }
    b[n] = F - lift[n];
}

// ---- PCG kernels ------------------------------------------------------------------
__global__ void k_matvec(FieldArgs f, const double* x, double* y) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= f.m.nnodes) return;
    int i, j, k;
    node_ijk(f.m, n, i, j, k);
    y[n] = apply_row<double>(f, n, i, j, k, x, f.coef);
}

// phi = u + g; a zero right-hand side has the lift alone as its solution
__global__ void k_phi_from_u(long long N, const double* u, const double* g, double* phi, const PcgState* S) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) phi[n] = S->bb == 0.0 ? g[n] : u[n] + g[n];
}
// PCG start vector: the last potential, or once two earlier solves exist its
// linear extrapolation 2 phi_{n-1} - phi_{n-2} (particles move the charge
// smoothly from step to step, so this start is closer); phi_prev <- phi.  The
// solve still stops on the same relative residual.
__global__ void k_u_from_phi(long long N, const int* ntype, const double* phi, double* phi_prev, const double* g,
                             double* u, const long long* hist) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double p = phi[n];
    const double start = (*hist >= 3) ? 2.0 * p - phi_prev[n] : p;
    u[n] = ntype[n] == -3 ? 0.0 : start - g[n];
    phi_prev[n] = p;
}

// ---- node field ---------------------------------------------------------------------
__global__ void k_node_E(FieldArgs f, const double* L, const unsigned char* imask, const int* ibase,
                         const double* it_data, const double* qT, const double* phi, double4* E, float4* Ef) {
    const Mesh& m = f.m;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    int i, j, k;
    node_ijk(m, n, i, j, k);
    double apl[3] = {0, 0, 0}, vpl = 0.0, aal[3] = {0, 0, 0}, val = 0.0;
    double ih = 1.0 / m.h, V3 = m.h * m.h * m.h;
    for (int c8 = 0; c8 < 8; ++c8) {
        int a, b, c; loff(c8, a, b, c);
        int ci = i - a, cj = j - b, ck = k - c;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
        long long cell = cell_id(m, ci, cj, ck);
        unsigned mk = imask[cell];
        int p = (ci + cj + ck) & 1;
        int T = ibase[cell];
        for (int t = 0; t < 5; ++t) {
            bool itet = (mk >> t) & 1;
            bool has = false;
            for (int v = 0; v < 4; ++v)
                if (cTf.vert[p][t][v] == c8) has = true;
            if (has) {
                double ph[4];
                long long nd0 = 0;
                for (int v = 0; v < 4; ++v) {
                    int av, bv, cv; loff(cTf.vert[p][t][v], av, bv, cv);
                    long long nd = node_id(m, ci + av, cj + bv, ck + cv);
                    if (v == 0) nd0 = nd;
                    ph[v] = phi[nd];
                }
                if (itet) {
                    const double* rec = it_data + (long long)T * IT_STRIDE;
                    double qt = qT[T];
                    double gp[3], gm[3];
                    for (int d = 0; d < 3; ++d) {
                        gp[d] = ph[0] * rec[IT_GP + d] + ph[1] * rec[IT_GP + 3 + d] + ph[2] * rec[IT_GP + 6 + d] +
                                ph[3] * rec[IT_GP + 9 + d] + qt * rec[IT_GP + 12 + d];
                        gm[d] = ph[0] * rec[IT_GM + d] + ph[1] * rec[IT_GM + 3 + d] + ph[2] * rec[IT_GM + 6 + d] +
                                ph[3] * rec[IT_GM + 9 + d] + qt * rec[IT_GM + 12 + d];
                    }
                    double vp = rec[IT_VOLP], vm = rec[IT_VOLM];
                    // the + piece is plasma on the object's surface only (not on the bedrock plane)
                    if (vp > 0.0 && rec[IT_KIND] == 0.0) {
                        for (int d = 0; d < 3; ++d) apl[d] += vp * gp[d];
                        vpl += vp;
                    }
                    for (int d = 0; d < 3; ++d) aal[d] += vp * gp[d] + vm * gm[d];
                    val += vp + vm;
                } else {
                    double g[3];
                    for (int d = 0; d < 3; ++d)
                        g[d] = (ph[0] * cTf.grad[p][t][0][d] + ph[1] * cTf.grad[p][t][1][d] +
                                ph[2] * cTf.grad[p][t][2][d] + ph[3] * cTf.grad[p][t][3][d]) * ih;
                    double V = cTf.vol[t] * V3;
                    if (L[nd0] >= 0.0) {
                        for (int d = 0; d < 3; ++d) apl[d] += V * g[d];
                        vpl += V;
                    }
                    for (int d = 0; d < 3; ++d) aal[d] += V * g[d];
                    val += V;
                }
            }
            if (itet) ++T;
        }
    }
    double4 e;
    if (vpl > 0.0) { e.x = -apl[0] / vpl; e.y = -apl[1] / vpl; e.z = -apl[2] / vpl; }
    else { e.x = -aal[0] / val; e.y = -aal[1] / val; e.z = -aal[2] / val; }
    e.w = 0.0;
    E[n] = e;
    if (Ef) Ef[n] = make_float4((float)e.x, (float)e.y, (float)e.z, 0.0f);
}

// Node field in FP32 (MIXED steps; the push reads only this copy).  Same
// reading as k_node_E: minus the volume-weighted mean of the element
// gradients around the node, plasma-side pieces preferred.  A block covers a
// 32 x 4 x 2 brick of nodes and stages phi of the brick and a one-node halo
// (34 x 6 x 4) in shared memory, converted to FP32 once.  An interior-regular
// node applies its parity's 27-point stencil (cFold); any other node its row of
// the set-up (27 x 3 coefficients and the q_T terms of its interface tets).
constexpr int NE_BX = 32, NE_BY = 4, NE_BZ = 2;
constexpr int NE_TX = NE_BX + 2, NE_TY = NE_BY + 2, NE_TZ = NE_BZ + 2;
constexpr int NE_FOLD = 97;   // the parity tables' stride in shared memory (not a multiple of the 32 banks)
__global__ void __launch_bounds__(NE_BX * NE_BY * NE_BZ) k_node_E_f(Mesh m, const int* row, long long R,
                                                                    const float* coef, const int* qoff,
                                                                    const int4* qent, const double* qT,
                                                                    const double* phi, float4* Ef) {
    __shared__ float ph[NE_TX * NE_TY * NE_TZ];
    __shared__ float sF[2 * NE_FOLD];
    const int i0 = blockIdx.x * NE_BX, j0 = blockIdx.y * NE_BY, k0 = blockIdx.z * NE_BZ;
    const int tid = threadIdx.x + NE_BX * (threadIdx.y + NE_BY * threadIdx.z);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y, k = k0 + threadIdx.z;
    const bool mine = i < m.NX && j < m.NY && k < m.NZ;
    const long long n = mine ? node_id(m, i, j, k) : 0;
    const int r = mine ? row[n] : -1;
    for (int q = tid; q < 2 * 81; q += NE_BX * NE_BY * NE_BZ) sF[(q / 81) * NE_FOLD + q % 81] = (&cFold[0][0])[q];
    for (int q = tid; q < NE_TX * NE_TY * NE_TZ; q += NE_BX * NE_BY * NE_BZ) {
        const int gi = i0 - 1 + q % NE_TX, gj = j0 - 1 + (q / NE_TX) % NE_TY, gk = k0 - 1 + q / (NE_TX * NE_TY);
        const bool in = gi >= 0 && gj >= 0 && gk >= 0 && gi < m.NX && gj < m.NY && gk < m.NZ;
        ph[q] = in ? (float)phi[node_id(m, gi, gj, gk)] : 0.0f;
    }
    __syncthreads();
    if (!mine) return;
    // the node in the staged brick; neighbour nb at ph[c + off(nb)]
    const float* c = ph + (threadIdx.x + 1) + NE_TX * ((threadIdx.y + 1) + NE_TY * (threadIdx.z + 1));
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
    if (r < 0) {
        const float* F = sF + ((i + j + k) & 1) * NE_FOLD;
#pragma unroll
        for (int nb = 0; nb < 27; ++nb) {
            const float f = c[(nb % 3 - 1) + NE_TX * ((nb / 3 % 3 - 1) + NE_TY * (nb / 9 - 1))];
            e0 += F[3 * nb] * f;
            e1 += F[3 * nb + 1] * f;
            e2 += F[3 * nb + 2] * f;
        }
        const float ih = 1.0f / (float)m.h;
        e0 *= ih; e1 *= ih; e2 *= ih;
    } else {
        const float* cf = coef + r;
#pragma unroll
        for (int nb = 0; nb < 27; ++nb) {
            const float f = c[(nb % 3 - 1) + NE_TX * ((nb / 3 % 3 - 1) + NE_TY * (nb / 9 - 1))];
            e0 += cf[(3 * nb) * R] * f;
            e1 += cf[(3 * nb + 1) * R] * f;
            e2 += cf[(3 * nb + 2) * R] * f;
        }
        const int q1 = qoff[r + 1];
        for (int q = qoff[r]; q < q1; ++q) {
            const int4 w = qent[q];
            const float qt = (float)qT[w.x];
            e0 += __int_as_float(w.y) * qt;
            e1 += __int_as_float(w.z) * qt;
            e2 += __int_as_float(w.w) * qt;
        }
    }
    Ef[n] = make_float4(e0, e1, e2, 0.f);
}

static void launch_node_E_f(const Ctx& c, cudaStream_t st) {
    const Mesh& m = c.mesh;
    dim3 grid((m.NX + NE_BX - 1) / NE_BX, (m.NY + NE_BY - 1) / NE_BY, (m.NZ + NE_BZ - 1) / NE_BZ);
    k_node_E_f<<<grid, dim3(NE_BX, NE_BY, NE_BZ), 0, st>>>(m, c.ne_row, c.ne_nrows, c.ne_coef, c.ne_qoff, c.ne_q,
                                                          c.qT, c.phi, c.Ef);
}


// ---- surface diagnostics: total collected charge, area-mean potential on Gamma_h ----
__global__ void k_surface_diag(Mesh m, long long nit, const int* it_cell, const int* it_t, const double* it_data,
                               const double* qT, const double* phi, double* partial, unsigned* ticket,
                               double* out) {
    long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    // the object's surface only: a bedrock-plane tet lies inside the object
    if (T < nit && it_data[T * IT_STRIDE + IT_KIND] == 0.0) {
        const double* rec = it_data + T * IT_STRIDE;
        int c = it_cell[T], t = it_t[T];
        int i = c % m.nx, j = (c / m.nx) % m.ny, k = c / (m.nx * m.ny);
        int p = (i + j + k) & 1;
        double s = qT[T] * rec[IT_SJ];
        for (int a = 0; a < 4; ++a) {
            int av, bv, cv; loff(cTf.vert[p][t][a], av, bv, cv);
            s += phi[node_id(m, i + av, j + bv, k + cv)] * rec[IT_S + a];
        }
        v[0] = s; v[1] = rec[IT_AREA];
    }
    double tot[2];
    if (grid_sum<2>(v, partial, ticket, tot) && threadIdx.x == 0) out[0] = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
}

__global__ void k_surface_charge(RhsArgs a, double* partial, unsigned* ticket, double* out) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[1] = {0};
    if (c < a.ncut) {
        int ns = *a.nspec;
        for (int s = 0; s < ns; ++s) v[0] += a.coefs[s] * (double)(long long)a.surf[(long long)s * a.ncut + c];
    }
    double tot[1];
    if (grid_sum<1>(v, partial, ticket, tot) && threadIdx.x == 0) out[0] = tot[0];
}

// ------------------------------------------------------------------------------------
static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }
// device count of solves (PCG start extrapolation), scalar slot 43
static long long* solve_hist(Ctx& c) { return (long long*)(c.scal + 43); }

// one node per thread: 256-thread blocks, or 64-thread ones for a mesh whose
// 256-thread grid would leave most SMs idle (these kernels are FP64-bound)
static int node_threads(long long N) { return N < 152LL * 256 ? 64 : 256; }
static unsigned node_blocks(long long N) {
    const int t = node_threads(N);
    return (unsigned)((N + t - 1) / t);
}

static FieldArgs fargs(Ctx& c) {
    FieldArgs f;
    f.m = c.mesh; f.o = c.obj; f.ntype = c.ntype; f.coef = c.patch_coef; f.coeff = c.patch_coeff;
    f.invdiag = c.invdiag; f.invdiagf = c.invdiagf;
    return f;
}

// device scratch layout in c.scal: [0..15] PcgState, [16..23] species coefs,
// [24] nspec (as int), [32..] diag outputs
static PcgState* pcg_state(Ctx& c) { return (PcgState*)c.scal; }
static double* coefs_dev(Ctx& c) { return c.scal + 16; }
static int* nspec_dev(Ctx& c) { return (int*)(c.scal + 24); }
static double* diag_dev(Ctx& c) { return c.scal + 32; }

static RhsArgs rargs(Ctx& c) {
    RhsArgs a;
    a.W = c.Wall;
    a.surf = c.surfall;
    a.coefs = coefs_dev(c);
    a.nspec = nspec_dev(c);
    a.ncut = c.ncut;
    return a;
}

static FluxRows flux_rows(const Ctx& c) { return FluxRows{c.ne_row, c.ne_qoff, c.ne_q, c.ne_qc}; }

cudaError_t launch_field_lift(Ctx& c) {
    FieldArgs f = fargs(c);
    k_matvec<<<nb(c.mesh.nnodes), 256, 0, c.stream>>>(f, c.gdir, c.lift);
    return cudaGetLastError();
}

cudaError_t launch_pcg_coop(Ctx& c, cudaStream_t st);   // pcg_coop.cu

// q_T, RHS, warm start, then the persistent PCG and the node field
// hybrid grid: the PIC nodes are the IFE nodes (r i, r j, r k); the push reads
// the node field there
__global__ void k_E_to_pic(Mesh pm, Mesh fm, int r, const double4* E, const float4* Ef, double4* Ep, float4* Efp,
                           int both) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= pm.nnodes) return;
    int i = (int)(n % pm.NX), j = (int)((n / pm.NX) % pm.NY), k = (int)(n / ((long long)pm.NX * pm.NY));
    long long f = node_id(fm, r * i, r * j, r * k);
    Efp[n] = Ef[f];
    if (both) Ep[n] = E[f];
}

cudaError_t launch_E_to_pic(const Ctx& c, cudaStream_t st, bool both) {
    if (c.refine == 1) return cudaSuccess;
    k_E_to_pic<<<nb(c.pmesh.nnodes), 256, 0, st>>>(c.pmesh, c.mesh, c.refine, c.E, c.Ef, c.Ep, c.Efp, both ? 1 : 0);
    return cudaGetLastError();
}

static cudaError_t solve_sequence(Ctx& c, cudaStream_t st, const double* Fext) {
    FieldArgs f = fargs(c);
    RhsArgs a = rargs(c);
    long long N = c.mesh.nnodes;
    if (!Fext) {
        if (c.ncut > 0) k_qcut<<<nb(c.ncut), 256, 0, st>>>(a, c.cut_area, c.qcut);
        if (c.nit > 0) k_qtets<<<nb(c.nit), 256, 0, st>>>(c.nit, c.it_acc, c.qcut, c.qT);
    }
    k_rhs<<<node_blocks(N), node_threads(N), 0, st>>>(f, a, flux_rows(c), c.qT, c.lift, c.b, Fext,
                                                       solve_hist(c));
    k_u_from_phi<<<nb(N), 256, 0, st>>>(N, c.ntype, c.phi, c.phi_prev, c.gdir, c.u, solve_hist(c));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pcg_coop(c, st);
    if (e != cudaSuccess) return e;
    if (c.precision == PIFEPIC_MIXED) launch_node_E_f(c, st);
    else k_node_E<<<node_blocks(N), node_threads(N), 0, st>>>(f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi,
                                                               c.E, c.Ef);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_E_to_pic(c, st, c.precision != PIFEPIC_MIXED);
}

// the solve's pieces around the PCG, for the batched step (batch.cu)
cudaError_t launch_solve_prefix(Ctx& c, cudaStream_t st) {
    FieldArgs f = fargs(c);
    RhsArgs a = rargs(c);
    long long N = c.mesh.nnodes;
    if (c.ncut > 0) k_qcut<<<nb(c.ncut), 256, 0, st>>>(a, c.cut_area, c.qcut);
    if (c.nit > 0) k_qtets<<<nb(c.nit), 256, 0, st>>>(c.nit, c.it_acc, c.qcut, c.qT);
    k_rhs<<<node_blocks(N), node_threads(N), 0, st>>>(f, a, flux_rows(c), c.qT, c.lift, c.b, nullptr,
                                                       solve_hist(c));
    k_u_from_phi<<<nb(N), 256, 0, st>>>(N, c.ntype, c.phi, c.phi_prev, c.gdir, c.u, solve_hist(c));
    return cudaGetLastError();
}
cudaError_t launch_solve_suffix(Ctx& c, cudaStream_t st) {
    FieldArgs f = fargs(c);
    if (c.precision == PIFEPIC_MIXED) launch_node_E_f(c, st);
    else k_node_E<<<node_blocks(c.mesh.nnodes), node_threads(c.mesh.nnodes), 0, st>>>(
        f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E, c.Ef);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_E_to_pic(c, st, c.precision != PIFEPIC_MIXED);
}

// kernels launched per solve
int solve_graph_fixed_kernels(const Ctx& c) { return (c.ncut > 0) + (c.nit > 0) + 4 + (c.refine > 1); }

// The solve as one CUDA graph (both precisions): q_T -> RHS -> warm start ->
// persistent PCG -> node field
cudaError_t build_pcg_graph(Ctx& c) {
    plan_pcg(c);
    if (c.pcg_exec) { cudaGraphExecDestroy(c.pcg_exec); c.pcg_exec = nullptr; }
    if (c.pcg_graph) { cudaGraphDestroy(c.pcg_graph); c.pcg_graph = nullptr; }
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = solve_sequence(c, cs, nullptr);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c.pcg_exec, g, 0);
    if (e == cudaSuccess) c.pcg_graph = g;
    else if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

static cudaError_t set_pcg_state(Ctx& c) {
    PcgState h = {};
    h.tol2 = c.tol * c.tol;
    h.maxit = c.maxit;
    h.inner_red2 = c.inner_red * c.inner_red;
    h.margin2 = c.inner_margin * c.inner_margin;
    return cudaMemcpyAsync(c.scal, &h, sizeof(PcgState), cudaMemcpyHostToDevice, c.stream);
}

cudaError_t launch_pcg(Ctx& c) {
    cudaError_t e = set_pcg_state(c);
    if (e != cudaSuccess) return e;
    return cudaGraphLaunch(c.pcg_exec, c.stream);
}


// standalone solve with an external node load (solver parity)
cudaError_t launch_solve_external(Ctx& c, const double* Fdev, int* iters, double* relres) {
    cudaError_t e = set_pcg_state(c);
    if (e == cudaSuccess) e = solve_sequence(c, c.stream, Fdev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return e;
    PcgState hs;
    e = scopy(c.stream, &hs, pcg_state(c), sizeof(PcgState), cudaMemcpyDeviceToHost);
    if (iters) *iters = hs.it;
    if (relres) *relres = hs.relres;
    c.last_iters = hs.it; c.last_relres = hs.relres; c.last_conv = hs.converged;
    return e;
}

struct StatArgs {
    const unsigned long long* ctrall;
    const int* bcount[MAX_SPECIES];
    const unsigned long long* mov_n[MAX_SPECIES];
    int nspecies, nblocks;
    const double* scal;
    const double* diag;   // surface charge, potential; null: not gathered
    const int* err;
    StatPack* out;
};

// one block of 256 threads
__global__ void k_stat_pack(StatArgs a) {
    __shared__ long long part[8];
    const int t = threadIdx.x;
    for (int i = t; i < MAX_SPECIES * NCTR; i += blockDim.x) a.out->ctr[i] = a.ctrall[i];
    if (t < MAX_SPECIES) a.out->count[t] = 0;
    for (int s = 0; s < a.nspecies && s < MAX_SPECIES; ++s) {   // (a.nspecies is the same in every thread)
        long long v = 0;
        if (a.bcount[s])
            for (int b = t; b < a.nblocks; b += blockDim.x) v += a.bcount[s][b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) part[t >> 5] = v;
        __syncthreads();
        if (t == 0) {
            long long tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
            if (a.mov_n[s]) tot += (long long)a.mov_n[s][0];
            a.out->count[s] = tot;
        }
        __syncthreads();
    }
    if (t == 0) {
        const PcgState* S = (const PcgState*)a.scal;
        a.out->it = S->it;
        a.out->converged = S->converged;
        a.out->relres = S->relres;
        a.out->it_total = ((const long long*)a.scal)[40];
        a.out->outer_total = ((const long long*)a.scal)[41];
        a.out->surface_charge = a.diag ? a.diag[0] : 0.0;
        a.out->surface_potential = a.diag ? a.diag[1] : 0.0;
        a.out->err = *a.err;
    }
}

cudaError_t gather_stats(Ctx& c, StatPack* out, bool diag) {
    double* d = diag_dev(c);
    if (diag) {
        RhsArgs ra = rargs(c);
        if (c.nit > 0)
            k_surface_diag<<<nb(c.nit), 256, 0, c.stream>>>(c.mesh, c.nit, c.it_cell, c.it_t, c.it_data, c.qT, c.phi,
                                                            c.red, c.red_ticket, d + 1);
        else
            cudaMemsetAsync(d + 1, 0, sizeof(double), c.stream);
        if (c.ncut > 0)
            k_surface_charge<<<nb(c.ncut), 256, 0, c.stream>>>(ra, c.red, c.red_ticket, d);
        else
            cudaMemsetAsync(d, 0, sizeof(double), c.stream);
    }
    StatArgs a = {};
    a.ctrall = c.ctrall;
    a.nspecies = (int)c.sp.size();
    for (int s = 0; s < a.nspecies && s < MAX_SPECIES; ++s) {
        a.bcount[s] = c.sp[s].bcount;
        a.mov_n[s] = c.sp[s].mov_n;
    }
    a.nblocks = c.nblocks;
    a.scal = c.scal;
    a.diag = diag ? d : nullptr;
    a.err = c.err_word;
    a.out = c.stat_dev;
    k_stat_pack<<<1, 256, 0, c.stream>>>(a);
    cudaError_t e = cudaMemcpyAsync(c.stat_host, c.stat_dev, sizeof(StatPack), cudaMemcpyDeviceToHost, c.stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return e;
    *out = *c.stat_host;
    c.last_iters = out->it;
    c.last_relres = out->relres;
    c.last_conv = out->converged;
    return cudaSuccess;
}

// FP64 node field from the current phi into E only (the FP32 copy the MIXED
// push reads is left as the step made it)
cudaError_t launch_node_E64(Ctx& c) {
    FieldArgs f = fargs(c);
    k_node_E<<<node_blocks(c.mesh.nnodes), node_threads(c.mesh.nnodes), 0, c.stream>>>(
        f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E, nullptr);
    return cudaGetLastError();
}

cudaError_t set_field_tables(const TetTables& t) {
    // per cube of parity p holding the node at its local corner c8: G = sum
    // over the cube's tets containing it of vol_t grad_t at each corner (h = 1),
    // V = sum of their vol_t; summed in FP64
    double G[2][8][8][3] = {}, V[2][8] = {};
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 5; ++q)
            for (int a = 0; a < 4; ++a) {
                const int c8 = t.vert[p][q][a];   // the tet contains local corner c8
                V[p][c8] += t.vol[q];
                for (int b = 0; b < 4; ++b)
                    for (int d = 0; d < 3; ++d) G[p][c8][t.vert[p][q][b]][d] += t.vol[q] * t.grad[p][q][b][d];
            }
    // the eight cubes around a node of parity P: the cube with the node at its
    // corner c8 = (a, b, c) has parity P + a + b + c, and its corner (x, y, z) is
    // the node's neighbour (x - a, y - b, z - c)
    double F[2][27][3] = {}, W[2] = {};
    for (int P = 0; P < 2; ++P)
        for (int c8 = 0; c8 < 8; ++c8) {
            const int a = c8 & 1, b = (c8 >> 1) & 1, cc = (c8 >> 2) & 1, pc = (P + a + b + cc) & 1;
            W[P] += V[pc][c8];
            for (int cn = 0; cn < 8; ++cn) {
                const int nb = ((cn & 1) - a + 1) + 3 * (((cn >> 1) & 1) - b + 1) + 9 * (((cn >> 2) & 1) - cc + 1);
                for (int d = 0; d < 3; ++d) F[P][nb][d] += G[pc][c8][cn][d];
            }
        }
    float Ff[2][81];
    for (int P = 0; P < 2; ++P)
        for (int nb = 0; nb < 27; ++nb)
            for (int d = 0; d < 3; ++d) Ff[P][3 * nb + d] = (float)(-F[P][nb][d] / W[P]);
    cudaError_t e = cudaMemcpyToSymbol(cTf, &t, sizeof(TetTables));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cFold, Ff, sizeof(Ff));
    return e;
}

cudaError_t launch_qtets(Ctx& c) {
    RhsArgs a = rargs(c);
    if (c.ncut > 0) k_qcut<<<nb(c.ncut), 256, 0, c.stream>>>(a, c.cut_area, c.qcut);
    if (c.nit > 0) k_qtets<<<nb(c.nit), 256, 0, c.stream>>>(c.nit, c.it_acc, c.qcut, c.qT);
    return cudaGetLastError();
}

// ======================================================================================
// Field solve that allocates nothing (pifepic_solve_field_noalloc).
//
// Some callers cannot call cudaMalloc once their run is under way: a serving
// loop whose device memory is handed out by a pool it does not own (a
// cudaMalloc there can fail or stall the whole process on a device
// synchronisation), or an embedding that forbids allocation after start-up.
// pifepic_solve_field allocates a staging buffer and builds a CUDA graph on
// every call, so those callers need this variant.  It reuses the context's
// operator (read only), takes the load F, the flux jumps q (NULL: none) and
// the output phi as caller-owned device arrays, and keeps every work vector of
// the PCG in one file-scope device array of fixed size, found once per device
// with cudaGetSymbolAddress.  It always runs the FP64 PCG, whatever the
// context's precision.
// ======================================================================================
constexpr long long NOALLOC_MAX_NODES = 131072;                  // 2^17 mesh nodes
constexpr long long NOALLOC_PARTIALS = 4 * (NOALLOC_MAX_NODES / 256 + 1);
constexpr long long NOALLOC_DOUBLES = 5 * NOALLOC_MAX_NODES + NOALLOC_PARTIALS + 32;
// layout: u, b, r, p, q (NOALLOC_MAX_NODES each) | partials | PcgState + ticket
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// the PCG steps of the graph version without the conditional handle; every
// launch after convergence returns at once, so the host can queue the
// iteration cap without waiting for the device
__global__ void k_na_init(FieldArgs f, const double* b, const double* q, double* r, double* p, double* partial,
                          unsigned* ticket, PcgState* S) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[3] = {0, 0, 0};
    if (n < f.m.nnodes) {
        double bn = b[n];
        double rn = (f.ntype[n] == -3) ? 0.0 : bn - q[n];
        double zn = f.invdiag[n] * rn;
        r[n] = rn;
        p[n] = zn;
        v[0] = bn * bn; v[1] = rn * rn; v[2] = rn * zn;
    }
    double tot[3];
    if (grid_sum<3>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->bb = tot[0]; S->rr = tot[1]; S->rz = tot[2];
        S->it = 0;
        S->converged = (tot[0] == 0.0) || (tot[1] <= S->tol2 * tot[0]);
        S->done = S->converged || (S->maxit <= 0);
        S->relres = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
    }
}

__global__ void k_na_spmv(FieldArgs f, const double* p, double* q, double* partial, unsigned* ticket, PcgState* S) {
    if (S->done) return;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (n < f.m.nnodes) {
        int i, j, k;
        node_ijk(f.m, n, i, j, k);
        double y = apply_row<double>(f, n, i, j, k, p, f.coef);
        q[n] = y;
        v[0] = p[n] * y;
    }
    double tot[1];
    if (grid_sum<1>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->pq = tot[0];
        S->alpha = S->rz / tot[0];
    }
}

__global__ void k_na_update(FieldArgs f, double* u, double* r, const double* p, const double* q, double* partial,
                            unsigned* ticket, PcgState* S) {
    if (S->done) return;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double alpha = S->alpha;
    double v[2] = {0, 0};
    if (n < f.m.nnodes) {
        double rn = r[n] - alpha * q[n];
        u[n] = u[n] + alpha * p[n];
        r[n] = rn;
        v[0] = rn * rn; v[1] = rn * f.invdiag[n] * rn;
    }
    double tot[2];
    if (grid_sum<2>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->rr = tot[0];
        S->beta = tot[1] / S->rz;
        S->rz = tot[1];
        S->it = S->it + 1;
        S->converged = tot[0] <= S->tol2 * S->bb;
        S->relres = sqrt(tot[0] / S->bb);
        S->done = S->converged || (S->it >= S->maxit);
    }
}

__global__ void k_na_dir(FieldArgs f, const double* r, double* p, const PcgState* S) {
    if (S->done) return;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < f.m.nnodes) p[n] = f.invdiag[n] * r[n] + S->beta * p[n];
}

__global__ void k_na_state(PcgState* S, unsigned* ticket, double tol2, int maxit) {
    PcgState s = {};
    s.tol2 = tol2;
    s.maxit = maxit;
    *S = s;
    *ticket = 0u;
}

// set-up once per device (with that device current): in host code the name of
// a __device__ array is a host-side stand-in, not a device address, so the
// address is looked up with cudaGetSymbolAddress and cached per device.  Two
// threads doing the first call on one device at once both look it up and
// store the same value (an atomic store, so neither sees a torn pointer).
static std::atomic<void*> g_noalloc_dev[64];

pifepic_status solve_field_noalloc(Ctx& c, const double* F, const double* q, double* phi, int* iters,
                                   double* relres) {
    long long N = c.mesh.nnodes;
    if (N > NOALLOC_MAX_NODES) {
        char b[256];
        snprintf(b, sizeof(b), "solve_field_noalloc: mesh has %lld nodes; the fixed scratch holds at most %lld",
                 N, NOALLOC_MAX_NODES);
        c.err = b;
        log_error(b);
        return PIFEPIC_EINVAL;
    }
    // the scratch address is per device and the kernels run on the context's
    // stream, so the context's device must be the current one
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        c.err = "solve_field_noalloc: no current device";
        log_error(c.err.c_str());
        return PIFEPIC_ECUDA;
    }
    if (dev != c.device || dev < 0 || dev >= 64) {
        char b[160];
        snprintf(b, sizeof(b), "solve_field_noalloc: current device %d is not the context's device %d", dev,
                 c.device);
        c.err = b;
        log_error(b);
        return PIFEPIC_EINVAL;
    }
    void* base_ptr = g_noalloc_dev[dev].load(std::memory_order_acquire);
    if (!base_ptr) {
        cudaError_t e = cudaGetSymbolAddress(&base_ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !base_ptr) {
            c.err = std::string("solve_field_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            log_error(c.err.c_str());
            return PIFEPIC_ECUDA;
        }
        g_noalloc_dev[dev].store(base_ptr, std::memory_order_release);
    }
    double* base = (double*)base_ptr;
    double* u = base;
    double* bvec = base + NOALLOC_MAX_NODES;
    double* r = base + 2 * NOALLOC_MAX_NODES;
    double* p = base + 3 * NOALLOC_MAX_NODES;
    double* qv = base + 4 * NOALLOC_MAX_NODES;
    double* partial = base + 5 * NOALLOC_MAX_NODES;
    PcgState* S = (PcgState*)(partial + NOALLOC_PARTIALS);
    unsigned* ticket = (unsigned*)(partial + NOALLOC_PARTIALS + 24);
    FieldArgs f = fargs(c);
    RhsArgs a = rargs(c);
    unsigned gb = nb(N);
    cudaStream_t st = c.stream;
    k_na_state<<<1, 1, 0, st>>>(S, ticket, c.tol * c.tol, c.maxit);
    k_rhs<<<gb, 256, 0, st>>>(f, a, flux_rows(c), q, c.lift, bvec, F, nullptr);
    cudaMemsetAsync(u, 0, sizeof(double) * N, st);
    k_matvec<<<gb, 256, 0, st>>>(f, u, qv);
    k_na_init<<<gb, 256, 0, st>>>(f, bvec, qv, r, p, partial, ticket, S);
    for (int it = 0; it < c.maxit; ++it) {
        k_na_spmv<<<gb, 256, 0, st>>>(f, p, qv, partial, ticket, S);
        k_na_update<<<gb, 256, 0, st>>>(f, u, r, p, qv, partial, ticket, S);
        k_na_dir<<<gb, 256, 0, st>>>(f, r, p, S);
    }
    k_phi_from_u<<<gb, 256, 0, st>>>(N, u, c.gdir, phi, S);
    cudaError_t e = cudaGetLastError();
    PcgState hs;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, S, sizeof(PcgState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        c.err = std::string("solve_field_noalloc: ") + cudaGetErrorString(e);
        log_error(c.err.c_str());
        return PIFEPIC_ECUDA;
    }
    if (iters) *iters = hs.it;
    if (relres) *relres = hs.relres;
    return PIFEPIC_OK;
}

}  // namespace pf
