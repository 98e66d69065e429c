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

#include "internal.h"

namespace pf {

__constant__ TetTables cTf;

struct PcgState {
    double bb, rz, rr, pq, alpha, beta, tol2, relres;
    int it, maxit, done, converged;
    // mixed mode: FP32 inner PCG inside FP64 refinement
    double rr64, inner_tol2, inner_bb;
    int inner_it, outer_it, inner_max, done_in;
};

struct FieldArgs {
    Mesh m;
    Object o;
    const int* ntype;
    const double* coef;       // patch rows [npatch][19]
    const float* coeff;
    const double* invdiag;
    const float* invdiagf;
};

static __device__ __forceinline__ void loff(int l, int& a, int& b, int& c) {
    a = l & 1; b = (l >> 1) & 1; c = (l >> 2) & 1;
}

// y_n = (A x)_n for the IFE operator; Dirichlet rows give 0 (x is 0 there)
template <typename T>
static __device__ __forceinline__ T apply_row(const FieldArgs& f, long long n, int i, int j, int k, const T* x,
                                              const T* coef) {
    const Mesh& m = f.m;
    int ty = f.ntype[n];
    if (ty == -3) return (T)0;
    const long long sx = 1, sy = m.NX, sz = (long long)m.NX * m.NY;
    bool xm = i > 0, xp = i < m.nx, ym = j > 0, yp = j < m.ny, zm = k > 0, zp = k < m.nz;
    if (ty >= 0) {
        const T* c = coef + (long long)ty * 19;
        T y = c[0] * x[n];
        if (xm) y += c[1] * x[n - sx];
        if (xp) y += c[2] * x[n + sx];
        if (ym) y += c[3] * x[n - sy];
        if (yp) y += c[4] * x[n + sy];
        if (zm) y += c[5] * x[n - sz];
        if (zp) y += c[6] * x[n + sz];
        if ((i + j + k) & 1) return y;
        if (xm && ym) y += c[7] * x[n - sx - sy];
        if (xp && ym) y += c[8] * x[n + sx - sy];
        if (xm && yp) y += c[9] * x[n - sx + sy];
        if (xp && yp) y += c[10] * x[n + sx + sy];
        if (xm && zm) y += c[11] * x[n - sx - sz];
        if (xp && zm) y += c[12] * x[n + sx - sz];
        if (xm && zp) y += c[13] * x[n - sx + sz];
        if (xp && zp) y += c[14] * x[n + sx + sz];
        if (ym && zm) y += c[15] * x[n - sy - sz];
        if (yp && zm) y += c[16] * x[n + sy - sz];
        if (ym && zp) y += c[17] * x[n - sy + sz];
        if (yp && zp) y += c[18] * x[n + sy + sz];
        return y;
    }
    // regular row: assembled P1 stencil of the 5-tet split with eps of the region;
    // each coefficient = (cubes sharing the edge) x (per-cube element integral)
    T eps = (T)(ty == -2 ? f.o.eps_minus : f.o.eps_plus);
    T h = (T)m.h;
    int cx = (int)xm + (int)xp, cy = (int)ym + (int)yp, cz = (int)zm + (int)zp;
    bool odd = (i + j + k) & 1;
    T y = (T)(cx * cy * cz) * (odd ? (T)0.5 : (T)0.75) * h * x[n];
    T ax = (T)0, ay = (T)0, az = (T)0;
    if (xm) ax += x[n - sx];
    if (xp) ax += x[n + sx];
    if (ym) ay += x[n - sy];
    if (yp) ay += x[n + sy];
    if (zm) az += x[n - sz];
    if (zp) az += x[n + sz];
    T h6 = h / (T)6;
    y -= h6 * ((T)(cy * cz) * ax + (T)(cx * cz) * ay + (T)(cx * cy) * az);
    if (!odd) {
        T dxy = (T)0, dxz = (T)0, dyz = (T)0;
        if (xm && ym) dxy += x[n - sx - sy];
        if (xp && ym) dxy += x[n + sx - sy];
        if (xm && yp) dxy += x[n - sx + sy];
        if (xp && yp) dxy += x[n + sx + sy];
        if (xm && zm) dxz += x[n - sx - sz];
        if (xp && zm) dxz += x[n + sx - sz];
        if (xm && zp) dxz += x[n - sx + sz];
        if (xp && zp) dxz += x[n + sx + sz];
        if (ym && zm) dyz += x[n - sy - sz];
        if (yp && zm) dyz += x[n + sy - sz];
        if (ym && zp) dyz += x[n - sy + sz];
        if (yp && zp) dyz += x[n + sy + sz];
        T h12 = h / (T)12;
        y -= h12 * ((T)cz * dxy + (T)cy * dxz + (T)cx * dyz);
    }
    return eps * y;
}

static __device__ __forceinline__ void node_ijk(const Mesh& m, long long n, int& i, int& j, int& k) {
    i = (int)(n % m.NX);
    j = (int)((n / m.NX) % m.NY);
    k = (int)(n / ((long long)m.NX * m.NY));
}

// ---- deterministic block reduction of NV doubles -----------------------------
template <int NV>
static __device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
    // sh: [NV][32]
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = v[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[q * 32 + w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < nw ? sh[q * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[q] = s;
        }
    }
    __syncthreads();
}

// writes block partials; returns true in the one block that arrives last,
// which then holds the grid totals in tot[]
template <int NV>
static __device__ bool grid_sum(double (&v)[NV], double* partial, unsigned* ticket, double (&tot)[NV]) {
    __shared__ double sh[NV * 32];
    __shared__ bool last;
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) partial[(long long)q * gridDim.x + blockIdx.x] = v[q];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
    for (int q = 0; q < NV; ++q) {
        s[q] = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s[q] += ((volatile double*)partial)[(long long)q * gridDim.x + b];
    }
    block_sum<NV>(s, sh);
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) tot[q] = s[q];
        *ticket = 0;
    }
    return true;
}

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

__global__ void k_rhs(FieldArgs f, RhsArgs a, const unsigned char* imask, const int* ibase, const double* it_data,
                      const double* qT, const double* lift, double* b, const double* Fext) {
    const Mesh& m = f.m;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
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
    if (ty >= 0) {   // touches interface tets: flux-jump load
        int i, j, k;
        node_ijk(m, n, i, j, k);
        for (int c8 = 0; c8 < 8; ++c8) {
            int aa, bb, cc; loff(c8, aa, bb, cc);
            int ci = i - aa, cj = j - bb, ck = k - cc;
            if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
            long long cell = cell_id(m, ci, cj, ck);
            unsigned mk = imask[cell];
            if (!mk) continue;
            int p = (ci + cj + ck) & 1;
            int T = ibase[cell];
            for (int t = 0; t < 5; ++t) {
                if (!((mk >> t) & 1)) continue;
                for (int v = 0; v < 4; ++v)
                    if (cTf.vert[p][t][v] == c8) F += qT[T] * it_data[(long long)T * IT_STRIDE + IT_C + v];
                ++T;
            }
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

// r = b - Au (Au in q); z = D^-1 r; p = z; bb, rr, rz
__global__ void k_pcg_init(FieldArgs f, const double* b, const double* q, double* r, double* p, double* partial,
                           unsigned* ticket, PcgState* S, cudaGraphConditionalHandle h) {
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
        bool done = (tot[0] == 0.0) || (tot[1] <= S->tol2 * tot[0]) || (S->maxit <= 0);
        S->done = done;
        S->converged = (tot[0] == 0.0) || (tot[1] <= S->tol2 * tot[0]);
        S->relres = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
        cudaGraphSetConditional(h, done ? 0u : 1u);
    }
}

// q = A p; pq
__global__ void k_pcg_spmv(FieldArgs f, const double* p, double* q, double* partial, unsigned* ticket,
                           PcgState* S, cudaGraphConditionalHandle h) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // the loop ends unless this iteration's update re-arms it
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
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

// u += alpha p; r -= alpha q; rr, rz; convergence
__global__ void k_pcg_update(FieldArgs f, double* u, double* r, const double* p, const double* q, double* partial,
                             unsigned* ticket, PcgState* S, cudaGraphConditionalHandle h, long long* it_total) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double alpha = S->alpha;
    double v[2] = {0, 0};
    if (n < f.m.nnodes) {
        double un = u[n] + alpha * p[n];
        double rn = r[n] - alpha * q[n];
        u[n] = un;
        r[n] = rn;
        double zn = f.invdiag[n] * rn;
        v[0] = rn * rn; v[1] = rn * zn;
    }
    double tot[2];
    if (grid_sum<2>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->rr = tot[0];
        S->beta = tot[1] / S->rz;
        S->rz = tot[1];
        S->it = S->it + 1;
        *it_total += 1;
        bool conv = tot[0] <= S->tol2 * S->bb;
        bool done = conv || (S->it >= S->maxit);
        S->done = done;
        S->converged = conv;
        S->relres = sqrt(tot[0] / S->bb);
        if (!done) cudaGraphSetConditional(h, 1u);
    }
}

__global__ void k_pcg_dir(FieldArgs f, const double* r, double* p, const PcgState* S) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= f.m.nnodes) return;
    if (S->done) return;
    p[n] = f.invdiag[n] * r[n] + S->beta * p[n];
}

// phi = u + g; a zero right-hand side has the lift alone as its solution
__global__ void k_phi_from_u(long long N, const double* u, const double* g, double* phi, const PcgState* S) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) phi[n] = S->bb == 0.0 ? g[n] : u[n] + g[n];
}
__global__ void k_u_from_phi(long long N, const int* ntype, const double* phi, const double* g, double* u) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) u[n] = ntype[n] == -3 ? 0.0 : phi[n] - g[n];
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
                    if (vp > 0.0) {
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

// ---- surface diagnostics: total collected charge, area-mean potential on Gamma_h ----
__global__ void k_surface_diag(Mesh m, long long nit, const int* it_cell, const int* it_t, const double* it_data,
                               const double* qT, const double* phi, double* partial, unsigned* ticket,
                               double* out) {
    long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (T < nit) {
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

cudaError_t launch_field_lift(Ctx& c) {
    FieldArgs f = fargs(c);
    k_matvec<<<nb(c.mesh.nnodes), 256, 0, c.stream>>>(f, c.gdir, c.lift);
    return cudaGetLastError();
}

static cudaError_t solve_prefix(Ctx& c, const double* Fext) {
    FieldArgs f = fargs(c);
    RhsArgs a = rargs(c);
    long long N = c.mesh.nnodes;
    if (!Fext) {
        if (c.ncut > 0) k_qcut<<<nb(c.ncut), 256, 0, c.stream>>>(a, c.cut_area, c.qcut);
        if (c.nit > 0) k_qtets<<<nb(c.nit), 256, 0, c.stream>>>(c.nit, c.it_acc, c.qcut, c.qT);
    }
    k_rhs<<<nb(N), 256, 0, c.stream>>>(f, a, c.imask, c.ibase, c.it_data, c.qT, c.lift, c.b, Fext);
    k_u_from_phi<<<nb(N), 256, 0, c.stream>>>(N, c.ntype, c.phi, c.gdir, c.u);
    k_matvec<<<nb(N), 256, 0, c.stream>>>(f, c.u, c.q);
    return cudaGetLastError();
}

static cudaError_t find_sink(cudaGraph_t g, cudaGraphNode_t* sink) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    e = cudaGraphGetNodes(g, nodes.data(), &n);
    if (e != cudaSuccess) return e;
    *sink = nullptr;
    for (auto nd : nodes) {
        size_t nout = 0;
        e = cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout);
        if (e != cudaSuccess) return e;
        if (nout == 0) *sink = nd;
    }
    return cudaSuccess;
}

// Build the solve graph:  q_T -> RHS -> r0 -> WHILE { spmv, update, dir } -> phi -> E
cudaError_t build_pcg_graph(Ctx& c) {
    if (c.pcg_exec) { cudaGraphExecDestroy(c.pcg_exec); c.pcg_exec = nullptr; }
    if (c.pcg_graph) { cudaGraphDestroy(c.pcg_graph); c.pcg_graph = nullptr; }
    cudaError_t e;
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g;
    e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return e; }
    cudaGraphConditionalHandle h;
    long long N = c.mesh.nnodes;
    unsigned gb = nb(N);
    FieldArgs f = fargs(c);
    PcgState* S = pcg_state(c);
    cudaStream_t keep = c.stream;
    cudaGraphNode_t sink, cond;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) goto fail;
    c.stream = cs;
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    solve_prefix(c, nullptr);
    k_pcg_init<<<gb, 256, 0, cs>>>(f, c.b, c.q, c.r, c.p, c.red, c.red_ticket, S, h);
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) goto fail;
    e = find_sink(g, &sink);
    if (e != cudaSuccess) goto fail;
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cond, g, &sink, nullptr, 1, &cp);
    if (e != cudaSuccess) goto fail;
    body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_pcg_spmv<<<gb, 256, 0, cs>>>(f, c.p, c.q, c.red, c.red_ticket, S, h);
    k_pcg_update<<<gb, 256, 0, cs>>>(f, c.u, c.r, c.p, c.q, c.red, c.red_ticket, S, h, (long long*)(c.scal + 40));
    k_pcg_dir<<<gb, 256, 0, cs>>>(f, c.r, c.p, S);
    e = cudaStreamEndCapture(cs, &body);
    if (e != cudaSuccess) goto fail;
    e = cudaStreamBeginCaptureToGraph(cs, g, &cond, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_phi_from_u<<<gb, 256, 0, cs>>>(N, c.u, c.gdir, c.phi, S);
    k_node_E<<<gb, 256, 0, cs>>>(f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E, c.Ef);
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) goto fail;
    e = cudaGraphInstantiate(&c.pcg_exec, g, 0);
    if (e != cudaSuccess) goto fail;
    c.pcg_graph = g;
    c.stream = keep;
    cudaStreamDestroy(cs);
    return cudaSuccess;
fail:
    c.stream = keep;
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

// kernels in the solve graph outside the PCG loop (3 more per iteration)
int solve_graph_fixed_kernels(const Ctx& c) { return (c.ncut > 0) + (c.nit > 0) + 6; }

cudaError_t launch_pcg(Ctx& c) {
    PcgState h = {};
    h.tol2 = c.tol * c.tol;
    h.maxit = c.maxit;
    cudaError_t e = cudaMemcpyAsync(c.scal, &h, sizeof(PcgState), cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return e;
    return cudaGraphLaunch(c.pcg_exec, c.stream);
}

cudaError_t launch_rhs(Ctx& c) { return cudaSuccess; }

// standalone solve with an external node load (solver parity): not graph-captured
cudaError_t launch_solve_external(Ctx& c, const double* Fdev, int* iters, double* relres) {
    FieldArgs f = fargs(c);
    long long N = c.mesh.nnodes;
    unsigned gb = nb(N);
    PcgState* S = pcg_state(c);
    PcgState hs = {};
    hs.tol2 = c.tol * c.tol;
    hs.maxit = c.maxit;
    cudaError_t e = cudaMemcpyAsync(S, &hs, sizeof(PcgState), cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return e;
    solve_prefix(c, Fdev);
    // run the same kernels with a host loop; the conditional handle is unused
    // outside a graph, so pass a zero handle and never call the setter path
    cudaGraph_t g;
    cudaGraphExec_t ge;
    cudaGraphConditionalHandle hnd;
    e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    e = cudaGraphConditionalHandleCreate(&hnd, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return e; }
    cudaStream_t cs;
    cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    cudaGraphNode_t sink = nullptr, cond;
    cudaGraphNodeParams cp = {};
    cudaGraph_t body;
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        k_pcg_init<<<gb, 256, 0, cs>>>(f, c.b, c.q, c.r, c.p, c.red, c.red_ticket, S, hnd);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = find_sink(g, &sink);
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cond, g, &sink, nullptr, 1, &cp);
    }
    if (e == cudaSuccess) {
        body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    }
    if (e == cudaSuccess) {
        k_pcg_spmv<<<gb, 256, 0, cs>>>(f, c.p, c.q, c.red, c.red_ticket, S, hnd);
        k_pcg_update<<<gb, 256, 0, cs>>>(f, c.u, c.r, c.p, c.q, c.red, c.red_ticket, S, hnd, (long long*)(c.scal + 40));
        k_pcg_dir<<<gb, 256, 0, cs>>>(f, c.r, c.p, S);
        e = cudaStreamEndCapture(cs, &body);
    }
    if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(cs, g, &cond, nullptr, 1, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            k_phi_from_u<<<gb, 256, 0, cs>>>(N, c.u, c.gdir, c.phi, S);
            k_node_E<<<gb, 256, 0, cs>>>(f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E, c.Ef);
            e = cudaStreamEndCapture(cs, &g);
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) {
        e = cudaGraphLaunch(ge, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        cudaGraphExecDestroy(ge);
    }
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return e;
    e = scopy(c.stream, &hs, S, sizeof(PcgState), cudaMemcpyDeviceToHost);
    if (iters) *iters = hs.it;
    if (relres) *relres = hs.relres;
    c.last_iters = hs.it; c.last_relres = hs.relres; c.last_conv = hs.converged;
    return e;
}

cudaError_t read_pcg_state(Ctx& c) {
    PcgState hs;
    cudaError_t e = cudaMemcpyAsync(&hs, c.scal, sizeof(PcgState), cudaMemcpyDeviceToHost, c.stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c.stream);
    c.last_iters = hs.it; c.last_relres = hs.relres; c.last_conv = hs.converged;
    return e;
}

cudaError_t launch_surface_diag(Ctx& c, double* out2) {
    double* d = diag_dev(c);
    RhsArgs a = rargs(c);
    if (c.nit > 0)
        k_surface_diag<<<nb(c.nit), 256, 0, c.stream>>>(c.mesh, c.nit, c.it_cell, c.it_t, c.it_data, c.qT, c.phi,
                                                        c.red, c.red_ticket, d + 1);
    else
        cudaMemsetAsync(d + 1, 0, sizeof(double), c.stream);
    if (c.ncut > 0)
        k_surface_charge<<<nb(c.ncut), 256, 0, c.stream>>>(a, c.red, c.red_ticket, d);
    else
        cudaMemsetAsync(d, 0, sizeof(double), c.stream);
    cudaError_t e = cudaMemcpyAsync(out2, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c.stream);
}

cudaError_t launch_node_E(Ctx& c) {
    FieldArgs f = fargs(c);
    k_node_E<<<nb(c.mesh.nnodes), 256, 0, c.stream>>>(f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E,
                                                      c.Ef);
    return cudaGetLastError();
}

cudaError_t set_field_tables(const TetTables& t) { return cudaMemcpyToSymbol(cTf, &t, sizeof(TetTables)); }

cudaError_t launch_qtets(Ctx& c) {
    RhsArgs a = rargs(c);
    if (c.ncut > 0) k_qcut<<<nb(c.ncut), 256, 0, c.stream>>>(a, c.cut_area, c.qcut);
    if (c.nit > 0) k_qtets<<<nb(c.nit), 256, 0, c.stream>>>(c.nit, c.it_acc, c.qcut, c.qT);
    return cudaGetLastError();
}

// ======================================================================================
// MIXED solve: FP32 PCG inside FP64 iterative refinement.  Each outer step forms
// the FP64 residual r = b - A u (FP64 operator, FP64 norms), solves A d = r in
// FP32 (FP32 vectors and operator, FP64 dot products) to a relative 1e-3, and
// adds d to u in FP64.  The outer test is the FP64 relative residual, so the
// result meets the same ||r|| <= tol ||b|| as the FP64 solve.
// ======================================================================================
constexpr double MIXED_INNER_TOL = 1e-3;
constexpr int MIXED_MAX_OUTER = 12;

__global__ void k_ref_res(FieldArgs f, const double* b, const double* u, double* r64, float* rf, float* uf, float* pf,
                          double* partial, unsigned* ticket, PcgState* S, cudaGraphConditionalHandle h_out,
                          cudaGraphConditionalHandle h_in, long long* outer_total) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[3] = {0, 0, 0};
    if (n < f.m.nnodes) {
        int i, j, k;
        node_ijk(f.m, n, i, j, k);
        double bn = b[n];
        double rn = (f.ntype[n] == -3) ? 0.0 : bn - apply_row<double>(f, n, i, j, k, u, f.coef);
        r64[n] = rn;
        float rfn = (float)rn;
        float zn = f.invdiagf[n] * rfn;
        rf[n] = rfn;
        uf[n] = 0.0f;
        pf[n] = zn;
        v[0] = bn * bn; v[1] = rn * rn; v[2] = (double)rfn * (double)zn;
    }
    double tot[3];
    if (grid_sum<3>(v, partial, ticket, tot) && threadIdx.x == 0) {
        if (S->outer_it == 0) S->bb = tot[0];
        double bb = S->bb;
        S->rr64 = tot[1];
        S->relres = bb > 0.0 ? sqrt(tot[1] / bb) : 0.0;
        bool conv = (bb == 0.0) || (tot[1] <= S->tol2 * bb);
        bool stop = conv || (S->outer_it >= MIXED_MAX_OUTER) || (S->it >= S->maxit);
        S->converged = conv;
        S->done = stop;
        S->rz = tot[2];
        S->inner_bb = tot[1];
        S->inner_it = 0;
        S->done_in = stop;
        S->outer_it = S->outer_it + 1;
        *outer_total += 1;
        cudaGraphSetConditional(h_out, stop ? 0u : 1u);
        cudaGraphSetConditional(h_in, stop ? 0u : 1u);
    }
}

__global__ void k_in_spmv(FieldArgs f, const float* p, float* q, double* partial, unsigned* ticket, PcgState* S,
                          cudaGraphConditionalHandle h_in) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_in, 0u);
    double v[1] = {0.0};
    if (n < f.m.nnodes) {
        int i, j, k;
        node_ijk(f.m, n, i, j, k);
        float y = apply_row<float>(f, n, i, j, k, p, f.coeff);
        q[n] = y;
        v[0] = (double)p[n] * (double)y;
    }
    double tot[1];
    if (grid_sum<1>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->pq = tot[0];
        S->alpha = S->rz / tot[0];
    }
}

__global__ void k_in_update(FieldArgs f, float* u, float* r, const float* p, const float* q, double* partial,
                            unsigned* ticket, PcgState* S, cudaGraphConditionalHandle h_in, long long* it_total) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float alpha = (float)S->alpha;
    double v[2] = {0, 0};
    if (n < f.m.nnodes) {
        float rn = r[n] - alpha * q[n];
        u[n] = u[n] + alpha * p[n];
        r[n] = rn;
        float zn = f.invdiagf[n] * rn;
        v[0] = (double)rn * (double)rn; v[1] = (double)rn * (double)zn;
    }
    double tot[2];
    if (grid_sum<2>(v, partial, ticket, tot) && threadIdx.x == 0) {
        S->beta = tot[1] / S->rz;
        S->rz = tot[1];
        S->inner_it = S->inner_it + 1;
        S->it = S->it + 1;
        *it_total += 1;
        bool stop = (tot[0] <= S->inner_tol2 * S->inner_bb) || (S->it >= S->maxit) || (S->inner_it >= S->inner_max);
        S->done_in = stop;
        if (!stop) cudaGraphSetConditional(h_in, 1u);
    }
}

__global__ void k_in_dir(FieldArgs f, const float* r, float* p, const PcgState* S) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= f.m.nnodes || S->done_in) return;
    p[n] = f.invdiagf[n] * r[n] + (float)S->beta * p[n];
}

__global__ void k_ref_add(long long N, double* u, const float* d) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) u[n] = u[n] + (double)d[n];
}

cudaError_t build_pcg_graph_mixed(Ctx& c) {
    if (c.pcg_exec) { cudaGraphExecDestroy(c.pcg_exec); c.pcg_exec = nullptr; }
    if (c.pcg_graph) { cudaGraphDestroy(c.pcg_graph); c.pcg_graph = nullptr; }
    cudaError_t e;
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g;
    e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return e; }
    long long N = c.mesh.nnodes;
    unsigned gb = nb(N);
    FieldArgs f = fargs(c);
    PcgState* S = pcg_state(c);
    long long* it_total = (long long*)(c.scal + 40);
    long long* outer_total = (long long*)(c.scal + 41);
    cudaStream_t keep = c.stream;
    cudaGraphConditionalHandle h_out, h_in;
    cudaGraphNode_t sink, cond_out, sink_b, cond_in;
    cudaGraphNodeParams po = {}, pi = {};
    cudaGraph_t body_out, body_in;
    e = cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) goto fail;
    c.stream = cs;
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    solve_prefix(c, nullptr);
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) goto fail;
    e = find_sink(g, &sink);
    if (e != cudaSuccess) goto fail;
    po.type = cudaGraphNodeTypeConditional;
    po.conditional.handle = h_out;
    po.conditional.type = cudaGraphCondTypeWhile;
    po.conditional.size = 1;
    e = cudaGraphAddNode(&cond_out, g, &sink, nullptr, 1, &po);
    if (e != cudaSuccess) goto fail;
    body_out = po.conditional.phGraph_out[0];
    e = cudaGraphConditionalHandleCreate(&h_in, body_out, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) goto fail;
    e = cudaStreamBeginCaptureToGraph(cs, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_ref_res<<<gb, 256, 0, cs>>>(f, c.b, c.u, c.r, c.rf, c.uf, c.pf, c.red, c.red_ticket, S, h_out, h_in, outer_total);
    e = cudaStreamEndCapture(cs, &body_out);
    if (e != cudaSuccess) goto fail;
    e = find_sink(body_out, &sink_b);
    if (e != cudaSuccess) goto fail;
    pi.type = cudaGraphNodeTypeConditional;
    pi.conditional.handle = h_in;
    pi.conditional.type = cudaGraphCondTypeWhile;
    pi.conditional.size = 1;
    e = cudaGraphAddNode(&cond_in, body_out, &sink_b, nullptr, 1, &pi);
    if (e != cudaSuccess) goto fail;
    body_in = pi.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_in_spmv<<<gb, 256, 0, cs>>>(f, c.pf, c.qf, c.red, c.red_ticket, S, h_in);
    k_in_update<<<gb, 256, 0, cs>>>(f, c.uf, c.rf, c.pf, c.qf, c.red, c.red_ticket, S, h_in, it_total);
    k_in_dir<<<gb, 256, 0, cs>>>(f, c.rf, c.pf, S);
    e = cudaStreamEndCapture(cs, &body_in);
    if (e != cudaSuccess) goto fail;
    e = cudaStreamBeginCaptureToGraph(cs, body_out, &cond_in, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_ref_add<<<gb, 256, 0, cs>>>(N, c.u, c.uf);
    e = cudaStreamEndCapture(cs, &body_out);
    if (e != cudaSuccess) goto fail;
    e = cudaStreamBeginCaptureToGraph(cs, g, &cond_out, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) goto fail;
    k_phi_from_u<<<gb, 256, 0, cs>>>(N, c.u, c.gdir, c.phi, S);
    k_node_E<<<gb, 256, 0, cs>>>(f, c.Lnode, c.imask, c.ibase, c.it_data, c.qT, c.phi, c.E, c.Ef);
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) goto fail;
    e = cudaGraphInstantiate(&c.pcg_exec, g, 0);
    if (e != cudaSuccess) goto fail;
    c.pcg_graph = g;
    c.stream = keep;
    cudaStreamDestroy(cs);
    return cudaSuccess;
fail:
    c.stream = keep;
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

cudaError_t launch_pcg_mixed(Ctx& c) {
    PcgState h = {};
    h.tol2 = c.tol * c.tol;
    h.maxit = c.maxit;
    h.inner_tol2 = MIXED_INNER_TOL * MIXED_INNER_TOL;
    h.inner_max = c.maxit;
    cudaError_t e = cudaMemcpyAsync(c.scal, &h, sizeof(PcgState), cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return e;
    return cudaGraphLaunch(c.pcg_exec, c.stream);
}

// ======================================================================================
// Field solve that allocates nothing (pifepic_solve_field_noalloc).
//
// Some callers cannot call cudaMalloc once their run is under way: a serving
// loop whose device memory is handed out by a pool it does not own, code that
// runs while a stream is being captured into a CUDA graph, or an embedding
// that forbids allocation after start-up.  pifepic_solve_field allocates a
// staging buffer and builds a CUDA graph on every call, so those callers need
// this variant.  It reuses the context's operator (read only), takes the load
// F, the flux jumps q and the output phi as caller-owned device arrays, and
// keeps every work vector of the PCG in one file-scope device array of fixed
// size, found once per device with cudaGetSymbolAddress.
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
// threads doing the first call on one device at once both store the same value.
static void* g_noalloc_dev[64];
static int g_noalloc_ready[64];

pifepic_status solve_field_noalloc(Ctx& c, const double* F, const double* q, double* phi, int* iters,
                                   double* relres) {
    long long N = c.mesh.nnodes;
    if (N > NOALLOC_MAX_NODES) {
        char b[256];
        snprintf(b, sizeof(b), "solve_field_noalloc: mesh has %lld nodes; the fixed scratch holds at most %lld",
                 N, NOALLOC_MAX_NODES);
        c.err = b;
        return PIFEPIC_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { c.err = "solve_field_noalloc: no device"; return PIFEPIC_ECUDA; }
    if (!g_noalloc_ready[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            c.err = std::string("solve_field_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return PIFEPIC_ECUDA;
        }
        g_noalloc_dev[dev] = ptr;
        g_noalloc_ready[dev] = 1;
    }
    double* base = (double*)g_noalloc_dev[dev];
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
    k_rhs<<<gb, 256, 0, st>>>(f, a, c.imask, c.ibase, c.it_data, q, c.lift, bvec, F);
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
        return PIFEPIC_ECUDA;
    }
    if (iters) *iters = hs.it;
    if (relres) *relres = hs.relres;
    return PIFEPIC_OK;
}

}  // namespace pf
