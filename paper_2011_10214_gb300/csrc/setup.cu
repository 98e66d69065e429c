// S0: interface and stiffness set-up on the GPU (compiled without FMA
// contraction so the node level set and tet classification are reproducible).
//
// Sec. 2.1 (Eqs. 2.1-2.5) poses -div(eps grad phi) = rho with [phi] = 0 and
// [eps d phi/dn] = q on the interface; Sec. 1 / 2.1 describe IFE functions as
// standard linear FE functions adjusted on interface elements to satisfy those
// conditions, with unchanged nodal degrees of freedom; Sec. 3.1.1 cuts each
// cubic PIC cell into 5 tetrahedra.  On each interface tet this file builds
// psi+ = a + b.x, psi- = psi+ + beta d(x) (d the signed distance to the plane
// of the linear interpolant's zero set, beta = ((eps+ - eps-) n.b - q)/eps-),
// fixed by the 4 nodal values through a 4x4 FP64 solve (4 basis functions +
// the unit jump function), its exact sub-volumes, Gamma_h area, element
// stiffness and unit-jump load.  Regular rows of the operator stay matrix-free;
// rows touching an interface tet become explicit 19-slot patch rows.
#include <math.h>

#include "internal.h"

namespace pf {

__constant__ TetTables cT;

cudaError_t set_tet_tables(const TetTables& t) { return cudaMemcpyToSymbol(cT, &t, sizeof(TetTables)); }

static __device__ __forceinline__ void loff(int l, int& a, int& b, int& c) {
    a = l & 1; b = (l >> 1) & 1; c = (l >> 2) & 1;
}

// ---------------------------------------------------------------------------
// node level set on the IFE mesh; the object lives in PIC cell units, so node
// (i, j, k) sits at (i, j, k) / refine (inv_r = 1 / refine, a power of two: exact)
__global__ void k_levelset(Mesh m, Object o, double inv_r, double* L) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    L[n] = level_set(o, (double)i * inv_r, (double)j * inv_r, (double)k * inv_r);
}

// interface tets: cut by the object's surface (also when the bedrock plane
// crosses the same tet: the surface alone then defines it), or inside the
// object and cut by the bedrock plane only; bad counts bedrock nodes outside
// the object
__global__ void k_classify(Mesh m, Object o, const double* L, unsigned char* mask, int* cnt, int* bad) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= m.ncells) return;
    int i = (int)(c % m.nx), j = (int)((c / m.nx) % m.ny), k = (int)(c / ((long long)m.nx * m.ny));
    int p = (i + j + k) & 1;
    bool neg[8], bneg[8];
    for (int l = 0; l < 8; ++l) {
        int a, b, cc; loff(l, a, b, cc);
        neg[l] = L[node_id(m, i + a, j + b, k + cc)] < 0.0;
        bneg[l] = o.bed && bed_level(o, k + cc) < 0.0;
        if (bneg[l] && !neg[l]) atomicAdd(bad, 1);
    }
    unsigned char mk = 0;
    int n = 0;
    for (int t = 0; t < 5; ++t) {
        int nm = 0, nbd = 0;
        for (int v = 0; v < 4; ++v) { nm += neg[cT.vert[p][t][v]]; nbd += bneg[cT.vert[p][t][v]]; }
        if ((nm > 0 && nm < 4) || (nm == 4 && nbd > 0 && nbd < 4)) { mk |= (unsigned char)(1u << t); ++n; }
    }
    mask[c] = mk;
    cnt[c] = n;
}

// ---- small dense helpers ------------------------------------------------------
static __device__ double tet_vol(const double* a, const double* b, const double* c, const double* d) {
    double u[3], v[3], w[3];
    for (int q = 0; q < 3; ++q) { u[q] = b[q] - a[q]; v[q] = c[q] - a[q]; w[q] = d[q] - a[q]; }
    double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                 u[2] * (v[0] * w[1] - v[1] * w[0]);
    return fabs(det) / 6.0;
}
static __device__ double tri_area(const double* a, const double* b, const double* c) {
    double u[3], v[3];
    for (int q = 0; q < 3; ++q) { u[q] = b[q] - a[q]; v[q] = c[q] - a[q]; }
    double x = u[1] * v[2] - u[2] * v[1], y = u[2] * v[0] - u[0] * v[2], z = u[0] * v[1] - u[1] * v[0];
    return 0.5 * sqrt(x * x + y * y + z * z);
}
// Gaussian elimination with partial pivoting: A (n x n) X = R (n x m), in place
template <int N, int M>
static __device__ void gauss_solve(double A[N][N], double R[N][M]) {
    for (int c = 0; c < N; ++c) {
        int piv = c;
        double best = fabs(A[c][c]);
        for (int r = c + 1; r < N; ++r)
            if (fabs(A[r][c]) > best) { best = fabs(A[r][c]); piv = r; }
        if (piv != c) {
            for (int q = 0; q < N; ++q) { double t = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = t; }
            for (int q = 0; q < M; ++q) { double t = R[c][q]; R[c][q] = R[piv][q]; R[piv][q] = t; }
        }
        for (int r = c + 1; r < N; ++r) {
            double f = A[r][c] / A[c][c];
            for (int q = c; q < N; ++q) A[r][q] -= f * A[c][q];
            for (int q = 0; q < M; ++q) R[r][q] -= f * R[c][q];
        }
    }
    for (int r = N - 1; r >= 0; --r) {
        for (int q = 0; q < M; ++q) {
            double s = R[r][q];
            for (int cc = r + 1; cc < N; ++cc) s -= A[r][cc] * R[cc][q];
            R[r][q] = s / A[r][r];
        }
    }
}

// linear IFE local space of one interface tet -> record (layout IT_*)
static __device__ void ife_tet(const double vx[4][3], const double Lv[4], double em, double ep, double V,
                               double* rec) {
    bool minus[4];
    for (int v = 0; v < 4; ++v) minus[v] = Lv[v] < 0.0;
    // gradient of the linear interpolant of L
    double M3[3][3], g3[3][1];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) M3[r][q] = vx[r + 1][q] - vx[0][q];
        g3[r][0] = Lv[r + 1] - Lv[0];
    }
    gauss_solve<3, 1>(M3, g3);
    double gn = sqrt(g3[0][0] * g3[0][0] + g3[1][0] * g3[1][0] + g3[2][0] * g3[2][0]);
    double n[3] = {g3[0][0] / gn, g3[1][0] / gn, g3[2][0] / gn};
    double dist[4];
    for (int v = 0; v < 4; ++v) dist[v] = Lv[v] / gn;
    double kappa = (ep - em) / em;
    double A[4][4], R[4][5];
    for (int v = 0; v < 4; ++v) {
        A[v][0] = 1.0;
        for (int q = 0; q < 3; ++q) A[v][1 + q] = vx[v][q] + (minus[v] ? dist[v] * kappa * n[q] : 0.0);
        for (int f = 0; f < 5; ++f) R[v][f] = (f == v) ? 1.0 : 0.0;
        R[v][4] = minus[v] ? dist[v] / em : 0.0;
    }
    gauss_solve<4, 5>(A, R);       // R now holds (a, b) per function
    double gp[5][3], gm[5][3];
    for (int f = 0; f < 5; ++f) {
        double bn = R[1][f] * n[0] + R[2][f] * n[1] + R[3][f] * n[2];
        double beta = kappa * bn - (f == 4 ? 1.0 / em : 0.0);
        for (int q = 0; q < 3; ++q) { gp[f][q] = R[1 + q][f]; gm[f][q] = R[1 + q][f] + beta * n[q]; }
    }
    // sub-volumes and Gamma_h triangles
    int mi[4], pl[4], nmi = 0, npl = 0;
    for (int v = 0; v < 4; ++v) { if (minus[v]) mi[nmi++] = v; else pl[npl++] = v; }
    double tri[2][3][3];
    int ntri = 0;
    double volm, volp;
    if (nmi == 1 || nmi == 3) {
        bool lone_minus = (nmi == 1);
        int u = lone_minus ? mi[0] : pl[0];
        const int* oth = lone_minus ? pl : mi;
        double fr[3];
        for (int e = 0; e < 3; ++e) {
            int w = oth[e];
            double t;
            if (lone_minus) {
                t = Lv[u] / (Lv[u] - Lv[w]);
                for (int q = 0; q < 3; ++q) tri[0][e][q] = vx[u][q] + t * (vx[w][q] - vx[u][q]);
                fr[e] = t;
            } else {
                t = Lv[w] / (Lv[w] - Lv[u]);
                for (int q = 0; q < 3; ++q) tri[0][e][q] = vx[w][q] + t * (vx[u][q] - vx[w][q]);
                fr[e] = 1.0 - t;
            }
        }
        ntri = 1;
        double vcut = V * fr[0] * fr[1] * fr[2];
        if (lone_minus) { volm = vcut; volp = V - vcut; } else { volp = vcut; volm = V - vcut; }
    } else {
        int a = mi[0], b = mi[1], c = pl[0], d = pl[1];
        double pac[3], pad[3], pbc[3], pbd[3];
        double tac = Lv[a] / (Lv[a] - Lv[c]), tad = Lv[a] / (Lv[a] - Lv[d]);
        double tbc = Lv[b] / (Lv[b] - Lv[c]), tbd = Lv[b] / (Lv[b] - Lv[d]);
        for (int q = 0; q < 3; ++q) {
            pac[q] = vx[a][q] + tac * (vx[c][q] - vx[a][q]);
            pad[q] = vx[a][q] + tad * (vx[d][q] - vx[a][q]);
            pbc[q] = vx[b][q] + tbc * (vx[c][q] - vx[b][q]);
            pbd[q] = vx[b][q] + tbd * (vx[d][q] - vx[b][q]);
        }
        volm = tet_vol(vx[a], pac, pad, pbd) + tet_vol(vx[a], pac, pbc, pbd) + tet_vol(vx[a], vx[b], pbc, pbd);
        volp = V - volm;
        for (int q = 0; q < 3; ++q) {
            tri[0][0][q] = pac[q]; tri[0][1][q] = pad[q]; tri[0][2][q] = pbd[q];
            tri[1][0][q] = pac[q]; tri[1][1][q] = pbd[q]; tri[1][2][q] = pbc[q];
        }
        ntri = 2;
    }
    double area = 0.0, S[5] = {0, 0, 0, 0, 0};
    for (int tr = 0; tr < ntri; ++tr) {
        double ar = tri_area(tri[tr][0], tri[tr][1], tri[tr][2]);
        area += ar;
        double cen[3];
        for (int q = 0; q < 3; ++q) cen[q] = (tri[tr][0][q] + tri[tr][1][q] + tri[tr][2][q]) / 3.0;
        for (int f = 0; f < 5; ++f) S[f] += ar * (R[0][f] + cen[0] * R[1][f] + cen[1] * R[2][f] + cen[2] * R[3][f]);
    }
    rec[IT_VOLP] = volp;
    rec[IT_VOLM] = volm;
    rec[IT_AREA] = area;
    for (int a = 0; a < 4; ++a) {
        for (int b = 0; b < 4; ++b) {
            double dp = gp[a][0] * gp[b][0] + gp[a][1] * gp[b][1] + gp[a][2] * gp[b][2];
            double dm = gm[a][0] * gm[b][0] + gm[a][1] * gm[b][1] + gm[a][2] * gm[b][2];
            rec[IT_K + 4 * a + b] = ep * volp * dp + em * volm * dm;
        }
        double dpj = gp[a][0] * gp[4][0] + gp[a][1] * gp[4][1] + gp[a][2] * gp[4][2];
        double dmj = gm[a][0] * gm[4][0] + gm[a][1] * gm[4][1] + gm[a][2] * gm[4][2];
        rec[IT_C + a] = -S[a] - (ep * volp * dpj + em * volm * dmj);
        rec[IT_S + a] = S[a];
    }
    for (int f = 0; f < 5; ++f)
        for (int q = 0; q < 3; ++q) { rec[IT_GP + 3 * f + q] = gp[f][q]; rec[IT_GM + 3 * f + q] = gm[f][q]; }
    rec[IT_SJ] = S[4];
}

__global__ void k_interface(Mesh m, Object o, const double* L, const unsigned char* mask, const int* ibase,
                            int* it_cell, int* it_t, double* it_data) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= m.ncells) return;
    unsigned mk = mask[c];
    if (!mk) return;
    int i = (int)(c % m.nx), j = (int)((c / m.nx) % m.ny), k = (int)(c / ((long long)m.nx * m.ny));
    int p = (i + j + k) & 1;
    int T = ibase[c];
    for (int t = 0; t < 5; ++t) {
        if (!((mk >> t) & 1)) continue;
        double vx[4][3], Lv[4], Lb[4];
        int nm = 0;
        for (int v = 0; v < 4; ++v) {
            int l = cT.vert[p][t][v];
            int a, b, cc; loff(l, a, b, cc);
            vx[v][0] = a * m.h; vx[v][1] = b * m.h; vx[v][2] = cc * m.h;
            Lv[v] = L[node_id(m, i + a, j + b, k + cc)];
            Lb[v] = o.bed ? bed_level(o, k + cc) : 0.0;
            nm += Lv[v] < 0.0;
        }
        double V = cT.vol[t] * m.h * m.h * m.h;
        double* rec = it_data + (long long)T * IT_STRIDE;
        if (nm > 0 && nm < 4) {      // the object's surface
            ife_tet(vx, Lv, o.eps_minus, o.eps_plus, V, rec);
            rec[IT_KIND] = 0.0;
        } else {                     // the bedrock plane: bedrock on the minus side
            ife_tet(vx, Lb, o.eps_bed, o.eps_minus, V, rec);
            rec[IT_AREA] = 0.0;
            rec[IT_KIND] = 1.0;
        }
        it_cell[T] = (int)c;
        it_t[T] = t;
        ++T;
    }
}

__global__ void k_cell_area(Mesh m, const unsigned char* mask, const int* ibase, const double* it_data,
                            int* cutflag, double* cellarea) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= m.ncells) return;
    unsigned mk = mask[c];
    double a = 0.0;
    int T = ibase[c];
    for (int t = 0; t < 5; ++t)
        if ((mk >> t) & 1) { a += it_data[(long long)T * IT_STRIDE + IT_AREA]; ++T; }
    cellarea[c] = a;
    cutflag[c] = a > 0.0 ? 1 : 0;
}

__global__ void k_cut_list(Mesh m, const int* cutflag, const long long* cutidx, const double* cellarea,
                           int* cut_cell, double* cut_area, int* own) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= m.ncells) return;
    if (cutflag[c]) {
        long long q = cutidx[c];
        cut_cell[q] = (int)c;
        cut_area[q] = cellarea[c];
        own[c] = (int)q;
    } else {
        own[c] = -1;
    }
}

// surface-charge target of a hit cell: its own cut index, else the first cut
// cell among the 26 neighbours ordered by L1 distance then (dz, dy, dx)
__global__ void k_cell_acc(Mesh m, const int* own, int* acc) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= m.ncells) return;
    int v = own[c];
    if (v < 0) {
        int i = (int)(c % m.nx), j = (int)((c / m.nx) % m.ny), k = (int)(c / ((long long)m.nx * m.ny));
        for (int d1 = 1; d1 <= 3 && v < 0; ++d1)
            for (int dz = -1; dz <= 1 && v < 0; ++dz)
                for (int dy = -1; dy <= 1 && v < 0; ++dy)
                    for (int dx = -1; dx <= 1 && v < 0; ++dx) {
                        if (abs(dx) + abs(dy) + abs(dz) != d1) continue;
                        int ii = i + dx, jj = j + dy, kk = k + dz;
                        if (ii < 0 || ii >= m.nx || jj < 0 || jj >= m.ny || kk < 0 || kk >= m.nz) continue;
                        v = own[cell_id(m, ii, jj, kk)];
                    }
    }
    acc[c] = v;
}

// cut-cell accumulator of each interface tet (-1 on the bedrock plane)
__global__ void k_it_acc(long long nit, const int* it_cell, const double* it_data, const int* own, int* it_acc) {
    long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (T >= nit) return;
    it_acc[T] = it_data[T * IT_STRIDE + IT_KIND] != 0.0 ? -1 : own[it_cell[T]];
}

// node kinds: Dirichlet (-3), touching an interface tet or in the bedrock
// (patch, flag 1), regular plus (-1) or minus (-2)
__global__ void k_node_kind(Mesh m, Object o, const double* L, const unsigned char* mask, const int* bcdir,
                            const double* bcval, int* ntype, int* patchflag, double* gdir) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    int face_on[6] = {i == 0, i == m.nx, j == 0, j == m.ny, k == 0, k == m.nz};
    int dface = -1;
    for (int f = 0; f < 6; ++f)
        if (face_on[f] && bcdir[f]) { dface = f; break; }
    patchflag[n] = 0;
    if (dface >= 0) { ntype[n] = -3; gdir[n] = bcval[dface]; return; }
    gdir[n] = 0.0;
    bool touch = o.bed && bed_level(o, k) < 0.0;
    for (int c8 = 0; c8 < 8 && !touch; ++c8) {
        int a, b, cc; loff(c8, a, b, cc);
        int ci = i - a, cj = j - b, ck = k - cc;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
        unsigned mk = mask[cell_id(m, ci, cj, ck)];
        if (!mk) continue;
        int p = (ci + cj + ck) & 1;
        for (int t = 0; t < 5; ++t) {
            if (!((mk >> t) & 1)) continue;
            for (int v = 0; v < 4; ++v)
                if (cT.vert[p][t][v] == c8) touch = true;
        }
    }
    if (touch) { patchflag[n] = 1; ntype[n] = 0; }
    else ntype[n] = (L[n] < 0.0) ? -2 : -1;
}

__global__ void k_patch_rows(Mesh m, Object o, const double* L, const unsigned char* mask, const int* ibase,
                             const double* it_data, const int* patchflag, const long long* patchidx,
                             int* ntype, long long* patch_node, double* coef, float* coeff, double* invdiag) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes || !patchflag[n]) return;
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    long long r = patchidx[n];
    ntype[n] = (int)r;
    patch_node[r] = n;
    double row[19];
    for (int s = 0; s < 19; ++s) row[s] = 0.0;
    for (int c8 = 0; c8 < 8; ++c8) {
        int a, b, cc; loff(c8, a, b, cc);
        int ci = i - a, cj = j - b, ck = k - cc;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
        long long cell = cell_id(m, ci, cj, ck);
        unsigned mk = mask[cell];
        int p = (ci + cj + ck) & 1;
        int T = ibase[cell];
        for (int t = 0; t < 5; ++t) {
            bool itet = (mk >> t) & 1;
            int kk = -1;
            for (int v = 0; v < 4; ++v)
                if (cT.vert[p][t][v] == c8) kk = v;
            if (kk >= 0) {
                double e[4];
                if (itet) {
                    const double* rec = it_data + (long long)T * IT_STRIDE;
                    for (int v = 0; v < 4; ++v) e[v] = rec[IT_K + 4 * kk + v];
                } else {
                    // a regular tet: the region of its first vertex
                    int l0 = cT.vert[p][t][0];
                    int a0, b0, c0; loff(l0, a0, b0, c0);
                    double eps = L[node_id(m, ci + a0, cj + b0, ck + c0)] < 0.0
                                     ? ((o.bed && bed_level(o, ck + c0) < 0.0) ? o.eps_bed : o.eps_minus)
                                     : o.eps_plus;
                    double s = eps * m.h * cT.vol[t];
                    for (int v = 0; v < 4; ++v)
                        e[v] = s * (cT.grad[p][t][kk][0] * cT.grad[p][t][v][0] +
                                     cT.grad[p][t][kk][1] * cT.grad[p][t][v][1] +
                                     cT.grad[p][t][kk][2] * cT.grad[p][t][v][2]);
                }
                for (int v = 0; v < 4; ++v) {
                    int l = cT.vert[p][t][v];
                    int av, bv, cv; loff(l, av, bv, cv);
                    int dx = av - a, dy = bv - b, dz = cv - cc;
                    int sl = cT.slot[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
                    row[sl] += e[v];
                }
            }
            if (itet) ++T;
        }
    }
    for (int s = 0; s < 19; ++s) { coef[r * 19 + s] = row[s]; coeff[r * 19 + s] = (float)row[s]; }
    invdiag[n] = 1.0 / row[0];
}

__global__ void k_invdiag_regular(Mesh m, Object o, const int* ntype, double* invdiag, float* invdiagf) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    int ty = ntype[n];
    if (ty >= 0) { invdiagf[n] = (float)invdiag[n]; return; }
    if (ty == -3) { invdiag[n] = 0.0; invdiagf[n] = 0.0f; return; }
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    int cx = (i > 0) + (i < m.nx), cy = (j > 0) + (j < m.ny), cz = (k > 0) + (k < m.nz);
    double eps = (ty == -2) ? o.eps_minus : o.eps_plus;
    double d = eps * (double)(cx * cy * cz) * (((i + j + k) & 1) ? 0.5 : 0.75) * m.h;
    invdiag[n] = 1.0 / d;
    invdiagf[n] = (float)(1.0 / d);
}

// ---------------------------------------------------------------------------
// exclusive scan of int flags -> long long offsets (two-level, deterministic)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

__global__ void k_scan_tiles(const int* in, long long n, long long* out, long long* tile_sum) {
    __shared__ long long sh[SCAN_T];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_I;
    long long v[SCAN_I], s = 0;
    for (int q = 0; q < SCAN_I; ++q) { v[q] = (base + q < n) ? in[base + q] : 0; s += v[q]; }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        long long t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    long long run = sh[threadIdx.x] - s;
    for (int q = 0; q < SCAN_I; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == SCAN_T - 1) tile_sum[blockIdx.x] = sh[SCAN_T - 1];
}

__global__ void k_scan_sums(long long* tile_sum, long long ntiles, long long* total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    for (long long t = 0; t < ntiles; ++t) { long long v = tile_sum[t]; tile_sum[t] = run; run += v; }
    *total = run;
}

__global__ void k_scan_add(long long* out, long long n, const long long* tile_sum) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) out[e] += tile_sum[e / SCAN_TILE];
}

static cudaError_t exclusive_scan(const int* in, long long n, long long* out, long long* total_dev,
                                  cudaStream_t st) {
    long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    long long* ts = nullptr;
    cudaError_t e = lib_malloc(&ts, sizeof(long long) * (ntiles > 0 ? ntiles : 1));
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_scan_tiles<<<(unsigned)ntiles, SCAN_T, 0, st>>>(in, n, out, ts);
        k_scan_sums<<<1, 32, 0, st>>>(ts, ntiles, total_dev);
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, ts);
    } else {
        cudaMemsetAsync(total_dev, 0, sizeof(long long), st);
    }
    e = cudaStreamSynchronize(st);
    lib_free(ts);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

__global__ void k_narrow(const long long* in, long long n, int* out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) out[e] = (int)in[e];
}

// ---------------------------------------------------------------------------
// photoelectron emission set-up (Sec. 5.2.2: generated at the sunlit surface by
// the local sunlight index).  Per interface tet: the Gamma_h triangles in cell
// units, the normal from the P1 gradient of the nodal level set, the sunlight
// index, a ray-marched shadow test from the Gamma_h centroid, and the
// fixed-point rate per step.  Operation order follows the definition exactly
// (this unit is compiled without FMA contraction).
// ---------------------------------------------------------------------------
constexpr double PHOTO_RAY_STEP = 0.25;

static __device__ void photo_cut(const double (&V)[4][3], const double (&Lv)[4], int u, int w, double (&out)[3]) {
    const double t = Lv[u] / (Lv[u] - Lv[w]);
    for (int d = 0; d < 3; ++d) out[d] = V[u][d] + t * (V[w][d] - V[u][d]);
}

static __device__ double photo_tri_area(const double (&P)[3][3]) {
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) { e1[d] = P[1][d] - P[0][d]; e2[d] = P[2][d] - P[0][d]; }
    const double c0 = e1[1] * e2[2] - e1[2] * e2[1], c1 = e1[2] * e2[0] - e1[0] * e2[2], c2 = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * sqrt((c0 * c0 + c1 * c1) + c2 * c2);
}

__global__ void k_photo_setup(Mesh m, Object obj, double inv_r, long long nit, const int* it_cell, const int* it_t,
                              const double* Lnode, const int* it_acc, double sx, double sy, double sz, double J,
                              double h2, double dt, double w, PhotoDev* rec, long long* Qall) {
    const long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (T >= nit) return;
    Qall[T] = 0;
    const int c = it_cell[T];
    const int ci = c % m.nx, cj = (c / m.nx) % m.ny, ck = c / (m.nx * m.ny);
    const int p = (ci + cj + ck) & 1, t = it_t[T];
    double V[4][3], Lv[4];
    for (int v = 0; v < 4; ++v) {
        const int l = cT.vert[p][t][v];
        V[v][0] = (double)(l & 1); V[v][1] = (double)((l >> 1) & 1); V[v][2] = (double)((l >> 2) & 1);
        Lv[v] = Lnode[node_id(m, ci + (l & 1), cj + ((l >> 1) & 1), ck + ((l >> 2) & 1))];
    }
    double g[3];
    for (int d = 0; d < 3; ++d) g[d] = Lv[0] * cT.grad[p][t][0][d];
    for (int v = 1; v < 4; ++v)
        for (int d = 0; d < 3; ++d) g[d] = g[d] + Lv[v] * cT.grad[p][t][v][d];
    const double gn = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
    double n[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
    const double S = fmax(0.0, (n[0] * sx + n[1] * sy) + n[2] * sz);
    if (!(S > 0.0) || it_acc[T] < 0) return;
    // Gamma_h triangles (cube-local), same cut and triangulation as the IFE set-up
    int mi[4], pl[4], nm = 0, np = 0;
    for (int v = 0; v < 4; ++v) {
        if (Lv[v] < 0.0) mi[nm++] = v;
        else pl[np++] = v;
    }
    PhotoDev d;
    double P[2][3][3];
    int ntri = 1;
    if (nm == 1) {
        for (int k = 0; k < 3; ++k) photo_cut(V, Lv, mi[0], pl[k], P[0][k]);
    } else if (nm == 3) {
        for (int k = 0; k < 3; ++k) photo_cut(V, Lv, mi[k], pl[0], P[0][k]);
    } else if (nm == 2) {
        double pac[3], pad[3], pbc[3], pbd[3];
        photo_cut(V, Lv, mi[0], pl[0], pac);
        photo_cut(V, Lv, mi[0], pl[1], pad);
        photo_cut(V, Lv, mi[1], pl[0], pbc);
        photo_cut(V, Lv, mi[1], pl[1], pbd);
        for (int e = 0; e < 3; ++e) {
            P[0][0][e] = pac[e]; P[0][1][e] = pad[e]; P[0][2][e] = pbd[e];
            P[1][0][e] = pac[e]; P[1][1][e] = pbd[e]; P[1][2][e] = pbc[e];
        }
        ntri = 2;
    } else {
        return;
    }
    const double base[3] = {(double)ci, (double)cj, (double)ck};
    for (int q = 0; q < ntri; ++q)
        for (int k = 0; k < 3; ++k)
            for (int e = 0; e < 3; ++e) P[q][k][e] = P[q][k][e] + base[e];
    const double a0 = photo_tri_area(P[0]);
    const double a1 = ntri > 1 ? photo_tri_area(P[1]) : 0.0;
    const double A = a0 + a1;
    if (!(A > 0.0)) return;
    double cen[3];
    for (int e = 0; e < 3; ++e) cen[e] = (a0 / 3.0) * ((P[0][0][e] + P[0][1][e]) + P[0][2][e]);
    if (ntri > 1)
        for (int e = 0; e < 3; ++e) cen[e] = cen[e] + (a1 / 3.0) * ((P[1][0][e] + P[1][1][e]) + P[1][2][e]);
    for (int e = 0; e < 3; ++e) cen[e] = cen[e] / A;
    // shadow: the ray towards the sun, sampled every quarter cell inside the box
    const long long kmax = 4ll * (m.nx + m.ny + m.nz) + 8;
    for (long long k = 1; k <= kmax; ++k) {
        const double tt = PHOTO_RAY_STEP * (double)k;
        const double qx = cen[0] + tt * sx, qy = cen[1] + tt * sy, qz = cen[2] + tt * sz;
        if (qx < 0.0 || qx > (double)m.nx || qy < 0.0 || qy > (double)m.ny || qz < 0.0 || qz > (double)m.nz) break;
        if (level_set(obj, qx * inv_r, qy * inv_r, qz * inv_r) < 0.0) return;   // the object in PIC units
    }
    const double R = J * S * (A * h2) * dt / w;
    const long long Q = (long long)rint(R * (double)(1ll << PHOTO_RATE_BITS));
    if (Q <= 0) return;
    // tangent basis: e = the axis least aligned with n (first on ties)
    const double an[3] = {fabs(n[0]), fabs(n[1]), fabs(n[2])};
    int ax = 0;
    if (an[1] < an[ax]) ax = 1;
    if (an[2] < an[ax]) ax = 2;
    const double ev[3] = {ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, ax == 2 ? 1.0 : 0.0};
    double cr[3] = {n[1] * ev[2] - n[2] * ev[1], n[2] * ev[0] - n[0] * ev[2], n[0] * ev[1] - n[1] * ev[0]};
    const double cl = sqrt((cr[0] * cr[0] + cr[1] * cr[1]) + cr[2] * cr[2]);
    for (int e = 0; e < 3; ++e) { d.n[e] = n[e]; d.t1[e] = cr[e] / cl; }
    d.t2[0] = n[1] * d.t1[2] - n[2] * d.t1[1];
    d.t2[1] = n[2] * d.t1[0] - n[0] * d.t1[2];
    d.t2[2] = n[0] * d.t1[1] - n[1] * d.t1[0];
    for (int q = 0; q < 2; ++q)
        for (int k = 0; k < 3; ++k)
            for (int e = 0; e < 3; ++e) d.P[q][k][e] = q < ntri ? P[q][k][e] : 0.0;
    d.area0 = a0;
    d.A = A;
    d.ntri = ntri;
    d.acc = it_acc[T];
    rec[T] = d;
    Qall[T] = Q;
}

__global__ void k_photo_flag(long long nit, const long long* Qall, int* flag) {
    const long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (T < nit) flag[T] = Qall[T] > 0 ? 1 : 0;
}

__global__ void k_photo_compact(long long nit, const long long* Qall, const PhotoDev* rec, const long long* pos,
                                PhotoDev* tets, long long* Q) {
    const long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (T >= nit || Qall[T] <= 0) return;
    tets[pos[T]] = rec[T];
    Q[pos[T]] = Qall[T];
}

#define CK(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { err = _e; goto done; } } while (0)

cudaError_t launch_setup(Ctx& c) {
    cudaError_t err = cudaSuccess;
    Mesh m = c.mesh;
    cudaStream_t st = c.stream;
    int* cnt = nullptr; long long* scan = nullptr; long long* tot = nullptr;
    int* flag = nullptr; double* carea = nullptr; int* own = nullptr;
    int* bcdir = nullptr; double* bcval = nullptr;
    int* bad = nullptr;
    long long hv = 0;
    long long nit_alloc = 1;
    long long nmax = m.nnodes > m.ncells ? m.nnodes : m.ncells;
    int hdir[6]; double hval[6];
    CK(lib_malloc(&cnt, sizeof(int) * nmax));
    CK(lib_malloc(&scan, sizeof(long long) * nmax));
    CK(lib_malloc(&tot, sizeof(long long)));
    CK(lib_malloc(&flag, sizeof(int) * m.ncells));
    CK(lib_malloc(&carea, sizeof(double) * m.ncells));
    CK(lib_malloc(&own, sizeof(int) * m.ncells));
    CK(lib_malloc(&bcdir, sizeof(int) * 6));
    CK(lib_malloc(&bcval, sizeof(double) * 6));
    CK(lib_malloc(&bad, sizeof(int)));

    c.bed_outside = false;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_levelset<<<nb(m.nnodes), 256, 0, st>>>(m, c.obj, 1.0 / (double)c.refine, c.Lnode);
    k_classify<<<nb(m.ncells), 256, 0, st>>>(m, c.obj, c.Lnode, c.imask, cnt, bad);
    CK(cudaGetLastError());
    {
        int hbad = 0;
        CK(scopy(st, &hbad, bad, sizeof(int), cudaMemcpyDeviceToHost));
        if (hbad) { c.bed_outside = true; err = cudaErrorInvalidValue; goto done; }
    }
    // interface-tet offsets per cell
    CK(exclusive_scan(cnt, m.ncells, scan, tot, st));
    CK(scopy(st, &hv, tot, sizeof(long long), cudaMemcpyDeviceToHost));
    c.nit = hv;
    k_narrow<<<nb(m.ncells), 256, 0, st>>>(scan, m.ncells, c.ibase);
    nit_alloc = c.nit > 0 ? c.nit : 1;
    CK(lib_malloc(&c.it_cell, sizeof(int) * nit_alloc));
    CK(lib_malloc(&c.it_t, sizeof(int) * nit_alloc));
    CK(lib_malloc(&c.it_data, sizeof(double) * IT_STRIDE * nit_alloc));
    CK(lib_malloc(&c.it_acc, sizeof(int) * nit_alloc));
    CK(lib_malloc(&c.qT, sizeof(double) * nit_alloc));
    CK(cudaMemsetAsync(c.qT, 0, sizeof(double) * nit_alloc, st));
    k_interface<<<nb(m.ncells), 256, 0, st>>>(m, c.obj, c.Lnode, c.imask, c.ibase, c.it_cell, c.it_t, c.it_data);
    k_cell_area<<<nb(m.ncells), 256, 0, st>>>(m, c.imask, c.ibase, c.it_data, flag, carea);
    CK(cudaGetLastError());
    CK(exclusive_scan(flag, m.ncells, scan, tot, st));
    CK(scopy(st, &hv, tot, sizeof(long long), cudaMemcpyDeviceToHost));
    c.ncut = hv;
    {
        long long nc;
        nc = c.ncut > 0 ? c.ncut : 1;
        CK(lib_malloc(&c.cut_cell, sizeof(int) * nc));
        CK(lib_malloc(&c.cut_area, sizeof(double) * nc));
        CK(lib_malloc(&c.qcut, sizeof(double) * nc));
        CK(cudaMemsetAsync(c.qcut, 0, sizeof(double) * nc, st));
    }
    k_cut_list<<<nb(m.ncells), 256, 0, st>>>(m, flag, scan, carea, c.cut_cell, c.cut_area, own);
    k_cell_acc<<<nb(m.ncells), 256, 0, st>>>(m, own, c.cell_acc);
    if (c.nit > 0) k_it_acc<<<nb(c.nit), 256, 0, st>>>(c.nit, c.it_cell, c.it_data, own, c.it_acc);
    CK(cudaGetLastError());
    // nodes
    for (int f = 0; f < 6; ++f) { hdir[f] = c.bc[f].kind == PIFEPIC_BC_DIRICHLET; hval[f] = c.bc[f].value; }
    CK(scopy(st, bcdir, hdir, sizeof(hdir), cudaMemcpyHostToDevice));
    CK(scopy(st, bcval, hval, sizeof(hval), cudaMemcpyHostToDevice));
    k_node_kind<<<nb(m.nnodes), 256, 0, st>>>(m, c.obj, c.Lnode, c.imask, bcdir, bcval, c.ntype, cnt, c.gdir);
    CK(cudaGetLastError());
    CK(exclusive_scan(cnt, m.nnodes, scan, tot, st));
    CK(scopy(st, &hv, tot, sizeof(long long), cudaMemcpyDeviceToHost));
    c.npatch = hv;
    {
        long long np;
        np = c.npatch > 0 ? c.npatch : 1;
        CK(lib_malloc(&c.patch_node, sizeof(long long) * np));
        CK(lib_malloc(&c.patch_coef, sizeof(double) * 19 * np));
        CK(lib_malloc(&c.patch_coeff, sizeof(float) * 19 * np));
    }
    k_patch_rows<<<nb(m.nnodes), 256, 0, st>>>(m, c.obj, c.Lnode, c.imask, c.ibase, c.it_data, cnt, scan,
                                               c.ntype, c.patch_node, c.patch_coef, c.patch_coeff, c.invdiag);
    k_invdiag_regular<<<nb(m.nnodes), 256, 0, st>>>(m, c.obj, c.ntype, c.invdiag, c.invdiagf);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
done:
    lib_free(cnt); lib_free(scan); lib_free(tot); lib_free(flag); lib_free(carea); lib_free(own);
    lib_free(bcdir); lib_free(bcval); lib_free(bad);
    return err;
}

// ---------------------------------------------------------------------------
// Node rows (once per set-up).  The node field is minus the volume-weighted
// mean of the element gradients around a node, plasma-side pieces preferred
// (the reading of Sec. 2.1 that k_node_E follows); on a fixed mesh and object
// that is a linear map of the potential at the node's 27 neighbours and of q_T
// on the interface tets containing the node.  A node that is not interior-
// regular (a cube absent, or a cube holding an interface tet) gets a row: those
// 27 x 3 coefficients in FP32 and its interface tets {T, 3 FP32 coefficients};
// the same tet list, with each tet's unit-jump load at the node in FP64, is
// the right-hand side's flux-jump term of the node (in the order the cubes and
// tets are visited, so the sums are those of visiting the cubes).
// ---------------------------------------------------------------------------
__global__ void k_node_rows_count(Mesh m, const unsigned char* mask, int* need, int* nq) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    bool irregular = i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz;
    int q = 0;
    for (int c8 = 0; c8 < 8; ++c8) {
        int a, b, cc; loff(c8, a, b, cc);
        int ci = i - a, cj = j - b, ck = k - cc;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
        unsigned mk = mask[cell_id(m, ci, cj, ck)];
        if (!mk) continue;
        irregular = true;
        int p = (ci + cj + ck) & 1;
        for (int t = 0; t < 5; ++t) {
            if (!((mk >> t) & 1)) continue;
            for (int v = 0; v < 4; ++v)
                if (cT.vert[p][t][v] == c8) ++q;
        }
    }
    need[n] = irregular ? 1 : 0;
    nq[n] = q;
}

constexpr int NR_T = 64;   // threads per block of the row fill (a 27 x 3 FP64 accumulator each in shared memory)

// visits the tets containing node (i, j, k): f(tet T or -1, cube parity p, tet t, the node's vertex index kk, cube
// corner (ci, cj, ck), cube corner offset (a, b, cc) of the node)
template <typename F>
static __device__ __forceinline__ void for_node_tets(const Mesh& m, int i, int j, int k, const unsigned char* mask,
                                                     const int* ibase, F f) {
    for (int c8 = 0; c8 < 8; ++c8) {
        int a, b, cc; loff(c8, a, b, cc);
        int ci = i - a, cj = j - b, ck = k - cc;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= m.nx || cj >= m.ny || ck >= m.nz) continue;
        long long cell = cell_id(m, ci, cj, ck);
        unsigned mk = mask[cell];
        int p = (ci + cj + ck) & 1;
        int T = ibase[cell];
        for (int t = 0; t < 5; ++t) {
            bool itet = (mk >> t) & 1;
            int kk = -1;
            for (int v = 0; v < 4; ++v)
                if (cT.vert[p][t][v] == c8) kk = v;
            if (kk >= 0) f(itet ? T : -1, p, t, kk, ci, cj, ck, a, b, cc);
            if (itet) ++T;
        }
    }
}

__global__ void __launch_bounds__(NR_T) k_node_rows_fill(Mesh m, const unsigned char* mask, const int* ibase,
                                                         const double* it_data, const double* L, const int* need,
                                                         const long long* rowscan, const long long* qscan,
                                                         long long R, int* row, float* coef, int* qoff, int4* qent,
                                                         double* qc) {
    __shared__ double acc[NR_T][81];
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= m.nnodes) return;
    if (!need[n]) { row[n] = -1; return; }
    int i = (int)(n % m.NX), j = (int)((n / m.NX) % m.NY), k = (int)(n / ((long long)m.NX * m.NY));
    const long long r = rowscan[n], q0 = qscan[n];
    row[n] = (int)r;
    qoff[r] = (int)q0;
    const double ih = 1.0 / m.h, V3 = m.h * m.h * m.h;
    // a piece is plasma: the + piece of a surface tet with volume, or a regular tet whose first vertex is outside
    // the object
    double vpl = 0.0, val = 0.0;
    for_node_tets(m, i, j, k, mask, ibase, [&](int T, int p, int t, int, int ci, int cj, int ck, int, int, int) {
        if (T >= 0) {
            const double* rec = it_data + (long long)T * IT_STRIDE;
            if (rec[IT_VOLP] > 0.0 && rec[IT_KIND] == 0.0) vpl += rec[IT_VOLP];
            val += rec[IT_VOLP] + rec[IT_VOLM];
        } else {
            int a0, b0, c0; loff(cT.vert[p][t][0], a0, b0, c0);
            const double V = cT.vol[t] * V3;
            if (L[node_id(m, ci + a0, cj + b0, ck + c0)] >= 0.0) vpl += V;
            val += V;
        }
    });
    // the plasma pieces alone where there are some, else every piece
    const bool pl_only = vpl > 0.0;
    const double vol = pl_only ? vpl : val;
    double* A = acc[threadIdx.x];
    for (int q = 0; q < 81; ++q) A[q] = 0.0;
    long long e = q0;
    for_node_tets(m, i, j, k, mask, ibase,
                  [&](int T, int p, int t, int kk, int ci, int cj, int ck, int a, int b, int cc) {
        int nbv[4];
        for (int v = 0; v < 4; ++v) {
            int av, bv, cv; loff(cT.vert[p][t][v], av, bv, cv);
            nbv[v] = (av - a + 1) + 3 * (bv - b + 1) + 9 * (cv - cc + 1);
        }
        if (T >= 0) {
            const double* rec = it_data + (long long)T * IT_STRIDE;
            const double vp = rec[IT_VOLP], vm = rec[IT_VOLM];
            const bool plus = vp > 0.0 && rec[IT_KIND] == 0.0;
            const double wp = pl_only ? (plus ? vp : 0.0) : vp, wm = pl_only ? 0.0 : vm;
            for (int v = 0; v < 4; ++v)
                for (int d = 0; d < 3; ++d)
                    A[nbv[v] * 3 + d] += wp * rec[IT_GP + 3 * v + d] + wm * rec[IT_GM + 3 * v + d];
            float cq[3];
            for (int d = 0; d < 3; ++d)
                cq[d] = (float)(-(wp * rec[IT_GP + 12 + d] + wm * rec[IT_GM + 12 + d]) / vol);
            qent[e] = make_int4(T, __float_as_int(cq[0]), __float_as_int(cq[1]), __float_as_int(cq[2]));
            qc[e] = rec[IT_C + kk];
            ++e;
        } else {
            int a0, b0, c0; loff(cT.vert[p][t][0], a0, b0, c0);
            const bool plus = L[node_id(m, ci + a0, cj + b0, ck + c0)] >= 0.0;
            const double w = (pl_only && !plus) ? 0.0 : cT.vol[t] * V3 * ih;
            for (int v = 0; v < 4; ++v)
                for (int d = 0; d < 3; ++d) A[nbv[v] * 3 + d] += w * cT.grad[p][t][v][d];
        }
    });
    for (int q = 0; q < 81; ++q) coef[(long long)q * R + r] = (float)(-A[q] / vol);
}

cudaError_t launch_node_rows(Ctx& c) {
    const Mesh& m = c.mesh;
    const long long N = m.nnodes;
    void* old[] = {c.ne_row, c.ne_coef, c.ne_qoff, c.ne_q, c.ne_qc};
    for (void* p : old) lib_free(p);
    c.ne_row = nullptr; c.ne_coef = nullptr; c.ne_qoff = nullptr; c.ne_q = nullptr; c.ne_qc = nullptr;
    c.ne_nrows = 0;
    cudaStream_t st = c.stream;
    int *need = nullptr, *nq = nullptr;
    long long *rowscan = nullptr, *qscan = nullptr, *tot = nullptr;
    long long R = 0, Q = 0;
    cudaError_t err = cudaSuccess;
    CK(lib_malloc(&need, sizeof(int) * N));
    CK(lib_malloc(&nq, sizeof(int) * N));
    CK(lib_malloc(&rowscan, sizeof(long long) * N));
    CK(lib_malloc(&qscan, sizeof(long long) * N));
    CK(lib_malloc(&tot, sizeof(long long)));
    k_node_rows_count<<<nb(N), 256, 0, st>>>(m, c.imask, need, nq);
    CK(cudaGetLastError());
    CK(exclusive_scan(need, N, rowscan, tot, st));
    CK(scopy(st, &R, tot, sizeof(long long), cudaMemcpyDeviceToHost));
    CK(exclusive_scan(nq, N, qscan, tot, st));
    CK(scopy(st, &Q, tot, sizeof(long long), cudaMemcpyDeviceToHost));
    {
        const long long r1 = R > 0 ? R : 1, q1 = Q > 0 ? Q : 1;
        int qend = (int)Q;
        CK(lib_malloc(&c.ne_row, sizeof(int) * N));
        CK(lib_malloc(&c.ne_coef, sizeof(float) * 81 * r1));
        CK(lib_malloc(&c.ne_qoff, sizeof(int) * (r1 + 1)));
        CK(lib_malloc(&c.ne_q, sizeof(int4) * q1));
        CK(lib_malloc(&c.ne_qc, sizeof(double) * q1));
        c.ne_nrows = R;
        k_node_rows_fill<<<(unsigned)((N + NR_T - 1) / NR_T), NR_T, 0, st>>>(
            m, c.imask, c.ibase, c.it_data, c.Lnode, need, rowscan, qscan, R, c.ne_row, c.ne_coef, c.ne_qoff, c.ne_q,
            c.ne_qc);
        CK(cudaGetLastError());
        CK(scopy(st, c.ne_qoff + R, &qend, sizeof(int), cudaMemcpyHostToDevice));
    }
done:
    lib_free(need); lib_free(nq); lib_free(rowscan); lib_free(qscan); lib_free(tot);
    return err;
}

// emission set-up for the context's photo species (all buffers (re)allocated
// here, outside any captured graph)
cudaError_t launch_photo_setup(Ctx& c, const double* sun, double density, double vth, double w) {
    void* old[] = {c.ph_tets, c.ph_Q, c.ph_carry, c.ph_cnt, c.ph_base, c.ph_tiles, c.ph_total};
    for (void* p : old) lib_free(p);
    c.ph_tets = nullptr; c.ph_Q = c.ph_carry = c.ph_base = c.ph_tiles = c.ph_total = nullptr; c.ph_cnt = nullptr;
    c.ph_ne = 0;
    const long long nit = c.nit;
    const double sl = sqrt((sun[0] * sun[0] + sun[1] * sun[1]) + sun[2] * sun[2]);
    const double s0 = sun[0] / sl, s1 = sun[1] / sl, s2 = sun[2] / sl;
    const double J = density * vth / sqrt(2.0 * 3.141592653589793);
    PhotoDev* rec = nullptr;
    long long *Qall = nullptr, *pos = nullptr, *tot = nullptr;
    int* flag = nullptr;
    cudaError_t err = cudaSuccess;
    long long ne = 0;
    const long long n1 = nit > 0 ? nit : 1;
    CK(lib_malloc(&rec, sizeof(PhotoDev) * n1));
    CK(lib_malloc(&Qall, sizeof(long long) * n1));
    CK(lib_malloc(&pos, sizeof(long long) * n1));
    CK(lib_malloc(&flag, sizeof(int) * n1));
    CK(lib_malloc(&tot, sizeof(long long)));
    CK(cudaMemsetAsync(Qall, 0, sizeof(long long) * n1, c.stream));
    CK(cudaMemsetAsync(rec, 0, sizeof(PhotoDev) * n1, c.stream));
    if (nit > 0) {
        k_photo_setup<<<nb(nit), 256, 0, c.stream>>>(c.mesh, c.obj, 1.0 / (double)c.refine, nit, c.it_cell, c.it_t,
                                                     c.Lnode, c.it_acc, s0, s1,
                                                     s2, J, c.mesh.h * c.mesh.h, c.dt, w, rec, Qall);
        k_photo_flag<<<nb(nit), 256, 0, c.stream>>>(nit, Qall, flag);
        CK(cudaGetLastError());
        CK(exclusive_scan(flag, nit, pos, tot, c.stream));
        CK(cudaMemcpyAsync(&ne, tot, sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    {
        const long long m1 = ne > 0 ? ne : 1;
        CK(lib_malloc(&c.ph_tets, sizeof(PhotoDev) * m1));
        CK(lib_malloc(&c.ph_Q, sizeof(long long) * m1));
        CK(lib_malloc(&c.ph_carry, sizeof(long long) * m1));
        CK(lib_malloc(&c.ph_cnt, sizeof(int) * m1));
        CK(lib_malloc(&c.ph_base, sizeof(long long) * m1));
        CK(lib_malloc(&c.ph_tiles, sizeof(long long) * (m1 / 2048 + 2)));
        CK(lib_malloc(&c.ph_total, sizeof(long long)));
        CK(cudaMemsetAsync(c.ph_carry, 0, sizeof(long long) * m1, c.stream));
        CK(cudaMemsetAsync(c.ph_total, 0, sizeof(long long), c.stream));
        if (ne > 0) k_photo_compact<<<nb(nit), 256, 0, c.stream>>>(nit, Qall, rec, pos, c.ph_tets, c.ph_Q);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c.stream));
        c.ph_ne = ne;
        c.ph_vth = vth;
    }
done:
    lib_free(rec); lib_free(Qall); lib_free(pos); lib_free(flag); lib_free(tot);
    return err;
}

}  // namespace pf
