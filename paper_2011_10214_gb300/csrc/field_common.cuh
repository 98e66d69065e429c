// Shared by the field-solve translation units: PCG scalar state, the operator
// arguments, the matrix-free row of the IFE operator (regular 7/19-point rows of
// the 5-tet P1 stencil, explicit 19-slot rows where a node touches an interface
// tet) and deterministic block / grid reductions.
#pragma once
#include "internal.h"

namespace pf {

struct PcgState {
    double bb, rz, rr, pq, alpha, beta, tol2, relres;
    int it, maxit, done, converged;
    // mixed mode (FP32 inner PCG inside FP64 refinement): refinement steps of
    // the last solve; an inner solve stops at max(margin2 tol2 bb, inner_red2 rr0)
    int outer_it;
    double inner_red2, margin2;
};
// the state shares the context's scalar block with other slots from double 16 on
static_assert(sizeof(PcgState) <= 16 * sizeof(double), "PcgState overlaps the scalar slots");

// h/6 and h/12 of the regular stencil in the working precision
template <typename T>
static __device__ __forceinline__ T h_over6(const Mesh& m) { return sizeof(T) == 8 ? (T)m.h6 : (T)m.h6f; }
template <typename T>
static __device__ __forceinline__ T h_over12(const Mesh& m) { return sizeof(T) == 8 ? (T)m.h12 : (T)m.h12f; }

struct FieldArgs {
    Mesh m;
    Object o;
    const int* ntype;
    const double* coef;       // patch rows [npatch][19]
    const float* coeff;
    const double* invdiag;
    const float* invdiagf;
};

// one instance of a batched solve (batch.cu, pcg_cluster.cu)
struct BatchItem {
    FieldArgs f;
    const double* b;
    double* u;
    double *r, *z, *p, *q;
    float *rf, *zf, *pf, *qf, *df;
    const double* g;
    double* phi;
    PcgState* S;
    long long* it_total;
    long long* outer_total;
    double tol2;
    double inner_red2, margin2;   // MIXED inner stop (as in PcgState)
    int maxit;
};

static __device__ __forceinline__ void loff(int l, int& a, int& b, int& c) {
    a = l & 1; b = (l >> 1) & 1; c = (l >> 2) & 1;
}

// load of a vector entry; CG = true reads through L2 only (bypassing L1), as a
// persistent kernel must for entries other blocks wrote since its last barrier
template <bool CG, typename T>
static __device__ __forceinline__ T ldx(const T* x, long long i) {
    if constexpr (CG) return __ldcg(x + i);
    else return x[i];
}

// y_n = (A x)_n for the IFE operator, the node's type ty (ntype) given;
// Dirichlet rows give 0 (x is 0 there).  ld(m) returns x_m (from global
// memory or from a shared-memory window).
template <typename T, typename LD>
static __device__ __forceinline__ T apply_row_ty(const FieldArgs& f, long long n, int i, int j, int k, int ty, LD ld,
                                                 const T* coef) {
    const Mesh& m = f.m;
    if (ty == -3) return (T)0;
    const long long sx = 1, sy = m.NX, sz = (long long)m.NX * m.NY;
    bool xm = i > 0, xp = i < m.nx, ym = j > 0, yp = j < m.ny, zm = k > 0, zp = k < m.nz;
    if (ty >= 0) {
        const T* c = coef + (long long)ty * 19;
        T y = c[0] * ld(n);
        if (xm) y += c[1] * ld(n - sx);
        if (xp) y += c[2] * ld(n + sx);
        if (ym) y += c[3] * ld(n - sy);
        if (yp) y += c[4] * ld(n + sy);
        if (zm) y += c[5] * ld(n - sz);
        if (zp) y += c[6] * ld(n + sz);
        if ((i + j + k) & 1) return y;
        if (xm && ym) y += c[7] * ld(n - sx - sy);
        if (xp && ym) y += c[8] * ld(n + sx - sy);
        if (xm && yp) y += c[9] * ld(n - sx + sy);
        if (xp && yp) y += c[10] * ld(n + sx + sy);
        if (xm && zm) y += c[11] * ld(n - sx - sz);
        if (xp && zm) y += c[12] * ld(n + sx - sz);
        if (xm && zp) y += c[13] * ld(n - sx + sz);
        if (xp && zp) y += c[14] * ld(n + sx + sz);
        if (ym && zm) y += c[15] * ld(n - sy - sz);
        if (yp && zm) y += c[16] * ld(n + sy - sz);
        if (ym && zp) y += c[17] * ld(n - sy + sz);
        if (yp && zp) y += c[18] * ld(n + sy + sz);
        return y;
    }
    // regular row: assembled P1 stencil of the 5-tet split with eps of the region;
    // each coefficient = (cubes sharing the edge) x (per-cube element integral)
    T eps = (T)(ty == -2 ? f.o.eps_minus : f.o.eps_plus);
    T h = (T)m.h;
    int cx = (int)xm + (int)xp, cy = (int)ym + (int)yp, cz = (int)zm + (int)zp;
    bool odd = (i + j + k) & 1;
    T y = (T)(cx * cy * cz) * (odd ? (T)0.5 : (T)0.75) * h * ld(n);
    T ax = (T)0, ay = (T)0, az = (T)0;
    if (xm) ax += ld(n - sx);
    if (xp) ax += ld(n + sx);
    if (ym) ay += ld(n - sy);
    if (yp) ay += ld(n + sy);
    if (zm) az += ld(n - sz);
    if (zp) az += ld(n + sz);
    const T h6 = h_over6<T>(m);
    y -= h6 * ((T)(cy * cz) * ax + (T)(cx * cz) * ay + (T)(cx * cy) * az);
    if (!odd) {
        T dxy = (T)0, dxz = (T)0, dyz = (T)0;
        if (xm && ym) dxy += ld(n - sx - sy);
        if (xp && ym) dxy += ld(n + sx - sy);
        if (xm && yp) dxy += ld(n - sx + sy);
        if (xp && yp) dxy += ld(n + sx + sy);
        if (xm && zm) dxz += ld(n - sx - sz);
        if (xp && zm) dxz += ld(n + sx - sz);
        if (xm && zp) dxz += ld(n - sx + sz);
        if (xp && zp) dxz += ld(n + sx + sz);
        if (ym && zm) dyz += ld(n - sy - sz);
        if (yp && zm) dyz += ld(n + sy - sz);
        if (ym && zp) dyz += ld(n - sy + sz);
        if (yp && zp) dyz += ld(n + sy + sz);
        const T h12 = h_over12<T>(m);
        y -= h12 * ((T)cz * dxy + (T)cy * dxz + (T)cx * dyz);
    }
    return eps * y;
}

// the same with the node's type read from ntype
template <typename T, typename LD>
static __device__ __forceinline__ T apply_row_ld(const FieldArgs& f, long long n, int i, int j, int k, LD ld,
                                                 const T* coef) {
    return apply_row_ty<T>(f, n, i, j, k, f.ntype[n], ld, coef);
}

// (A x)_n in FP64 for the refinement residual: a regular row with all six
// neighbours present (no interface tet, not Dirichlet) takes the interior
// closed form of apply_row_ld's regular branch -- eps [(4 or 6) h x_n - 4 h/6
// (six face neighbours) - (even nodes) 2 h/12 (twelve edge neighbours)], the
// same sums in the same order, without the per-node integer weights and their
// conversions (FP64 issues slowly on this part); any other row goes through
// apply_row_ld
template <typename LD>
static __device__ __forceinline__ double apply_row64(const FieldArgs& f, long long n, int i, int j, int k, LD ld,
                                                     const double* coef) {
    const Mesh& m = f.m;
    const int ty = f.ntype[n];
    if (ty >= 0 || ty == -3 || i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz)
        return apply_row_ld<double>(f, n, i, j, k, ld, coef);
    const long long sx = 1, sy = m.NX, sz = (long long)m.NX * m.NY;
    const double eps = ty == -2 ? f.o.eps_minus : f.o.eps_plus;
    const bool odd = (i + j + k) & 1;
    double y = (odd ? 4.0 : 6.0) * m.h * ld(n);
    const double ax = ld(n - sx) + ld(n + sx), ay = ld(n - sy) + ld(n + sy), az = ld(n - sz) + ld(n + sz);
    y -= (4.0 * m.h6) * ((ax + ay) + az);
    if (!odd) {
        const double dxy = ((ld(n - sx - sy) + ld(n + sx - sy)) + ld(n - sx + sy)) + ld(n + sx + sy);
        const double dxz = ((ld(n - sx - sz) + ld(n + sx - sz)) + ld(n - sx + sz)) + ld(n + sx + sz);
        const double dyz = ((ld(n - sy - sz) + ld(n + sy - sz)) + ld(n - sy + sz)) + ld(n + sy + sz);
        y -= (2.0 * m.h12) * ((dxy + dxz) + dyz);
    }
    return eps * y;
}

// Row kinds for the masked regular stencil: the six neighbour-presence flags,
// the node parity, the region, and whether the row is general (an interface
// patch row) or Dirichlet (zero).
enum : unsigned short {
    RK_XM = 1, RK_XP = 2, RK_YM = 4, RK_YP = 8, RK_ZM = 16, RK_ZP = 32, RK_ODD = 64, RK_INNER = 128,
    RK_GENERAL = 256, RK_DIRICHLET = 512
};

static __device__ __forceinline__ unsigned short row_kind(const FieldArgs& f, long long n, int i, int j, int k) {
    const Mesh& m = f.m;
    const int ty = f.ntype[n];
    if (ty == -3) return RK_DIRICHLET;
    if (ty >= 0) return RK_GENERAL;
    unsigned short kd = 0;
    if (i > 0) kd |= RK_XM;
    if (i < m.nx) kd |= RK_XP;
    if (j > 0) kd |= RK_YM;
    if (j < m.ny) kd |= RK_YP;
    if (k > 0) kd |= RK_ZM;
    if (k < m.nz) kd |= RK_ZP;
    if ((i + j + k) & 1) kd |= RK_ODD;
    if (ty == -2) kd |= RK_INNER;
    return kd;
}

// A regular row (kind without RK_GENERAL / RK_DIRICHLET) of the operator of
// apply_row_ld, branch-free: absent neighbours are read (any finite value) and
// multiplied by zero.  ld(o) returns x at offset o from the node; NX, NXY are
// the strides.  Same closed form as the regular branch of apply_row_ld
// (summation order differs).
template <typename T, typename LD>
static __device__ __forceinline__ T regular_row_masked_ld(LD ld, int NX, int NXY, unsigned kd, T h, T h6, T h12,
                                                          T eps_plus, T eps_minus) {
    const T mxm = (kd & RK_XM) ? (T)1 : (T)0, mxp = (kd & RK_XP) ? (T)1 : (T)0;
    const T mym = (kd & RK_YM) ? (T)1 : (T)0, myp = (kd & RK_YP) ? (T)1 : (T)0;
    const T mzm = (kd & RK_ZM) ? (T)1 : (T)0, mzp = (kd & RK_ZP) ? (T)1 : (T)0;
    const bool odd = kd & RK_ODD;
    const T eps = (kd & RK_INNER) ? eps_minus : eps_plus;
    const T cx = mxm + mxp, cy = mym + myp, cz = mzm + mzp;
    const T ax = mxm * ld(-1) + mxp * ld(1);
    const T ay = mym * ld(-NX) + myp * ld(NX);
    const T az = mzm * ld(-NXY) + mzp * ld(NXY);
    T y = cx * cy * cz * (odd ? (T)0.5 : (T)0.75) * h * ld(0);
    y -= h6 * (cy * cz * ax + cx * cz * ay + cx * cy * az);
    if (!odd) {
        const T dxy = (mxm * mym) * ld(-1 - NX) + (mxp * mym) * ld(1 - NX) + (mxm * myp) * ld(-1 + NX) +
                      (mxp * myp) * ld(1 + NX);
        const T dxz = (mxm * mzm) * ld(-1 - NXY) + (mxp * mzm) * ld(1 - NXY) + (mxm * mzp) * ld(-1 + NXY) +
                      (mxp * mzp) * ld(1 + NXY);
        const T dyz = (mym * mzm) * ld(-NX - NXY) + (myp * mzm) * ld(NX - NXY) + (mym * mzp) * ld(-NX + NXY) +
                      (myp * mzp) * ld(NX + NXY);
        y -= h12 * (cz * dxy + cy * dxz + cx * dyz);
    }
    return eps * y;
}

// the same row over a window in shared memory; wc points at the node's entry
template <typename T>
static __device__ __forceinline__ T regular_row_masked(const T* wc, int NX, int NXY, unsigned kd, T h, T h6, T h12,
                                                       T eps_plus, T eps_minus) {
    return regular_row_masked_ld<T>([&](int o) { return wc[o]; }, NX, NXY, kd, h, h6, h12, eps_plus, eps_minus);
}

// The 19 coefficients of row n of the same operator, in the slot order of
// apply_row_ld (centre, -x, +x, -y, +y, -z, +z, then -x-y, +x-y, -x+y, +x+y,
// -x-z, +x-z, -x+z, +x+z, -y-z, +y-z, -y+z, +y+z); slots apply_row_ld skips
// (a neighbour outside the mesh, a diagonal of an odd node, a Dirichlet row)
// are zero.
template <typename T>
static __device__ __forceinline__ void row_coeffs(const FieldArgs& f, long long n, int i, int j, int k,
                                                  const T* coef, T (&c)[19]) {
    const Mesh& m = f.m;
#pragma unroll
    for (int q = 0; q < 19; ++q) c[q] = (T)0;
    const int ty = f.ntype[n];
    if (ty == -3) return;
    const bool xm = i > 0, xp = i < m.nx, ym = j > 0, yp = j < m.ny, zm = k > 0, zp = k < m.nz;
    const bool odd = (i + j + k) & 1;
    const bool has[19] = {true, xm, xp, ym, yp, zm, zp, xm && ym, xp && ym, xm && yp, xp && yp,
                          xm && zm, xp && zm, xm && zp, xp && zp, ym && zm, yp && zm, ym && zp, yp && zp};
    if (ty >= 0) {
        const T* r = coef + (long long)ty * 19;
#pragma unroll
        for (int q = 0; q < 19; ++q)
            if (has[q] && (q < 7 || !odd)) c[q] = r[q];
        return;
    }
    const T eps = (T)(ty == -2 ? f.o.eps_minus : f.o.eps_plus);
    const T h = (T)m.h;
    const int cx = (int)xm + (int)xp, cy = (int)ym + (int)yp, cz = (int)zm + (int)zp;
    c[0] = eps * ((T)(cx * cy * cz) * (odd ? (T)0.5 : (T)0.75) * h);
    const T a6 = eps * h_over6<T>(m);
    const T ax = -a6 * (T)(cy * cz), ay = -a6 * (T)(cx * cz), az = -a6 * (T)(cx * cy);
    const T axis[6] = {ax, ax, ay, ay, az, az};
#pragma unroll
    for (int q = 1; q < 7; ++q) c[q] = has[q] ? axis[q - 1] : (T)0;
    if (odd) return;
    const T a12 = eps * h_over12<T>(m);
    const T dxy = -a12 * (T)cz, dxz = -a12 * (T)cy, dyz = -a12 * (T)cx;
#pragma unroll
    for (int q = 7; q < 19; ++q) c[q] = has[q] ? (q < 11 ? dxy : q < 15 ? dxz : dyz) : (T)0;
}

template <typename T, bool CG = false>
static __device__ __forceinline__ T apply_row(const FieldArgs& f, long long n, int i, int j, int k, const T* x,
                                              const T* coef) {
    return apply_row_ld<T>(f, n, i, j, k, [&](long long m) { return ldx<CG>(x, m); }, coef);
}

static __device__ __forceinline__ void node_ijk(const Mesh& m, long long n, int& i, int& j, int& k) {
    // node counts stay below 2^31 (mesh limits 2047 x 2047 x 1023 cells): 32-bit division
    unsigned u = (unsigned)n, NX = (unsigned)m.NX, NXY = (unsigned)m.NX * (unsigned)m.NY;
    unsigned kk = u / NXY, rem = u - kk * NXY;
    unsigned jj = rem / NX;
    i = (int)(rem - jj * NX);
    j = (int)jj;
    k = (int)kk;
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

// deterministic block sum of NV values of type A (thread 0 gets the totals);
// A = float keeps the MIXED inner loop off the FP64 pipe, which issues a warp
// instruction only every few dozen cycles on this part
template <typename A, int NV>
static __device__ __forceinline__ void block_sum_t(A (&v)[NV], A* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        A s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[q * 32 + w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            A s = lane < nw ? sh[q * 32 + lane] : (A)0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[q] = s;
        }
    }
    __syncthreads();
}

static __device__ __forceinline__ unsigned long long atom_add_release(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
static __device__ __forceinline__ void red_add_release(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ void red_add_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// writes block partials; returns true in the one block that arrives last,
// which then holds the grid totals in tot[]
template <int NV>
static __device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partial, unsigned* ticket, double (&tot)[NV]) {
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

}  // namespace pf
