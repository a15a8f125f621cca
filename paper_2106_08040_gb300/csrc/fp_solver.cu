// Batched Fokker-Planck solver for Neel rotation (Sec. 2.1, Eq. FP-general,
// Eq. convection, Eq. mean_magmom_FP) on sm_103a.
//
// One CTA owns one instance at a time (persistent loop over instances).  The
// real-SH coefficient vector c (N = (L+1)^2 doubles), every Radau stage and
// the FP32 factors live in shared memory; nothing is streamed from HBM per
// step except the L1/L2-resident coupling tables shared by all instances.
//
// Time step: S-stage Radau IIA (S = 3: order 5, S = 5: order 9; L-stable),
// simplified Newton:
//   residual   R_i = -Z_i + h sum_j a_ij A(t + c_j h)(y + Z_j)         FP64
//   correction (Lam - h_f Abar) dW = K R,  dZ = T dW (h_f / h)          FP32
// Abar = A(t_f + h_f) is frozen over several steps.  Lam - h_f Abar splits into
// one real and (S-1)/2 complex systems, each block-tridiagonal in |m|; every
// system is factorised (block Thomas) into explicit FP32 inverses of its
// Schur-complement diagonal blocks, one warp per system (Gauss-Jordan with
// partial pivoting in registers), and solved by one warp per system.
// Embedded error estimate filtered through the real factor; steps land on
// every output sample time.
#include <cuda_runtime.h>
#include <stdint.h>
#include "fp_internal.h"

#define NT 256
#define NWARP (NT / 32)
#define FULLMASK 0xffffffffu

__constant__ FpRadau c_radau[2];      // [0]: 3 stages, [1]: 5 stages
template <int S> __device__ __forceinline__ const FpRadau& RAD() { return c_radau[S == 5 ? 1 : 0]; }
__constant__ double c_glx[FP_NGL];
__constant__ double c_glw[FP_NGL];

struct KArgs {
    DevTab tab;
    DevBlk blk;
    fp_material mat;
    fp_drive drv;
    fp_tol tol;
    const fp_instance* inst;
    int n;
    double* m_out;
    double* dmdt_out;
    int* status;
    int* stats;
    int S_out;
    int L_launch;
};

// slot -> scalar group: W, ZR, RZ, RX, RY, GZ, GX, GY
__host__ __device__ constexpr int grp_of(int k) {
    return k < 2 ? 0 : k < 4 ? 1 : k < 5 ? 2 : k < 7 ? 3 : k < 9 ? 4 : k < 11 ? 5 : k < 15 ? 6 : 7;
}

struct AScal { double s[8]; };

// ---------------------------------------------------------------- layout ----
__host__ __device__ inline int nblk(int mu, int L) { return mu == 0 ? L + 1 : 2 * (L + 1 - mu); }
// column stride of a stored inverse block: odd, so the lanes of a column-split matvec hit distinct banks
__host__ __device__ inline int ldb(int n) { return n | 1; }
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Layout {
    int N, L, nmax;
    size_t y, Z, F, f0, yb, diag, rr, zr, rc, zc, dnv, upv, fr, fc, Xr, Xc, ic, total;
    size_t fsum;
};

template <int S>
__host__ __device__ inline Layout make_layout(int L) {
    constexpr int NC = (S - 1) / 2;
    Layout ly;
    ly.L = L;
    ly.N = (L + 1) * (L + 1);
    ly.nmax = (2 * L > L + 1) ? 2 * L : L + 1;
    size_t fsum = 0;
    for (int mu = 0; mu <= L; ++mu) fsum += (size_t)nblk(mu, L) * ldb(nblk(mu, L));
    ly.fsum = fsum;
    const size_t N = ly.N, nm2 = (size_t)ly.nmax * ly.nmax;
    size_t o = 0;
    ly.y = o;    o = al16(o + N * 8);
    ly.Z = o;    o = al16(o + (size_t)S * N * 8);
    ly.F = o;    o = al16(o + (size_t)S * N * 8);
    ly.f0 = o;   o = al16(o + N * 8);
    ly.yb = o;   o = al16(o + (size_t)S * N * 8);
    ly.diag = o; o = al16(o + N * 8);
    ly.rr = o;   o = al16(o + N * 4);
    ly.zr = o;   o = al16(o + N * 4);
    ly.rc = o;   o = al16(o + (size_t)NC * N * 8);
    ly.zc = o;   o = al16(o + (size_t)NC * N * 8);
    ly.dnv = o;  o = al16(o + N * FP_NLT * 4);
    ly.upv = o;  o = al16(o + N * FP_NLT * 4);
    ly.fr = o;   o = al16(o + fsum * 4);
    ly.fc = o;   o = al16(o + (size_t)NC * fsum * 8);
    ly.Xr = o;   o = al16(o + nm2 * 4);
    ly.Xc = o;   o = al16(o + (size_t)NC * nm2 * 8);
    ly.ic = ly.fr;                                     // initial-state scratch aliases the factors
    size_t ic_end = ly.ic + (size_t)FP_NGL * (L + 1) * 8;
    ly.total = o > ic_end ? o : al16(ic_end);
    return ly;
}

size_t fp_solver_smem_bytes(int stages, int L) {
    return stages == 5 ? make_layout<5>(L).total : make_layout<3>(L).total;
}

// --------------------------------------------------- scalar/complex ops ----
__device__ __forceinline__ float cabs1(float a) { return fabsf(a); }
__device__ __forceinline__ float cabs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ float cmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float cfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma(float a, float2 b, float2 c) { return make_float2(fmaf(a, b.x, c.x), fmaf(a, b.y, c.y)); }
__device__ __forceinline__ float crecip(float a) { return 1.f / a; }
__device__ __forceinline__ float2 crecip(float2 a) {
    float d = 1.f / (a.x * a.x + a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ float cneg(float a) { return -a; }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float cshfl(float a, int p) { return __shfl_sync(FULLMASK, a, p); }
__device__ __forceinline__ float2 cshfl(float2 a, int p) {
    return make_float2(__shfl_sync(FULLMASK, a.x, p), __shfl_sync(FULLMASK, a.y, p));
}
__device__ __forceinline__ float cshfl_xor(float a, int o) { return __shfl_xor_sync(FULLMASK, a, o); }
__device__ __forceinline__ float2 cshfl_xor(float2 a, int o) {
    return make_float2(__shfl_xor_sync(FULLMASK, a.x, o), __shfl_xor_sync(FULLMASK, a.y, o));
}
__device__ __forceinline__ float cadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float cadd_real(float a, float v) { return a + v; }
__device__ __forceinline__ float2 cadd_real(float2 a, float v) { return make_float2(a.x + v, a.y); }
template <class T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ float czero<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// ------------------------------------------------------------- helpers ----
// max that keeps NaN visible (fmaxf drops it): a NaN input yields +inf
__device__ __forceinline__ float nanmax(float a, float b) { return (b != b || a != a) ? __int_as_float(0x7f800000) : fmaxf(a, b); }

__device__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(FULLMASK, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = red[0];
    for (int i = 1; i < NWARP; ++i) r = nanmax(r, red[i]);
    return r;
}

__device__ void field_nframe(const KArgs& A, const double* R, const double* off, double t, double* B) {
    const double twopi = 6.283185307179586476925286766559;
    double bl[3];
    for (int k = 0; k < 3; ++k)
        bl[k] = off[k] + A.drv.amp[k] * sin(twopi * A.drv.freq[k] * t + A.drv.phase[k]);
    for (int r = 0; r < 3; ++r) B[r] = R[3 * r] * bl[0] + R[3 * r + 1] * bl[1] + R[3 * r + 2] * bl[2];
}

__device__ __forceinline__ AScal make_scal(const FpParams& P, const double* B) {
    AScal s;
    s.s[0] = -0.5 * P.p4;
    s.s[1] = -P.p3;
    s.s[2] = -P.p1 * B[2];
    s.s[3] = -P.p1 * B[0];
    s.s[4] = -P.p1 * B[1];
    s.s[5] = -P.p2 * B[2];
    s.s[6] = -P.p2 * B[0];
    s.s[7] = -P.p2 * B[1];
    return s;
}

// row i of A x (FP64, matrix-free from the closed-form tables)
__device__ __forceinline__ double apply_row(int i, const double* __restrict__ x, const AScal& sc,
                                            const double* __restrict__ diag, int N, const DevTab& T) {
    const double* cf = T.coef + (size_t)i * FP_NSLOT;
    const int* sr = T.src + (size_t)i * FP_NSLOT;
    double g[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = 0.0;
#pragma unroll
    for (int k = 0; k < FP_NSLOT; ++k) {
        int j = __ldg(sr + k);
        double v = ((unsigned)j < (unsigned)N) ? x[j] : 0.0;
        g[grp_of(k)] = fma(__ldg(cf + k), v, g[grp_of(k)]);
    }
    double acc = diag[i] * x[i];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc = fma(sc.s[q], g[q], acc);
    return acc;
}

__device__ void apply_A(const double* __restrict__ x, double* __restrict__ y, const AScal& sc,
                        const double* __restrict__ diag, int N, const DevTab& T) {
    for (int i = threadIdx.x; i < N; i += NT) y[i] = apply_row(i, x, sc, diag, N, T);
}

// ------------------------------------------------------- per-CTA state ----
template <int S>
struct Ctx {
    Layout ly;
    int L, N;
    double *y, *Z, *F, *f0, *yb, *diag;
    float *rr, *zr;
    float2 *rc, *zc;
    float *dnv, *upv;
    float* fr;
    float2* fc;
    float* Xr;
    float2* Xc;
    int* boff;
    int* foff;
    // block structure of degree L
    const int* glob;
    const uint8_t *sb_k, *sb_g, *dn_k, *dn_g, *up_k, *up_g, *dnT;
    const float *sb_cf, *dn_cf, *up_cf;
};

// ------------------------------------------- factorisation (block Thomas) --
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// A group of GW warps assembles the Schur-complement block
// D~_mu = D_mu - C_mu X_{mu-1} of one system (lane = row, warp gw owns the
// columns [gw*CPW, gw*CPW + CPW)) and inverts it in place by Gauss-Jordan with
// partial pivoting: the warp owning pivot column k picks the pivot row and
// publishes the column multipliers through shared memory, one named barrier
// per pivot.  The inverse is stored column-major (out[c * n + r] = Inv[r][c]).
// n <= 32.
template <class T, int S, int GW>
__device__ void group_factor_block(Ctx<S>& C, int mu, T shift, const float* gs, float h, const T* Xprev, T* out,
                                   int* pp, T* colbuf, int gw, int barid) {
    constexpr int CPW = 32 / GW;
    const int lane = threadIdx.x & 31;
    const int L = C.L, n = nblk(mu, L), bo = C.boff[mu];
    const int j0 = gw * CPW;
    T a[CPW];
    if (lane < n) {
        const int b = bo + lane;
        const int g = __ldg(C.glob + b);
        const T dv = cadd_real(shift, (float)(-(double)h * C.diag[g]));
        int ks[FP_NSB];
        float vs[FP_NSB];
#pragma unroll
        for (int p = 0; p < FP_NSB; ++p) {
            ks[p] = __ldg(C.sb_k + b * FP_NSB + p);
            vs[p] = ks[p] == 255 ? 0.f : gs[__ldg(C.sb_g + b * FP_NSB + p)] * __ldg(C.sb_cf + b * FP_NSB + p);
        }
        int kd[FP_NLT];
        float vd[FP_NLT];
#pragma unroll
        for (int p = 0; p < FP_NLT; ++p) {
            kd[p] = mu > 0 ? __ldg(C.dn_k + b * FP_NLT + p) : 255;
            vd[p] = kd[p] == 255 ? 0.f : C.dnv[b * FP_NLT + p];
        }
#pragma unroll
        for (int jj = 0; jj < CPW; ++jj) {
            const int j = j0 + jj;
            T v = j == lane ? dv : czero<T>();
            if (j < n) {
#pragma unroll
                for (int p = 0; p < FP_NSB; ++p) v = cadd_real(v, ks[p] == j ? vs[p] : 0.f);
#pragma unroll
                for (int p = 0; p < FP_NLT; ++p)
                    if (kd[p] != 255) v = cfma(-vd[p], Xprev[kd[p] * n + j], v);
            }
            a[jj] = v;
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < CPW; ++jj) a[jj] = cadd_real(czero<T>(), j0 + jj == lane ? 1.f : 0.f);
    }
    bool used = lane >= n;
    int myk = -1;
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        const int owner = k / CPW, kk = k - owner * CPW;
        T* cb = colbuf + (k & 1) * 32;
        if (gw == owner) {
            T ak = a[0];
#pragma unroll
            for (int jj = 1; jj < CPW; ++jj) ak = jj == kk ? a[jj] : ak;
            const float v = used ? 0.f : cabs1(ak);
            unsigned key = (__float_as_uint(v) & ~31u) | (unsigned)lane;
            key = __reduce_max_sync(FULLMASK, key);
            const int p = (int)(key & 31u);
            const T pinv = crecip(cshfl(ak, p));
            cb[lane] = lane == p ? pinv : cneg(cmul(ak, pinv));
            if (lane == 0) pp[k] = p;
        }
        named_bar(barid, 32 * GW);
        const int p = pp[k];
        const T mlt = cb[lane];                 // pinv on the pivot row, -a_ik / a_pk elsewhere
        const bool ispiv = lane == p;
#pragma unroll
        for (int jj = 0; jj < CPW; ++jj) {
            const T prj = cshfl(a[jj], p);
            const T upd = ispiv ? cmul(prj, mlt) : cfma(mlt, prj, a[jj]);
            a[jj] = (j0 + jj == k) ? mlt : upd;
        }
        if (ispiv) { used = true; myk = k; }
    }
    if (lane < n && myk >= 0) {
#pragma unroll
        for (int jj = 0; jj < CPW; ++jj) {
            const int j = j0 + jj;
            if (j < n) {
                const int pj = pp[j];
                if (pj < n) out[pj * ldb(n) + myk] = a[jj];  // pj >= n only for a singular block
            }
        }
    }
}

// X_mu = Inv_mu B_mu (n x n2, row-major) for one system; one warp per column c
// (lane = row r).  B_mu[k][c] is the coupling of row k (block mu) to row c
// (block mu+1), reached through the dn list of row c and its back pointer.
template <class T, int S>
__device__ __forceinline__ void x_column(Ctx<S>& C, int mu, int c, const T* inv, T* X) {
    const int lane = threadIdx.x & 31;
    const int L = C.L, n = nblk(mu, L), n2 = nblk(mu + 1, L);
    const int bc = C.boff[mu + 1] + c, bo = C.boff[mu];
    T acc = czero<T>();
#pragma unroll
    for (int p = 0; p < FP_NLT; ++p) {
        const int k = __ldg(C.dn_k + bc * FP_NLT + p);
        if (k == 255) continue;
        const int q = __ldg(C.dnT + bc * FP_NLT + p);
        const float bv = q == 255 ? 0.f : C.upv[(bo + k) * FP_NLT + q];
        if (lane < n) acc = cfma(bv, inv[k * ldb(n) + lane], acc);
    }
    if (lane < n) X[lane * n2 + c] = acc;
}

template <int S> struct Groups {
    static constexpr int NC = (S - 1) / 2;
    static constexpr int NSYS = 1 + NC;
    static constexpr int GW = NWARP / NSYS >= 4 ? 4 : (NWARP / NSYS >= 2 ? 2 : 1);   // warps per system
};

template <int S>
__device__ void factorize(Ctx<S>& C, const AScal& sc, double h, int* pp, float2* colbuf) {
    constexpr int NC = Groups<S>::NC;
    constexpr int NSYS = Groups<S>::NSYS;
    constexpr int GW = Groups<S>::GW;
    const int L = C.L, N = C.N;
    float gs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) gs[q] = (float)(-h * sc.s[q]);
    for (int e = threadIdx.x; e < N * FP_NLT; e += NT) {
        int kd = __ldg(C.dn_k + e), ku = __ldg(C.up_k + e);
        C.dnv[e] = kd == 255 ? 0.f : gs[__ldg(C.dn_g + e)] * __ldg(C.dn_cf + e);
        C.upv[e] = ku == 255 ? 0.f : gs[__ldg(C.up_g + e)] * __ldg(C.up_cf + e);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int sys = w / GW, gw = w - sys * GW;
    const size_t nm2 = (size_t)C.ly.nmax * C.ly.nmax;
    for (int mu = 0; mu <= L; ++mu) {
        if (sys == 0) {
            group_factor_block<float, S, GW>(C, mu, (float)RAD<S>().gam, gs, (float)h, C.Xr, C.fr + C.foff[mu],
                                             pp, (float*)colbuf, gw, 1);
        } else if (sys <= NC) {
            const int q = sys - 1;
            const float2 shift = make_float2((float)RAD<S>().alp[q], -(float)RAD<S>().bet[q]);
            group_factor_block<float2, S, GW>(C, mu, shift, gs, (float)h, C.Xc + q * nm2,
                                              C.fc + (size_t)q * C.ly.fsum + C.foff[mu], pp + 32 * sys,
                                              colbuf + 64 * sys, gw, 1 + sys);
        }
        __syncthreads();
        if (mu < L) {
            const int n2 = nblk(mu + 1, L);
            for (int item = w; item < NSYS * n2; item += NWARP) {
                const int sy = item / n2, c = item - sy * n2;
                if (sy == 0) x_column<float, S>(C, mu, c, C.fr + C.foff[mu], C.Xr);
                else x_column<float2, S>(C, mu, c, C.fc + (size_t)(sy - 1) * C.ly.fsum + C.foff[mu],
                                         C.Xc + (sy - 1) * nm2);
            }
            __syncthreads();
        }
    }
}

// ----------------------------------------------------- warp-group solve --
// Block-Thomas solve of one system with its explicit block inverses by a group
// of GW warps: row r of a block is handled by GW lanes (r = gw*RPW + lane%RPW,
// part = lane/RPW) that split the matvec columns and reduce with shuffles.
// rhs (block order) is overwritten; the solution ends in z.
template <class T, int S, int GW>
__device__ void group_solve(Ctx<S>& C, const T* __restrict__ inv, T* rhs, T* z, int gw, int barid) {
    constexpr int RPW = 32 / GW;
    const int lane = threadIdx.x & 31;
    const int rl = lane % RPW, part = lane / RPW, r = gw * RPW + rl;
    const int L = C.L;
    for (int mu = 0; mu <= L; ++mu) {
        const int n = nblk(mu, L), ld = ldb(n), bo = C.boff[mu], fo = C.foff[mu];
        if (mu > 0 && part == 0 && r < n) {
            const int b = bo + r, bp = C.boff[mu - 1];
            T v = rhs[b];
#pragma unroll
            for (int p = 0; p < FP_NLT; ++p) {
                const int k = __ldg(C.dn_k + b * FP_NLT + p);
                if (k != 255) v = cfma(-C.dnv[b * FP_NLT + p], z[bp + k], v);
            }
            rhs[b] = v;
        }
        named_bar(barid, 32 * GW);
        T acc = czero<T>();
        if (r < n) {
#pragma unroll 4
            for (int c = part; c < n; c += GW) acc = cfma(inv[fo + c * ld + r], rhs[bo + c], acc);
        }
#pragma unroll
        for (int o = RPW; o < 32; o <<= 1) acc = cadd(acc, cshfl_xor(acc, o));
        if (part == 0 && r < n) z[bo + r] = acc;
        named_bar(barid, 32 * GW);
    }
    for (int mu = L - 1; mu >= 0; --mu) {
        const int n = nblk(mu, L), ld = ldb(n), bo = C.boff[mu], fo = C.foff[mu], bn = C.boff[mu + 1];
        if (part == 0 && r < n) {
            const int b = bo + r;
            T v = czero<T>();
#pragma unroll
            for (int p = 0; p < FP_NLT; ++p) {
                const int k = __ldg(C.up_k + b * FP_NLT + p);
                if (k != 255) v = cfma(C.upv[b * FP_NLT + p], z[bn + k], v);
            }
            rhs[b] = v;
        }
        named_bar(barid, 32 * GW);
        T acc = czero<T>();
        if (r < n) {
#pragma unroll 4
            for (int c = part; c < n; c += GW) acc = cfma(inv[fo + c * ld + r], rhs[bo + c], acc);
        }
#pragma unroll
        for (int o = RPW; o < 32; o <<= 1) acc = cadd(acc, cshfl_xor(acc, o));
        if (part == 0 && r < n) z[bo + r] = cfma(-1.f, acc, z[bo + r]);
        named_bar(barid, 32 * GW);
    }
}

// ----------------------------------------------------- initial state -----
// Projection of the Boltzmann density f ~ exp(bT B.m + sigma z^2) (easy-axis
// frame) on the real SH basis.  The azimuthal integral is exact through the
// modified Bessel functions: int exp(k cos(p - pB)) cos(mu p) dp = 2 pi I_mu(k) cos(mu pB);
// the polar integral uses FP_NGL Gauss-Legendre nodes.  I_mu(k) e^{-k} by the
// backward ratio recurrence r_mu = k / (2 mu + k r_{mu+1}) normalised with
// e^k = I_0 + 2 sum_mu I_mu.
template <int S>
__device__ void initial_state(Ctx<S>& C, const FpParams& P, const double* B, unsigned char* smem) {
    const int L = C.L;
    double* E = (double*)(smem + C.ly.ic);   // [FP_NGL][L+1]
    const double pi = 3.14159265358979323846;
    double Bp = sqrt(B[0] * B[0] + B[1] * B[1]);
    double Babs = sqrt(Bp * Bp + B[2] * B[2]);
    double phiB = atan2(B[1], B[0]);
    double shift = P.bT * Babs + P.sigma;
    for (int i = threadIdx.x; i < FP_NGL; i += NT) {
        double x = c_glx[i], s = sqrt(fmax(0.0, 1.0 - x * x));
        double kap = P.bT * Bp * s;
        int M = (kap > (double)L ? (int)kap : L) + 40;
        if (M > 200) M = 200;
        double r[201];
        r[M] = 0.0;
        double rn = 0.0;
        for (int mu = M - 1; mu >= 1; --mu) { rn = kap / (2.0 * mu + kap * rn); r[mu] = rn; }
        double prod = 1.0, sum = 0.0;
        for (int mu = 1; mu < M; ++mu) { prod *= r[mu]; sum += prod; }
        double I0t = 1.0 / (1.0 + 2.0 * sum);
        double base = c_glw[i] * exp(P.bT * B[2] * x + P.sigma * x * x + kap - shift) * 2.0 * pi;
        prod = I0t;
        E[i * (L + 1)] = base * prod;
        for (int mu = 1; mu <= L; ++mu) { prod *= r[mu]; E[i * (L + 1) + mu] = base * prod; }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double sq2 = 1.4142135623730950488;
    for (int mu = w; mu <= L; mu += NWARP) {
        double xs[FP_NGL / 32], q1[FP_NGL / 32], q2[FP_NGL / 32], ev[FP_NGL / 32];
#pragma unroll
        for (int q = 0; q < FP_NGL / 32; ++q) {
            int i = lane + 32 * q;
            double x = c_glx[i], s = sqrt(fmax(0.0, 1.0 - x * x));
            double v = 1.0 / sqrt(4.0 * pi);
            for (int nu = 1; nu <= mu; ++nu) v *= sqrt((2.0 * nu + 1.0) / (2.0 * nu)) * s;
            xs[q] = x; q1[q] = 0.0; q2[q] = v; ev[q] = E[i * (L + 1) + mu];
        }
        double cphi = cos(mu * phiB), sphi = sin(mu * phiB);
        for (int l = mu; l <= L; ++l) {
            double part = 0.0;
            double a = 0.0, b = 0.0;
            if (l >= mu + 2) {
                a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)mu * mu));
                b = sqrt((((double)l - 1.0) * (l - 1.0) - (double)mu * mu) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            }
#pragma unroll
            for (int q = 0; q < FP_NGL / 32; ++q) {
                double cur;
                if (l == mu) cur = q2[q];
                else if (l == mu + 1) cur = sqrt(2.0 * mu + 3.0) * xs[q] * q2[q];
                else cur = a * (xs[q] * q2[q] - b * q1[q]);
                if (l > mu) { q1[q] = q2[q]; q2[q] = cur; }
                part += cur * ev[q];
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULLMASK, part, o);
            if (lane == 0) {
                int g0 = l * l + l;
                if (mu == 0) C.y[g0] = part;
                else { C.y[g0 + mu] = sq2 * part * cphi; C.y[g0 - mu] = sq2 * part * sphi; }
            }
        }
    }
    __syncthreads();
    double norm = 1.0 / (C.y[0] * sqrt(4.0 * pi));
    __syncthreads();
    for (int i = threadIdx.x; i < C.N; i += NT) C.y[i] *= norm;
    __syncthreads();
}

// ---------------------------------------------------------------- kernel --
__device__ __forceinline__ double sample_time(const fp_drive& d, int j) {
    return ((double)d.warmup_periods + (double)j / (double)d.samples_per_period) * d.period;
}

template <int S>
__global__ void __launch_bounds__(NT, 1) fp_solve_kernel(KArgs A) {
    constexpr int NC = (S - 1) / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_boff[FP_L_MAX + 2], s_foff[FP_L_MAX + 2];
    __shared__ int s_pp[32 * (1 + NC)];
    __shared__ float2 s_colbuf[64 * (1 + NC)];
    __shared__ float s_red[NWARP];
    __shared__ double s_R[9], s_off[3], s_dm[3];
    __shared__ AScal s_scj[S];          // operator scalars at the stage times
    __shared__ double s_Pm[S * S];      // predictor matrix

    Ctx<S> C;
    C.ly = make_layout<S>(A.L_launch);
    C.y = (double*)(smem + C.ly.y);
    C.Z = (double*)(smem + C.ly.Z);
    C.F = (double*)(smem + C.ly.F);
    C.f0 = (double*)(smem + C.ly.f0);
    C.yb = (double*)(smem + C.ly.yb);
    C.diag = (double*)(smem + C.ly.diag);
    C.rr = (float*)(smem + C.ly.rr);
    C.zr = (float*)(smem + C.ly.zr);
    C.rc = (float2*)(smem + C.ly.rc);
    C.zc = (float2*)(smem + C.ly.zc);
    C.dnv = (float*)(smem + C.ly.dnv);
    C.upv = (float*)(smem + C.ly.upv);
    C.fr = (float*)(smem + C.ly.fr);
    C.fc = (float2*)(smem + C.ly.fc);
    C.Xr = (float*)(smem + C.ly.Xr);
    C.Xc = (float2*)(smem + C.ly.Xc);
    C.boff = s_boff;
    C.foff = s_foff;
    const DevTab& T = A.tab;
    const double sq43 = sqrt(4.0 * 3.14159265358979323846 / 3.0);
    const int w = threadIdx.x >> 5;

    for (int inst = blockIdx.x; inst < A.n; inst += gridDim.x) {
        const fp_instance in = A.inst[inst];
        const int L = in.L;
        const bool bad = !(L >= 2 && L <= A.L_launch && in.d > 0.0 && in.K >= 0.0 && in.flags == 0);
        if (bad) {
            for (int e = threadIdx.x; e < A.S_out * 3; e += NT) {
                if (A.m_out) A.m_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
                if (A.dmdt_out) A.dmdt_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
            }
            if (threadIdx.x == 0) {
                A.status[inst] = FP_STATUS_BAD_INPUT;
                if (A.stats) for (int q = 0; q < 4; ++q) A.stats[inst * 4 + q] = 0;
            }
            continue;
        }
        C.L = L;
        C.N = (L + 1) * (L + 1);
        const int N = C.N;
        {
            const int o = A.blk.off[L];
            C.glob = A.blk.glob + o;
            C.sb_k = A.blk.sb_k + (size_t)o * FP_NSB;
            C.sb_g = A.blk.sb_g + (size_t)o * FP_NSB;
            C.sb_cf = A.blk.sb_cf + (size_t)o * FP_NSB;
            C.dn_k = A.blk.dn_k + (size_t)o * FP_NLT;
            C.dn_g = A.blk.dn_g + (size_t)o * FP_NLT;
            C.dn_cf = A.blk.dn_cf + (size_t)o * FP_NLT;
            C.up_k = A.blk.up_k + (size_t)o * FP_NLT;
            C.up_g = A.blk.up_g + (size_t)o * FP_NLT;
            C.up_cf = A.blk.up_cf + (size_t)o * FP_NLT;
            C.dnT = A.blk.dnT + (size_t)o * FP_NLT;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int bo = 0, fo = 0;
            for (int mu = 0; mu <= L + 1; ++mu) {
                s_boff[mu] = bo; s_foff[mu] = fo;
                if (mu <= L) { int nb = nblk(mu, L); bo += nb; fo += nb * ldb(nb); }
            }
            fp_rotation(in.theta, in.phi, s_R);
            for (int k = 0; k < 3; ++k) s_off[k] = in.h_off[k];
        }
        __syncthreads();
        const FpParams P = fp_derive(A.mat, in.K, in.d);
        double R[9], off[3];
        for (int k = 0; k < 9; ++k) R[k] = s_R[k];
        for (int k = 0; k < 3; ++k) off[k] = s_off[k];
        for (int i = threadIdx.x; i < N; i += NT)
            C.diag[i] = -P.D * __ldg(T.lam + i) - 0.5 * P.p4 * __ldg(T.wdiag + i);

        double B[3];
        field_nframe(A, R, off, 0.0, B);
        initial_state<S>(C, P, B, smem);

        const double T_s = A.drv.period / A.drv.samples_per_period;     // sample spacing = h_max
        const double rtol = A.tol.rtol, atol = A.tol.atol;
        const float kappa = 0.02f;
        double t = 0.0;
        double h = fmin(T_s, 0.01 * (0.5 / P.D));
        int jn = 0, nsteps = 0, nrej = 0, nit = 0, nfac = 0, status = FP_STATUS_OK;
        bool have_pred = false, fac_valid = false, force_refac = false;
        int since_fac = 0;
        double h_f = 0.0, h_old = 0.0;
        float eta = 1.0f;

        AScal sc0 = make_scal(P, B);
        apply_A(C.y, C.f0, sc0, C.diag, N, T);            // f0 = A(t) y
        __syncthreads();

        auto write_sample = [&](int j, double tj) {
            // <m> and d<m>/dt at t_j (l = 1 rows of A(t_j) y), rotated back to the lab frame
            if (threadIdx.x < 3) {
                double Bs[3];
                field_nframe(A, R, off, tj, Bs);
                AScal ss = make_scal(P, Bs);
                int row = threadIdx.x == 0 ? 3 : threadIdx.x;   // x' <- (1,1), y' <- (1,-1), z' <- (1,0)
                s_dm[threadIdx.x] = sq43 * apply_row(row, C.y, ss, C.diag, N, T);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double mp[3] = {sq43 * C.y[3], sq43 * C.y[1], sq43 * C.y[2]};
                double dp[3] = {s_dm[0], s_dm[1], s_dm[2]};
                size_t o = ((size_t)inst * A.S_out + j) * 3;
                for (int k = 0; k < 3; ++k) {
                    double mk = R[k] * mp[0] + R[3 + k] * mp[1] + R[6 + k] * mp[2];
                    double dk = R[k] * dp[0] + R[3 + k] * dp[1] + R[6 + k] * dp[2];
                    if (A.m_out) A.m_out[o + k] = mk;
                    if (A.dmdt_out) A.dmdt_out[o + k] = dk;
                }
            }
            __syncthreads();
        };

        if (sample_time(A.drv, 0) <= 0.0) { write_sample(0, 0.0); jn = 1; }

        float ym = 0.f;
        for (int i = threadIdx.x; i < N; i += NT) ym = nanmax(ym, fabsf((float)C.y[i]));
        double ymax = block_max(ym, s_red);
        if (!(ymax <= 3.0e38)) status = FP_STATUS_NONFINITE;      // initial state

        while (status == FP_STATUS_OK && jn < A.S_out) {
            if (nsteps + nrej >= A.tol.max_steps) { status = FP_STATUS_MAXSTEPS; break; }
            if (h < 1e-6 * T_s) { status = FP_STATUS_STEP_UNDERFLOW; break; }
            const double tt = sample_time(A.drv, jn);
            // split the rest of the sample interval into equal steps of at most h, so
            // the step (and with it the factorisation) changes rarely
            const double rem = tt - t;
            const double nrem = ceil(rem / fmin(h, T_s) * (1.0 - 1e-12));
            const bool last = nrem <= 1.0;
            const double hs = last ? rem : rem / nrem;
            const double rat = fac_valid ? hs / h_f : 0.0;
            if (!fac_valid || force_refac || rat < 0.8 || rat > 1.25 || since_fac >= A.tol.refactor_every) {
                if (threadIdx.x == 0) {
                    double Bf[3];
                    field_nframe(A, R, off, t + hs, Bf);
                    s_scj[0] = make_scal(P, Bf);
                }
                __syncthreads();
                const AScal sf = s_scj[0];
                __syncthreads();
                factorize<S>(C, sf, hs, s_pp, s_colbuf);
                h_f = hs; fac_valid = true; force_refac = false; since_fac = 0; ++nfac;
            }
            // per-step scalars, computed once (one lane each) and shared: the operator
            // scalars at the S stage times and the predictor matrix
            if (w == 0) {
                const int lane = threadIdx.x & 31;
                if (lane < S) {
                    double Bj[3];
                    field_nframe(A, R, off, t + RAD<S>().c[lane] * hs, Bj);
                    s_scj[lane] = make_scal(P, Bj);
                }
                if (have_pred && lane < S * S) {
                    const int i = lane / S, j = lane - i * S;
                    const double tau_i = 1.0 + RAD<S>().c[i] * (hs / h_old);
                    const double nj = RAD<S>().c[j];
                    double lj = tau_i / nj;
                    for (int k = 0; k < S; ++k)
                        if (k != j) lj *= (tau_i - RAD<S>().c[k]) / (nj - RAD<S>().c[k]);
                    s_Pm[lane] = lj - (j == S - 1 ? 1.0 : 0.0);
                }
            }
            __syncthreads();
            // predictor from the previous collocation polynomial (nodes 0, c_1..c_S)
            if (have_pred) {
                for (int i = threadIdx.x; i < N; i += NT) {
                    double zo[S];
#pragma unroll
                    for (int j = 0; j < S; ++j) zo[j] = C.Z[j * N + i];
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        double v = 0.0;
#pragma unroll
                        for (int j = 0; j < S; ++j) v = fma(s_Pm[k * S + j], zo[j], v);
                        C.Z[k * N + i] = v;
                    }
                }
            } else {
                for (int i = threadIdx.x; i < S * N; i += NT) C.Z[i] = 0.0;
            }
            __syncthreads();
            const double sc_err = atol + rtol * ymax;
            const float fscale = (float)(h_f / hs);
            bool conv = false, nonfinite = false;
            float prev = 3.0e38f, theta = 0.f;
            eta = powf(fmaxf(eta, 1e-7f), 0.8f);
            for (int it = 0; it < A.tol.newton_max_iter; ++it) {
                // F_j = A(t + c_j h)(y + Z_j) for all stages in one pass, FP64
                for (int e = threadIdx.x; e < S * N; e += NT) C.yb[e] = C.y[e % N] + C.Z[e];
                __syncthreads();
                for (int e = threadIdx.x; e < S * N; e += NT) {
                    const int j = e / N, i = e - j * N;
                    C.F[e] = apply_row(i, C.yb + j * N, s_scj[j], C.diag, N, T);
                }
                __syncthreads();
                // residual R = -Z + h a F (FP64) -> right-hand sides K R (FP32, block order)
                for (int b = threadIdx.x; b < N; b += NT) {
                    const int i = __ldg(C.glob + b);
                    double fv[S];
                    float Rk[S];
#pragma unroll
                    for (int j = 0; j < S; ++j) fv[j] = C.F[j * N + i];
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        double acc = 0.0;
#pragma unroll
                        for (int j = 0; j < S; ++j) acc = fma(RAD<S>().a[k][j], fv[j], acc);
                        Rk[k] = (float)fma(hs, acc, -C.Z[k * N + i]);
                    }
                    float q[S];
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        float acc = 0.f;
#pragma unroll
                        for (int j = 0; j < S; ++j) acc = fmaf((float)RAD<S>().K[k][j], Rk[j], acc);
                        q[k] = acc;
                    }
                    C.rr[b] = q[0];
#pragma unroll
                    for (int p = 0; p < NC; ++p) C.rc[p * N + b] = make_float2(q[1 + 2 * p], q[2 + 2 * p]);
                }
                __syncthreads();
                {
                    constexpr int GW = Groups<S>::GW;
                    const int sys = w / GW, gw = w - sys * GW;
                    if (sys == 0) group_solve<float, S, GW>(C, C.fr, C.rr, C.zr, gw, 1);
                    else if (sys <= NC)
                        group_solve<float2, S, GW>(C, C.fc + (size_t)(sys - 1) * C.ly.fsum, C.rc + (sys - 1) * N,
                                                   C.zc + (sys - 1) * N, gw, 1 + sys);
                }
                __syncthreads();
                // Z += T dW (h_f / h)
                float dm = 0.f;
                for (int b = threadIdx.x; b < N; b += NT) {
                    const int i = __ldg(C.glob + b);
                    float dW[S];
                    dW[0] = fscale * C.zr[b];
#pragma unroll
                    for (int p = 0; p < NC; ++p) {
                        float2 v = C.zc[p * N + b];
                        dW[1 + 2 * p] = fscale * v.x;
                        dW[2 + 2 * p] = fscale * v.y;
                    }
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        float dz = 0.f;
#pragma unroll
                        for (int j = 0; j < S; ++j) dz = fmaf((float)RAD<S>().T[k][j], dW[j], dz);
                        C.Z[k * N + i] += (double)dz;
                        dm = nanmax(dm, fabsf(dz));
                    }
                }
                const float dmax = block_max(dm, s_red);
                ++nit;
                if (!(dmax <= 3.0e38f)) { nonfinite = true; break; }
                if (it >= 1) {
                    theta = dmax / prev;
                    if (theta >= 0.99f) break;
                    eta = theta / (1.f - theta);
                }
                if (eta * dmax <= kappa * (float)sc_err || dmax <= 1e-3f * (float)sc_err) { conv = true; break; }
                prev = dmax;
            }
            if (nonfinite) { status = FP_STATUS_NONFINITE; break; }
            if (!conv) {
                ++nrej;
                if (since_fac == 0 && hs <= 1e-6 * T_s) { status = FP_STATUS_NEWTON_FAIL; break; }
                if (since_fac == 0) h = hs * 0.5;      // fresh factors did not converge: shrink the step
                have_pred = false; force_refac = true; eta = 1.0f;
                __syncthreads();
                continue;
            }
            if (theta > 0.1f) force_refac = true;       // slow contraction: refresh the factors next step
            // embedded error estimate, filtered through the real factor
            for (int b = threadIdx.x; b < N; b += NT) {
                const int i = __ldg(C.glob + b);
                double ev = hs * RAD<S>().g0 * C.f0[i];
#pragma unroll
                for (int j = 0; j < S; ++j) ev = fma(RAD<S>().e[j], C.Z[j * N + i], ev);
                C.rr[b] = (float)ev;
            }
            __syncthreads();
            if (w < Groups<S>::GW) group_solve<float, S, Groups<S>::GW>(C, C.fr, C.rr, C.zr, w, 1);
            __syncthreads();
            float em = 0.f;
            const float escale = (float)(RAD<S>().gam * h_f / hs);
            for (int b = threadIdx.x; b < N; b += NT) em = nanmax(em, fabsf(escale * C.zr[b]));
            const double en = (double)block_max(em, s_red) / sc_err;
            if (!(en < 1e300)) { status = FP_STATUS_NONFINITE; break; }
            const double fac = en > 0.0 ? 0.9 * (double)powf((float)en, -1.f / (S + 1)) : 4.0;
            if (en <= 1.0) {
                float ymx = 0.f;
                for (int i = threadIdx.x; i < N; i += NT) {
                    C.y[i] += C.Z[(S - 1) * N + i];
                    ymx = nanmax(ymx, fabsf((float)C.y[i]));
                }
                ymax = block_max(ymx, s_red);
                if (!(ymax <= 3.0e38)) { status = FP_STATUS_NONFINITE; break; }
                ++nsteps; ++since_fac;
                t = last ? tt : t + hs;
                {   // f0 = A(t) y at the accepted point, for the next error estimate
                    if (threadIdx.x == 0) {
                        double Bn[3];
                        field_nframe(A, R, off, t, Bn);
                        s_scj[0] = make_scal(P, Bn);
                    }
                    __syncthreads();
                    const AScal sn = s_scj[0];
                    apply_A(C.y, C.f0, sn, C.diag, N, T);
                    __syncthreads();
                }
                if (last) { write_sample(jn, tt); ++jn; }
                double hn = hs * fmin(4.0, fmax(0.2, fac));
                if (last && hs < h) hn = fac < 1.0 ? fmin(h, hn) : h;
                // keep the factorised step when the controller asks for a small change
                if (fac_valid && hn >= 0.9 * h_f && hn <= 1.2 * h_f) hn = fmax(h_f, hs);
                h = fmin(hn, T_s);
                h_old = hs;
                have_pred = true;
            } else {
                ++nrej;
                h = hs * fmax(0.1, fac);
                have_pred = false;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            A.status[inst] = status;
            if (A.stats) {
                A.stats[inst * 4 + 0] = nsteps; A.stats[inst * 4 + 1] = nrej;
                A.stats[inst * 4 + 2] = nit;    A.stats[inst * 4 + 3] = nfac;
            }
        }
        for (int e = jn * 3 + threadIdx.x; e < A.S_out * 3; e += NT) {
            if (A.m_out) A.m_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
            if (A.dmdt_out) A.dmdt_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------- host launch ----
int fp_launch_solve(int stages, const DevTab* tab, const DevBlk* blk, const fp_material* mat, const fp_drive* drv,
                    const fp_tol* tol, const fp_instance* d_inst, int n, int L_launch, double* d_m, double* d_dmdt,
                    int* d_status, int* d_stats, int grid, cudaStream_t st) {
    KArgs A;
    A.tab = *tab;
    A.blk = *blk;
    A.mat = *mat;
    A.drv = *drv;
    A.tol = *tol;
    A.inst = d_inst;
    A.n = n;
    A.m_out = d_m;
    A.dmdt_out = d_dmdt;
    A.status = d_status;
    A.stats = d_stats;
    A.S_out = drv->output_periods * drv->samples_per_period;
    A.L_launch = L_launch;
    size_t sm = fp_solver_smem_bytes(stages, L_launch);
    cudaError_t e;
    if (stages == 5) {
        e = cudaFuncSetAttribute(fp_solve_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        fp_solve_kernel<5><<<grid, NT, sm, st>>>(A);
    } else {
        e = cudaFuncSetAttribute(fp_solve_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        fp_solve_kernel<3><<<grid, NT, sm, st>>>(A);
    }
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
}

int fp_upload_constants(const FpRadau* r3, const FpRadau* r5, const double* glx, const double* glw) {
    if (cudaMemcpyToSymbol(c_radau, r3, sizeof(FpRadau), 0) != cudaSuccess) return FP_ECUDA;
    if (cudaMemcpyToSymbol(c_radau, r5, sizeof(FpRadau), sizeof(FpRadau)) != cudaSuccess) return FP_ECUDA;
    if (cudaMemcpyToSymbol(c_glx, glx, sizeof(double) * FP_NGL) != cudaSuccess) return FP_ECUDA;
    if (cudaMemcpyToSymbol(c_glw, glw, sizeof(double) * FP_NGL) != cudaSuccess) return FP_ECUDA;
    return FP_OK;
}
