// Batched Fokker-Planck solver for Neel rotation (Sec. 2.1, Eq. FP-general,
// Eq. convection, Eq. mean_magmom_FP) on sm_103a.
//
// One CTA owns one instance at a time (persistent loop over instances, taken
// from a work counter).  The real-SH coefficient vector c (N = (L+1)^2
// doubles) and every Radau stage live in shared memory; the FP32 factors too
// with 3 stages up to degree FP_L_SMEM, otherwise in a global slot per CTA
// that stays in L2 (5 stages: two CTAs per SM).  Nothing is streamed from HBM
// per step except the L1/L2-resident coupling tables shared by all instances.
//
// Time step: S-stage Radau IIA (S = 3: order 5, S = 5: order 9; L-stable),
// simplified Newton:
//   residual   R_i = -Z_i + h sum_j a_ij A(t + c_j h)(y + Z_j)         FP64
//   correction (Lam - h_f Abar) dW = K R,  dZ = T dW (h_f / h)          FP32
// Abar = A(t_f + h_f) is frozen over several steps.  Lam - h_f Abar splits into
// one real and (S-1)/2 complex systems, each block-tridiagonal in |m|; every
// system is factorised (block Thomas) into explicit FP32 inverses of its
// Schur-complement diagonal blocks by a group of warps per system
// (Gauss-Jordan with partial pivoting in registers, one named barrier per
// pivot) and solved by the same group.
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
    const int* order;       // queue slot -> instance index (NULL: identity)
    int* queue;             // dynamic work counter, zero at launch (NULL: static round robin)
    unsigned char* fac;     // global factor scratch (degrees above FP_L_SMEM): fac_stride bytes per CTA
    size_t fac_stride;
};

// slot -> scalar group: W, ZR, RZ, RX, RY, GZ, GX, GY
__host__ __device__ constexpr int grp_of(int k) {
    return k < 2 ? 0 : k < 4 ? 1 : k < 5 ? 2 : k < 7 ? 3 : k < 9 ? 4 : k < 11 ? 5 : k < 15 ? 6 : 7;
}

// slot -> group of the forward apply: anisotropy, x', y', z' (coef4 table)
__host__ __device__ constexpr int grp4_of(int k) {
    return k < 4 ? 0 : k == 4 ? 3 : k < 7 ? 1 : k < 9 ? 2 : k < 11 ? 3 : k < 15 ? 1 : 2;
}

// operator scalars: s per slot group (factorisation, adjoint) and s4 per
// forward-apply group (-p3, -p1 B'_x, -p1 B'_y, -p1 B'_z)
struct AScal { double s[8]; double s4[4]; };

// ---------------------------------------------------------------- layout ----
__host__ __device__ inline int nblk(int mu, int L) { return mu == 0 ? L + 1 : 2 * (L + 1 - mu); }
// column stride of a stored inverse block: odd, so the lanes of a column-split matvec hit distinct banks
__host__ __device__ inline int ldb(int n) { return n | 1; }
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Step-control constants of the forward integration (library defaults):
// the Newton iteration stops when eta * |dZ| <= FP_KAPPA * tolerance; factors
// are reused while h / h_factor stays in [FP_HRAT_LO, FP_HRAT_HI] and are
// refreshed after a step whose contraction rate exceeded FP_THETA_REFAC.
#ifndef FP_KAPPA
#define FP_KAPPA 0.2f
#endif
#ifndef FP_THETA_REFAC
#define FP_THETA_REFAC 0.05f
#endif
#ifndef FP_HRAT_LO
#define FP_HRAT_LO 0.8
#endif
#ifndef FP_HRAT_HI
#define FP_HRAT_HI 1.25
#endif

struct Layout {
    int N, L, nmax;
    size_t y, Z, F, f0, yb, diag, rr, zr, rc, zc, dnv, upv, fr, fc, Xr, Xc, lam, aw, ic, total;
    size_t fsum;
    bool gfac;              // factors in global memory (five stages, or degree above FP_L_SMEM); fr, fc are then offsets into it
    size_t fac_bytes;       // bytes of the factors of one instance
};

// ADJ adds the adjoint state lambda (N) and one more stage-sized buffer (S N).
template <int S, bool ADJ = false>
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
    // five-stage factors (131 KB at degree 16) live in a global, L2-resident
    // slot per CTA (the solve: two CTAs per SM; the adjoint: the slot opens
    // its workspace); three-stage factors stay in shared memory up to degree
    // FP_L_SMEM
    ly.gfac = L > FP_L_SMEM || S == 5;
    ly.fac_bytes = al16(fsum * 4) + al16((size_t)NC * fsum * 8);
    if (ly.gfac) {
        ly.fr = 0;
        ly.fc = al16(fsum * 4);
    } else {
        ly.fr = o;   o = al16(o + fsum * 4);
        ly.fc = o;   o = al16(o + (size_t)NC * fsum * 8);
    }
    ly.Xr = o;   o = al16(o + nm2 * 4);
    ly.Xc = o;   o = al16(o + (size_t)NC * nm2 * 8);
    ly.lam = o;  if (ADJ) o = al16(o + N * 8);
    ly.aw = o;   if (ADJ) o = al16(o + (size_t)S * N * 8);
    if (ly.gfac) {                                     // initial-state scratch of its own
        ly.ic = o;
        o = al16(o + (size_t)FP_NGL * (L + 1) * 8);
        ly.total = o;
    } else {
        ly.ic = ly.fr;                                 // initial-state scratch aliases the factors
        size_t ic_end = ly.ic + (size_t)FP_NGL * (L + 1) * 8;
        ly.total = o > ic_end ? o : al16(ic_end);
    }
    return ly;
}

size_t fp_solver_smem_bytes(int stages, int L) {
    return stages == 5 ? make_layout<5>(L).total : make_layout<3>(L).total;
}
size_t fp_solver_fac_bytes(int stages, int L) {
    const Layout ly = stages == 5 ? make_layout<5>(L) : make_layout<3>(L);
    return ly.gfac ? ly.fac_bytes : 0;
}
int fp_solver_ctas_per_sm(int stages, int L) { return stages == 5 && L <= FP_L_SMEM ? 2 : 1; }
size_t fp_solver_fac_scratch_bytes(int stages, int L, int num_sms) {
    return (size_t)num_sms * fp_solver_ctas_per_sm(stages, L) * fp_solver_fac_bytes(stages, L);
}
size_t fp_adjoint_smem_bytes(int stages, int L) {
    return stages == 5 ? make_layout<5, true>(L).total : make_layout<3, true>(L).total;
}
// global factor doubles at the head of each adjoint CTA's workspace (0 when the
// factors fit in shared memory), even so that every CTA's slot is 16-byte aligned
static size_t adjoint_fac_doubles(int stages, int L) {
    const Layout ly = stages == 5 ? make_layout<5, true>(L) : make_layout<3, true>(L);
    return ly.gfac ? ((ly.fac_bytes + 15) / 16) * 2 : 0;
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
__device__ __forceinline__ float crecip(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float2 crecip(float2 a) {
    float d = __frcp_rn(a.x * a.x + a.y * a.y);
    return make_float2(a.x * d, -a.y * d);
}
// a[idx] for a register array of power-of-two length M (log2 M select levels)
template <class T, int M>
__device__ __forceinline__ T tree_pick(const T* a, int idx) {
    T t[M];
#pragma unroll
    for (int i = 0; i < M; ++i) t[i] = a[i];
#pragma unroll
    for (int w = M / 2; w >= 1; w /= 2) {
#pragma unroll
        for (int i = 0; i < w; ++i) t[i] = (idx & w) ? t[i + w] : t[i];
    }
    return t[0];
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
    s.s4[0] = -P.p3;
    s.s4[1] = -P.p1 * B[0];
    s.s4[2] = -P.p1 * B[1];
    s.s4[3] = -P.p1 * B[2];
    return s;
}

// row i of A x (FP64, matrix-free from the closed-form tables, slots grouped
// by the four forward-apply scalars)
__device__ __forceinline__ double apply_row(int i, const double* __restrict__ x, const AScal& sc,
                                            const double* __restrict__ diag, int N, const DevTab& T) {
    const double* cf = T.coef4 + i;
    const int* sr = T.src + i;
    const int ld = T.nrow;
    double g[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) g[q] = 0.0;
#pragma unroll
    for (int k = 0; k < FP_NSLOT; ++k) {
        int j = __ldg(sr + k * ld);
        double v = ((unsigned)j < (unsigned)N) ? x[j] : 0.0;
        g[grp4_of(k)] = fma(__ldg(cf + k * ld), v, g[grp4_of(k)]);
    }
    double acc = diag[i] * x[i];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = fma(sc.s4[q], g[q], acc);
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
    double *y, *Z, *F, *f0, *yb, *diag, *lam, *aw;
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
    const uint8_t *sb_k, *sb_g, *dn_k, *dn_g, *up_k, *up_g, *dnT, *upT;
    const float *sb_cf, *dn_cf, *up_cf;
};

// ------------------------------------------- factorisation (block Thomas) --
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// A group of GW warps assembles the Schur-complement block
// D~_mu = D_mu - C_mu X_{mu-1} of one system (lane = row, RS row slots per
// lane: rows lane + 32 s, warp gw owns the columns [gw*CPW, gw*CPW + CPW)) and
// inverts it in place by Gauss-Jordan with partial pivoting: the warp owning
// pivot column k picks the pivot row and publishes the column multipliers
// through shared memory, one named barrier per pivot.  The inverse is stored
// column-major (out[c * ldb(n) + r] = Inv[r][c]).  n <= 32 RS.
template <class T, int S, int GW, int RS = 1>
__device__ void group_factor_block(Ctx<S>& C, int mu, T shift, const float* gs, float h, const T* Xprev, T* out,
                                   int* pp, T* colbuf, int gw, int barid) {
    constexpr int NB = 32 * RS;             // largest block (rows and columns)
    constexpr int CPW = NB / GW;
    constexpr unsigned RMASK = (unsigned)NB - 1u;
    const int lane = threadIdx.x & 31;
    const int L = C.L, n = nblk(mu, L), bo = C.boff[mu];
    const int j0 = gw * CPW;
    T a[RS][CPW];
    bool used[RS];
    int myk[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) {
        const int r = lane + 32 * s;
        used[s] = r >= n;
        myk[s] = -1;
        if (r < n) {
            const int b = bo + r;
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
                T v = j == r ? dv : czero<T>();
                if (j < n) {
#pragma unroll
                    for (int p = 0; p < FP_NSB; ++p) v = cadd_real(v, ks[p] == j ? vs[p] : 0.f);
#pragma unroll
                    for (int p = 0; p < FP_NLT; ++p)
                        if (kd[p] != 255) v = cfma(-vd[p], Xprev[kd[p] * n + j], v);
                }
                a[s][jj] = v;
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < CPW; ++jj) a[s][jj] = cadd_real(czero<T>(), j0 + jj == r ? 1.f : 0.f);
        }
    }
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        const int owner = k / CPW, kk = k - owner * CPW;
        T* cb = colbuf + (k & 1) * NB;
        if (gw == owner) {
            T ak[RS];
            unsigned key = 0u;
#pragma unroll
            for (int s = 0; s < RS; ++s) {
                ak[s] = tree_pick<T, CPW>(a[s], kk);
                const float v = used[s] ? 0.f : cabs1(ak[s]);
                key = max(key, (__float_as_uint(v) & ~RMASK) | (unsigned)(lane + 32 * s));
            }
            key = __reduce_max_sync(FULLMASK, key);
            const int p = (int)(key & RMASK);
            T akp = ak[0];
#pragma unroll
            for (int s = 1; s < RS; ++s) akp = (p >> 5) == s ? ak[s] : akp;
            const T pinv = crecip(cshfl(akp, p & 31));
#pragma unroll
            for (int s = 0; s < RS; ++s) {
                const int r = lane + 32 * s;
                cb[r] = r == p ? pinv : cneg(cmul(ak[s], pinv));
            }
            if (lane == 0) pp[k] = p;
        }
        named_bar(barid, 32 * GW);
        const int p = pp[k];
        const int ps = p >> 5, pl = p & 31;
        T mlt[RS];                               // pinv on the pivot row, -a_ik / a_pk elsewhere
#pragma unroll
        for (int s = 0; s < RS; ++s) mlt[s] = cb[lane + 32 * s];
#pragma unroll
        for (int jj = 0; jj < CPW; ++jj) {
            T src = a[0][jj];
#pragma unroll
            for (int s = 1; s < RS; ++s) src = ps == s ? a[s][jj] : src;
            const T prj = cshfl(src, pl);
#pragma unroll
            for (int s = 0; s < RS; ++s) {
                const bool ispiv = lane + 32 * s == p;
                const T upd = ispiv ? cmul(prj, mlt[s]) : cfma(mlt[s], prj, a[s][jj]);
                a[s][jj] = (j0 + jj == k) ? mlt[s] : upd;
            }
        }
#pragma unroll
        for (int s = 0; s < RS; ++s)
            if (lane + 32 * s == p) { used[s] = true; myk[s] = k; }
    }
#pragma unroll
    for (int s = 0; s < RS; ++s) {
        if (lane + 32 * s < n && myk[s] >= 0) {
#pragma unroll
            for (int jj = 0; jj < CPW; ++jj) {
                const int j = j0 + jj;
                if (j < n) {
                    const int pj = pp[j];
                    if (pj < n) out[pj * ldb(n) + myk[s]] = a[s][jj];  // pj >= n only for a singular block
                }
            }
        }
    }
}

// X_mu = Inv_mu B_mu (n x n2, row-major) for one system; one warp per column c
// (lane = row r).  B_mu[k][c] is the coupling of row k (block mu) to row c
// (block mu+1), reached through the dn list of row c and its back pointer.
template <class T, int S, int RS = 1>
__device__ __forceinline__ void x_column(Ctx<S>& C, int mu, int c, const T* inv, T* X) {
    const int lane = threadIdx.x & 31;
    const int L = C.L, n = nblk(mu, L), n2 = nblk(mu + 1, L);
    const int bc = C.boff[mu + 1] + c, bo = C.boff[mu];
    T acc[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) acc[s] = czero<T>();
#pragma unroll
    for (int p = 0; p < FP_NLT; ++p) {
        const int k = __ldg(C.dn_k + bc * FP_NLT + p);
        if (k == 255) continue;
        const int q = __ldg(C.dnT + bc * FP_NLT + p);
        const float bv = q == 255 ? 0.f : C.upv[(bo + k) * FP_NLT + q];
#pragma unroll
        for (int s = 0; s < RS; ++s)
            if (lane + 32 * s < n) acc[s] = cfma(bv, inv[k * ldb(n) + lane + 32 * s], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < RS; ++s)
        if (lane + 32 * s < n) X[(lane + 32 * s) * n2 + c] = acc[s];
}

template <int S> struct Groups {
    static constexpr int NC = (S - 1) / 2;
    static constexpr int NSYS = 1 + NC;
    static constexpr int GW = NWARP / NSYS >= 4 ? 4 : (NWARP / NSYS >= 2 ? 2 : 1);   // warps per system
};

// per-system scratch of the factorisation: pivot rows (FP_PP_SYS ints) and the
// double-buffered multiplier column (FP_CB_SYS entries), sized for 64-row blocks
#define FP_PP_SYS 64
#define FP_CB_SYS 128

template <int S, int RS = 1>
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
            group_factor_block<float, S, GW, RS>(C, mu, (float)RAD<S>().gam, gs, (float)h, C.Xr, C.fr + C.foff[mu],
                                                 pp, (float*)colbuf, gw, 1);
        } else if (sys <= NC) {
            const int q = sys - 1;
            const float2 shift = make_float2((float)RAD<S>().alp[q], -(float)RAD<S>().bet[q]);
            group_factor_block<float2, S, GW, RS>(C, mu, shift, gs, (float)h, C.Xc + q * nm2,
                                                  C.fc + (size_t)q * C.ly.fsum + C.foff[mu], pp + FP_PP_SYS * sys,
                                                  colbuf + FP_CB_SYS * sys, gw, 1 + sys);
        }
        __syncthreads();
        if (mu < L) {
            const int n2 = nblk(mu + 1, L);
            for (int item = w; item < NSYS * n2; item += NWARP) {
                const int sy = item / n2, c = item - sy * n2;
                if (sy == 0) x_column<float, S, RS>(C, mu, c, C.fr + C.foff[mu], C.Xr);
                else x_column<float2, S, RS>(C, mu, c, C.fc + (size_t)(sy - 1) * C.ly.fsum + C.foff[mu],
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
template <class T, int S, int GW, bool TRANS, int RS = 1>
__device__ void group_solve(Ctx<S>& C, const T* __restrict__ inv, T* rhs, T* z, int gw, int barid) {
    // TRANS solves M^T x = b with the same factors: the forward sweep uses
    // B^T (values reached through dnT), the backward sweep C^T (through upT) and
    // the block inverses transposed.
    constexpr int RPW = 32 * RS / GW;       // rows per warp (GW warps cover blocks of up to 32 RS rows)
    constexpr int NPART = 32 / RPW;         // lanes sharing one row's columns
    static_assert(RPW <= 32, "a warp holds at most 32 rows");
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
                if (k == 255) continue;
                float cv;
                if (TRANS) {
                    const int q = __ldg(C.dnT + b * FP_NLT + p);
                    cv = q == 255 ? 0.f : C.upv[(bp + k) * FP_NLT + q];
                } else {
                    cv = C.dnv[b * FP_NLT + p];
                }
                v = cfma(-cv, z[bp + k], v);
            }
            rhs[b] = v;
        }
        named_bar(barid, 32 * GW);
        T acc = czero<T>();
        if (r < n) {
#pragma unroll 4
            for (int c = part; c < n; c += NPART)
                acc = cfma(inv[fo + (TRANS ? r * ld + c : c * ld + r)], rhs[bo + c], acc);
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
                if (k == 255) continue;
                float cv;
                if (TRANS) {
                    const int q = __ldg(C.upT + b * FP_NLT + p);
                    cv = q == 255 ? 0.f : C.dnv[(bn + k) * FP_NLT + q];
                } else {
                    cv = C.upv[b * FP_NLT + p];
                }
                v = cfma(cv, z[bn + k], v);
            }
            rhs[b] = v;
        }
        named_bar(barid, 32 * GW);
        T acc = czero<T>();
        if (r < n) {
#pragma unroll 4
            for (int c = part; c < n; c += NPART)
                acc = cfma(inv[fo + (TRANS ? r * ld + c : c * ld + r)], rhs[bo + c], acc);
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
__device__ void initial_state(Ctx<S>& C, const FpParams& P, const double* B, unsigned char* smem, double* out) {
    const int L = C.L;
    double* E = (double*)(smem + C.ly.ic);   // [FP_NGL][L+1]; aliases the factor storage
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
                if (mu == 0) out[g0] = part;
                else { out[g0 + mu] = sq2 * part * cphi; out[g0 - mu] = sq2 * part * sphi; }
            }
        }
    }
    __syncthreads();
    double norm = 1.0 / (out[0] * sqrt(4.0 * pi));
    __syncthreads();
    for (int i = threadIdx.x; i < C.N; i += NT) out[i] *= norm;
    __syncthreads();
}

// ---------------------------------------------------------------- kernel --
__device__ __forceinline__ double sample_time(const fp_drive& d, int j) {
    return ((double)d.warmup_periods + (double)j / (double)d.samples_per_period) * d.period;
}

// Shared (per-CTA) scalars of the instance being integrated.
template <int S>
struct Shared {
    int boff[FP_L_MAX + 2], foff[FP_L_MAX + 2];
    int pp[FP_PP_SYS * (1 + (S - 1) / 2)];
    float2 colbuf[FP_CB_SYS * (1 + (S - 1) / 2)];
    float red[NWARP];
    double dred[NWARP * 12];
    double R[9], off[3], dm[4];          // dm[3]: |<m>|^2 of the last written sample
    AScal scj[S];          // operator scalars at the stage times
    double Pm[S * S];      // predictor matrix
};

template <int S, bool ADJ>
__device__ void bind_smem(Ctx<S>& C, unsigned char* smem, int L_launch, Shared<S>& sh, unsigned char* fac) {
    C.ly = make_layout<S, ADJ>(L_launch);
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
    unsigned char* fb = C.ly.gfac ? fac : smem;       // factors: shared memory, or this CTA's global scratch
    C.fr = (float*)(fb + C.ly.fr);
    C.fc = (float2*)(fb + C.ly.fc);
    C.Xr = (float*)(smem + C.ly.Xr);
    C.Xc = (float2*)(smem + C.ly.Xc);
    C.lam = (double*)(smem + C.ly.lam);
    C.aw = (double*)(smem + C.ly.aw);
    C.boff = sh.boff;
    C.foff = sh.foff;
}

__device__ __forceinline__ bool instance_ok(const fp_instance& in, int L_launch) {
    return in.L >= 2 && in.L <= L_launch && in.d > 0.0 && in.K >= 0.0 && in.flags == 0;
}

// Per-instance setup: block structure pointers and offsets, rotation, offset
// field, FP64 diagonal of A.  Returns the Neel constants.
template <int S>
__device__ FpParams setup_instance(Ctx<S>& C, const KArgs& A, const fp_instance& in, Shared<S>& sh) {
    const int L = in.L;
    C.L = L;
    C.N = (L + 1) * (L + 1);
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
    C.upT = A.blk.upT + (size_t)o * FP_NLT;
    __syncthreads();
    if (threadIdx.x == 0) {
        int bo = 0, fo = 0;
        for (int mu = 0; mu <= L + 1; ++mu) {
            sh.boff[mu] = bo; sh.foff[mu] = fo;
            if (mu <= L) { int nb = nblk(mu, L); bo += nb; fo += nb * ldb(nb); }
        }
        fp_rotation(in.theta, in.phi, sh.R);
        for (int k = 0; k < 3; ++k) sh.off[k] = in.h_off[k];
    }
    __syncthreads();
    const FpParams P = fp_derive(A.mat, in.K, in.d);
    for (int i = threadIdx.x; i < C.N; i += NT)
        C.diag[i] = -P.D * __ldg(A.tab.lam + i) - 0.5 * P.p4 * __ldg(A.tab.wdiag + i);
    __syncthreads();
    return P;
}

// Simplified Newton iteration for the collocation stages Z (in C.Z, initial
// guess already set) of the step (t, hs) from C.y; stage scalars in sh.scj.
struct NewtonResult { bool conv, nonfinite; float theta, dmax; int iters; };

template <int S, int RS = 1>
__device__ NewtonResult newton_stages(Ctx<S>& C, const DevTab& T, double hs, double h_f, double sc_err, float& eta,
                                      float kappa, int maxit, Shared<S>& sh) {
    constexpr int NC = (S - 1) / 2;
    const int N = C.N, w = threadIdx.x >> 5;
    const float fscale = (float)(h_f / hs);
    NewtonResult res{false, false, 0.f, 0.f, 0};
    float prev = 3.0e38f;
    eta = powf(fmaxf(eta, 1e-7f), 0.8f);
    for (int it = 0; it < maxit; ++it) {
        // F_j = A(t + c_j h)(y + Z_j) for all stages in one pass, FP64
        for (int e = threadIdx.x; e < S * N; e += NT) C.yb[e] = C.y[e % N] + C.Z[e];
        __syncthreads();
        for (int e = threadIdx.x; e < S * N; e += NT) {
            const int j = e / N, i = e - j * N;
            C.F[e] = apply_row(i, C.yb + j * N, sh.scj[j], C.diag, N, T);
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
            if (sys == 0) group_solve<float, S, GW, false, RS>(C, C.fr, C.rr, C.zr, gw, 1);
            else if (sys <= NC)
                group_solve<float2, S, GW, false, RS>(C, C.fc + (size_t)(sys - 1) * C.ly.fsum, C.rc + (sys - 1) * N,
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
        const float dmax = block_max(dm, sh.red);
        ++res.iters;
        res.dmax = dmax;
        if (!(dmax <= 3.0e38f)) { res.nonfinite = true; break; }
        if (it >= 1) {
            res.theta = dmax / prev;
            if (res.theta >= 0.99f) break;
            eta = res.theta / (1.f - res.theta);
        }
        if (eta * dmax <= kappa * (float)sc_err || dmax <= 1e-3f * kappa * (float)sc_err) { res.conv = true; break; }
        prev = dmax;
    }
    return res;
}

// operator scalars at the S stage times of (t, hs) and, if pred, the
// predictor matrix; one lane each, shared through sh
template <int S>
__device__ void stage_scalars(const KArgs& A, const FpParams& P, const double* R, const double* off, double t,
                              double hs, bool pred, double h_old, Shared<S>& sh) {
    const int lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) == 0) {
        // one drive component per lane (lane = 3 j + k), then lane j rotates
        // stage j's field into the easy-axis frame
        const double twopi = 6.283185307179586476925286766559;
        double bk = 0.0;
        if (lane < 3 * S) {
            const int j = lane / 3, k = lane - 3 * j;
            bk = off[k] + A.drv.amp[k] * sin(twopi * A.drv.freq[k] * (t + RAD<S>().c[j] * hs) + A.drv.phase[k]);
        }
        double bl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) bl[k] = __shfl_sync(FULLMASK, bk, (3 * lane + k) & 31);
        if (lane < S) {
            double Bj[3];
            for (int r = 0; r < 3; ++r) Bj[r] = R[3 * r] * bl[0] + R[3 * r + 1] * bl[1] + R[3 * r + 2] * bl[2];
            sh.scj[lane] = make_scal(P, Bj);
        }
    } else if ((threadIdx.x >> 5) == 1) {
        if (pred && lane < S * S) {
            const int i = lane / S, j = lane - i * S;
            const double tau_i = 1.0 + RAD<S>().c[i] * (hs / h_old);
            const double nj = RAD<S>().c[j];
            double lj = tau_i / nj;
            for (int k = 0; k < S; ++k)
                if (k != j) lj *= (tau_i - RAD<S>().c[k]) / (nj - RAD<S>().c[k]);
            sh.Pm[lane] = lj - (j == S - 1 ? 1.0 : 0.0);
        }
    }
    __syncthreads();
}

template <int S>
__device__ void predict_stages(Ctx<S>& C, bool pred, Shared<S>& sh) {
    const int N = C.N;
    if (pred) {
        for (int i = threadIdx.x; i < N; i += NT) {
            double zo[S];
#pragma unroll
            for (int j = 0; j < S; ++j) zo[j] = C.Z[j * N + i];
#pragma unroll
            for (int k = 0; k < S; ++k) {
                double v = 0.0;
#pragma unroll
                for (int j = 0; j < S; ++j) v = fma(sh.Pm[k * S + j], zo[j], v);
                C.Z[k * N + i] = v;
            }
        }
    } else {
        for (int i = threadIdx.x; i < S * N; i += NT) C.Z[i] = 0.0;
    }
    __syncthreads();
}

// factorise the iteration matrices for step hs with the operator scalars sc of
// its end point (stage S of the step, c_S = 1)
template <int S, int RS = 1>
__device__ void refactor_at(Ctx<S>& C, const AScal& sc, double hs, Shared<S>& sh) {
    factorize<S, RS>(C, sc, hs, sh.pp, sh.colbuf);
}

// factorise the iteration matrices for step hs ending at t + hs
template <int S>
__device__ void refactor(Ctx<S>& C, const KArgs& A, const FpParams& P, const double* R, const double* off, double t,
                         double hs, Shared<S>& sh) {
    if (threadIdx.x == 0) {
        double Bf[3];
        field_nframe(A, R, off, t + hs, Bf);
        sh.scj[0] = make_scal(P, Bf);
    }
    __syncthreads();
    const AScal sf = sh.scj[0];
    __syncthreads();
    factorize<S>(C, sf, hs, sh.pp, sh.colbuf);
}

// Adaptive integration of one instance over the whole schedule.  SOLVE mode
// writes <m>, d<m>/dt at every sample; REC mode instead records every accepted
// step (t, h, sample index or -1, and the (t, h) its iteration matrices were
// factorised at) in rec_steps and the state before every CKPT-th step in
// rec_ckpt, so that a replay can use exactly the same factors.
#define FP_CKPT 64
#define FP_REC 5            // doubles recorded per accepted step
struct FwdOut { int status, nsteps, nrej, nit, nfac; };

template <int S, bool REC, int RS = 1>
__device__ FwdOut forward_instance(Ctx<S>& C, const KArgs& A, int inst, const FpParams& P, Shared<S>& sh,
                                   double* rec_steps, double* rec_ckpt, int max_rec) {
    const DevTab& T = A.tab;
    const int N = C.N;
    const double sq43 = sqrt(4.0 * 3.14159265358979323846 / 3.0);
    double R[9], off[3];
    for (int k = 0; k < 9; ++k) R[k] = sh.R[k];
    for (int k = 0; k < 3; ++k) off[k] = sh.off[k];
    double B[3];
    field_nframe(A, R, off, 0.0, B);
    initial_state<S>(C, P, B, (unsigned char*)C.y - C.ly.y, C.y);
    static_assert(!(REC && RS != 1), "the adjoint records steps of the single-slot factorisation only");

    const double T_s = A.drv.period / A.drv.samples_per_period;     // sample spacing = h_max
    const double rtol = A.tol.rtol, atol = A.tol.atol;
    double t = 0.0;
    double h = fmin(T_s, 0.01 * (0.5 / P.D));
    FwdOut out{FP_STATUS_OK, 0, 0, 0, 0};
    int jn = 0;
    bool have_pred = false, fac_valid = false, force_refac = false;
    int since_fac = 0;
    double h_f = 0.0, h_old = 0.0, t_f = 0.0;
    float eta = 1.0f;

    {
        const AScal sc0 = make_scal(P, B);
        apply_A(C.y, C.f0, sc0, C.diag, N, T);                 // f0 = A(t) y
        __syncthreads();
    }
    auto write_sample = [&](int j, const AScal& ss) {
        if (REC) return;
        // <m> and d<m>/dt at t_j (l = 1 rows of A(t_j) y, ss = operator scalars
        // at t_j), rotated back to the lab frame
        if (threadIdx.x < 3) {
            int row = threadIdx.x == 0 ? 3 : threadIdx.x;   // x' <- (1,1), y' <- (1,-1), z' <- (1,0)
            sh.dm[threadIdx.x] = sq43 * apply_row(row, C.y, ss, C.diag, N, T);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double mp[3] = {sq43 * C.y[3], sq43 * C.y[1], sq43 * C.y[2]};
            double dp[3] = {sh.dm[0], sh.dm[1], sh.dm[2]};
            sh.dm[3] = mp[0] * mp[0] + mp[1] * mp[1] + mp[2] * mp[2];
            size_t o = ((size_t)inst * A.S_out + j) * 3;
            for (int k = 0; k < 3; ++k) {
                double mk = R[k] * mp[0] + R[3 + k] * mp[1] + R[6 + k] * mp[2];
                double dk = R[k] * dp[0] + R[3 + k] * dp[1] + R[6 + k] * dp[2];
                if (A.m_out) A.m_out[o + k] = mk;
                if (A.dmdt_out) A.dmdt_out[o + k] = dk;
            }
        }
        __syncthreads();
        // the mean of unit vectors has norm <= 1; beyond that the truncated
        // operator at this L is not dissipative for the instance
        if (sh.dm[3] > (1.0 + 1e-6) * (1.0 + 1e-6) && out.status == FP_STATUS_OK) out.status = FP_STATUS_UNRESOLVED;
    };

    if (sample_time(A.drv, 0) <= 0.0) { write_sample(0, make_scal(P, B)); jn = 1; }

    float ym = 0.f;
    for (int i = threadIdx.x; i < N; i += NT) ym = nanmax(ym, fabsf((float)C.y[i]));
    double ymax = block_max(ym, sh.red);
    if (!(ymax <= 3.0e38)) out.status = FP_STATUS_NONFINITE;      // initial state

    while (out.status == FP_STATUS_OK && jn < A.S_out) {
        if (out.nsteps + out.nrej >= A.tol.max_steps || (REC && out.nsteps >= max_rec)) {
            out.status = FP_STATUS_MAXSTEPS;
            break;
        }
        if (h < 1e-6 * T_s) { out.status = FP_STATUS_STEP_UNDERFLOW; break; }
        const double tt = sample_time(A.drv, jn);
        // split the rest of the sample interval into equal steps of at most h, so
        // the step (and with it the factorisation) changes rarely
        const double rem = tt - t;
        const double nrem = ceil(rem / fmin(h, T_s) * (1.0 - 1e-12));
        const bool last = nrem <= 1.0;
        const double hs = last ? rem : rem / nrem;
        stage_scalars<S>(A, P, R, off, t, hs, have_pred, h_old, sh);
        const AScal s_end = sh.scj[S - 1];           // operator scalars at t + hs (c_S = 1)
        const double rat = fac_valid ? hs / h_f : 0.0;
        if (!fac_valid || force_refac || rat < FP_HRAT_LO || rat > FP_HRAT_HI || since_fac >= A.tol.refactor_every) {
            refactor_at<S, RS>(C, s_end, hs, sh);
            h_f = hs; t_f = t; fac_valid = true; force_refac = false; since_fac = 0; ++out.nfac;
        }
        if (REC && out.nsteps % FP_CKPT == 0) {       // checkpoint the state before this step
            double* ck = rec_ckpt + (size_t)(out.nsteps / FP_CKPT) * N;
            for (int i = threadIdx.x; i < N; i += NT) ck[i] = C.y[i];
        }
        predict_stages<S>(C, have_pred, sh);
        const double sc_err = atol + rtol * ymax;
        const NewtonResult nr = newton_stages<S, RS>(C, T, hs, h_f, sc_err, eta, FP_KAPPA, A.tol.newton_max_iter, sh);
        out.nit += nr.iters;
        if (nr.nonfinite) { out.status = FP_STATUS_NONFINITE; break; }
        if (!nr.conv) {
            ++out.nrej;
            if (since_fac == 0 && hs <= 1e-6 * T_s) { out.status = FP_STATUS_NEWTON_FAIL; break; }
            if (since_fac == 0) h = hs * 0.5;      // fresh factors did not converge: shrink the step
            have_pred = false; force_refac = true; eta = 1.0f;
            __syncthreads();
            continue;
        }
        if (nr.theta > FP_THETA_REFAC) force_refac = true;   // slow contraction: refresh the factors next step
        // embedded error estimate, filtered through the real factor
        for (int b = threadIdx.x; b < N; b += NT) {
            const int i = __ldg(C.glob + b);
            double ev = hs * RAD<S>().g0 * C.f0[i];
#pragma unroll
            for (int j = 0; j < S; ++j) ev = fma(RAD<S>().e[j], C.Z[j * N + i], ev);
            C.rr[b] = (float)ev;
        }
        __syncthreads();
        if ((threadIdx.x >> 5) < Groups<S>::GW)
            group_solve<float, S, Groups<S>::GW, false, RS>(C, C.fr, C.rr, C.zr, threadIdx.x >> 5, 1);
        __syncthreads();
        float em = 0.f;
        const float escale = (float)(RAD<S>().gam * h_f / hs);
        for (int b = threadIdx.x; b < N; b += NT) em = nanmax(em, fabsf(escale * C.zr[b]));
        const double en = (double)block_max(em, sh.red) / sc_err;
        if (!(en < 1e300)) { out.status = FP_STATUS_NONFINITE; break; }
        const double fac = en > 0.0 ? 0.9 * (double)powf((float)en, -1.f / (S + 1)) : 4.0;
        if (en <= 1.0) {
            if (REC && threadIdx.x == 0) {
                double* r = rec_steps + (size_t)out.nsteps * FP_REC;
                r[0] = t; r[1] = hs; r[2] = last ? (double)jn : -1.0; r[3] = t_f; r[4] = h_f;
            }
            float ymx = 0.f;
            for (int i = threadIdx.x; i < N; i += NT) {
                C.y[i] += C.Z[(S - 1) * N + i];
                ymx = nanmax(ymx, fabsf((float)C.y[i]));
            }
            ymax = block_max(ymx, sh.red);
            if (!(ymax <= 3.0e38)) { out.status = FP_STATUS_NONFINITE; break; }
            ++out.nsteps; ++since_fac;
            t = last ? tt : t + hs;
            // f0 = A(t) y at the accepted point, for the next error estimate
            apply_A(C.y, C.f0, s_end, C.diag, N, T);
            __syncthreads();
            if (last) { write_sample(jn, s_end); ++jn; }
            double hn = hs * fmin(4.0, fmax(0.2, fac));
            if (last && hs < h) hn = fac < 1.0 ? fmin(h, hn) : h;
            // keep the factorised step when the controller asks for a small change
            if (fac_valid && hn >= 0.9 * h_f && hn <= 1.2 * h_f) hn = fmax(h_f, hs);
            h = fmin(hn, T_s);
            h_old = hs;
            have_pred = true;
        } else {
            ++out.nrej;
            h = hs * fmax(0.1, fac);
            have_pred = false;
        }
        __syncthreads();
    }
    if (!REC) {
        for (int e = jn * 3 + threadIdx.x; e < A.S_out * 3; e += NT) {
            if (A.m_out) A.m_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
            if (A.dmdt_out) A.dmdt_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
        }
    }
    __syncthreads();
    return out;
}

template <int S, int RS>
// five stages: 128 registers a thread, two CTAs per SM (factors in global memory)
__global__ void __launch_bounds__(NT, S == 5 ? 2 : 1) fp_solve_kernel(KArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared<S> sh;
    Ctx<S> C;
    bind_smem<S, false>(C, smem, A.L_launch, sh, A.fac ? A.fac + (size_t)blockIdx.x * A.fac_stride : nullptr);
    __shared__ int s_slot;
    // instances come either round robin (slot = blockIdx.x + k gridDim.x) or,
    // with a work counter, one at a time in the caller's order, so CTAs that
    // finish early take the next instance (uneven per-instance cost)
    for (int k = 0;; ++k) {
        int slot;
        if (A.queue) {
            if (threadIdx.x == 0) s_slot = atomicAdd(A.queue, 1);
            __syncthreads();
            slot = s_slot;
            __syncthreads();
        } else {
            slot = blockIdx.x + k * gridDim.x;
        }
        if (slot >= A.n) break;
        const int inst = A.order ? A.order[slot] : slot;
        const fp_instance in = A.inst[inst];
        if (!instance_ok(in, A.L_launch)) {
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
        const FpParams P = setup_instance<S>(C, A, in, sh);
        const FwdOut o = forward_instance<S, false, RS>(C, A, inst, P, sh, nullptr, nullptr, 0);
        if (threadIdx.x == 0) {
            A.status[inst] = o.status;
            if (A.stats) {
                A.stats[inst * 4 + 0] = o.nsteps; A.stats[inst * 4 + 1] = o.nrej;
                A.stats[inst * 4 + 2] = o.nit;    A.stats[inst * 4 + 3] = o.nfac;
            }
        }
        __syncthreads();
    }
}

// ============================================================ adjoint =======
// Discrete adjoint of the Radau integration (frozen step sequence).  With
// G = I - h (a x I) blkdiag(A_j) the step is c_{n+1} = e_S^T G^{-1} (1 x c_n), so
//   G^T zeta = e_S x lambda_{n+1},  lambda_n = sum_i zeta_i,
//   dJ/dp += h sum_j xi_j^T (dA_j/dp) Y_j,  xi_j = sum_i a_ij zeta_i,
// plus the readout terms at the sample times and the initial-state term.

// row i of A^T x (FP64) from the column view of the tables
__device__ __forceinline__ double apply_row_T(int i, const double* __restrict__ x, const AScal& sc,
                                              const double* __restrict__ diag, int N, const DevTab& T) {
    double acc = diag[i] * x[i];
#pragma unroll 4
    for (int q = 0; q < FP_NCT; ++q) {
        const FpPair pr = T.colT[(size_t)q * T.nrow + i];
        if ((unsigned)pr.row >= (unsigned)N) continue;
        acc = fma(sc.s[grp_of(pr.slot)] * __ldg(T.coef + (size_t)pr.slot * T.nrow + pr.row), x[pr.row], acc);
    }
    return acc;
}

// derivative scalars of A w.r.t. (K, d, theta, phi) at lab field Blab:
// A = dl*Lap + dw*Wdiag + sum_g s_g T_g with dl = -D, dw = -p4/2
struct DScal { double s[8]; double dl, dw; };

__device__ void dscal_all(const fp_material& mt, const FpParams& P, double d, double th, double ph, const double* Blab,
                          DScal* out) {
    const double gt = mt.gamma / (1.0 + mt.alpha * mt.alpha);
    for (int q = 0; q < 4; ++q) {
        for (int g = 0; g < 8; ++g) out[q].s[g] = 0.0;
        out[q].dl = 0.0;
        out[q].dw = 0.0;
    }
    // K: p3 = 2 gt K / Ms, p4 = alpha p3
    out[0].s[0] = -mt.alpha * gt / mt.Ms;
    out[0].s[1] = -2.0 * gt / mt.Ms;
    out[0].dw = -mt.alpha * gt / mt.Ms;
    // d: D ~ d^-3
    out[1].dl = 3.0 * P.D / d;
    // angles: B' = R(theta, phi) Blab
    const double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
    const double dRt[9] = {-st * cp, -st * sp, -ct, 0.0, 0.0, 0.0, ct * cp, ct * sp, -st};
    const double dRp[9] = {-ct * sp, ct * cp, 0.0, -cp, -sp, 0.0, -st * sp, st * cp, 0.0};
    for (int q = 0; q < 2; ++q) {
        const double* dR = q == 0 ? dRt : dRp;
        double Bp[3];
        for (int r = 0; r < 3; ++r) Bp[r] = dR[3 * r] * Blab[0] + dR[3 * r + 1] * Blab[1] + dR[3 * r + 2] * Blab[2];
        DScal& o = out[2 + q];
        o.s[2] = -P.p1 * Bp[2]; o.s[3] = -P.p1 * Bp[0]; o.s[4] = -P.p1 * Bp[1];
        o.s[5] = -P.p2 * Bp[2]; o.s[6] = -P.p2 * Bp[0]; o.s[7] = -P.p2 * Bp[1];
    }
}

__device__ void lab_field(const KArgs& A, const double* off, double t, double* Bl) {
    const double twopi = 6.283185307179586476925286766559;
    for (int k = 0; k < 3; ++k) Bl[k] = off[k] + A.drv.amp[k] * sin(twopi * A.drv.freq[k] * t + A.drv.phase[k]);
}

// block reduction of 10 doubles per thread; every thread gets the sums
__device__ void block_sum10(double* v, double* red) {
#pragma unroll
    for (int q = 0; q < 10; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(FULLMASK, v[q], o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 10; ++q) red[(threadIdx.x >> 5) * 12 + q] = v[q];
    __syncthreads();
    for (int q = 0; q < 10; ++q) {
        double s = 0.0;
        for (int w = 0; w < NWARP; ++w) s += red[w * 12 + q];
        v[q] = s;
    }
    __syncthreads();
}

// bilinear forms xi^T T_g y per scalar group g (8), xi^T Lap y, xi^T Wdiag y
__device__ void bilinear(const double* xi, const double* yv, int N, const DevTab& T, double* beta) {
    for (int q = 0; q < 10; ++q) beta[q] = 0.0;
    for (int i = threadIdx.x; i < N; i += NT) {
        const double xv = xi[i];
        const double* cf = T.coef + i;
        const int* sr = T.src + i;
#pragma unroll
        for (int k = 0; k < FP_NSLOT; ++k) {
            int j = __ldg(sr + (size_t)k * T.nrow);
            double v = ((unsigned)j < (unsigned)N) ? yv[j] : 0.0;
            beta[grp_of(k)] = fma(xv * __ldg(cf + (size_t)k * T.nrow), v, beta[grp_of(k)]);
        }
        beta[8] = fma(xv * __ldg(T.lam + i), yv[i], beta[8]);
        beta[9] = fma(xv * __ldg(T.wdiag + i), yv[i], beta[9]);
    }
}

__device__ __forceinline__ double dot_dscal(const DScal& d, const double* beta) {
    double s = d.dl * beta[8] + d.dw * beta[9];
    for (int g = 0; g < 8; ++g) s = fma(d.s[g], beta[g], s);
    return s;
}

// Readout at a sample time: u_c = p_c . R^T sqrt(4pi/3) (A(t) c)_{l=1} with the lab
// cotangent g = sum_c (dJ/du_c) p_c.  Adds A^T-term to lambda, direct terms to grad.
template <int S>
__device__ void readout_adjoint(Ctx<S>& C, const KArgs& A, const FpParams& P, const fp_instance& in, const double* R,
                                const double* off, double t, const double* g, const double* cst, double* grad,
                                Shared<S>& sh) {
    const DevTab& T = A.tab;
    const int N = C.N;
    const double sq43 = sqrt(4.0 * 3.14159265358979323846 / 3.0);
    if (threadIdx.x == 0) {
        double Bl[3], Bp[3];
        lab_field(A, off, t, Bl);
        for (int r = 0; r < 3; ++r) Bp[r] = R[3 * r] * Bl[0] + R[3 * r + 1] * Bl[1] + R[3 * r + 2] * Bl[2];
        const AScal sc = make_scal(P, Bp);
        // v' = R g in the easy-axis frame, rows (1,1), (1,-1), (1,0) = x', y', z'
        double vp[3];
        for (int r = 0; r < 3; ++r) vp[r] = R[3 * r] * g[0] + R[3 * r + 1] * g[1] + R[3 * r + 2] * g[2];
        const int rows[3] = {3, 1, 2};
        // lambda += sqrt(4pi/3) A^T e with e_rows = vp  (scatter over the three rows' couplings)
        for (int q = 0; q < 3; ++q) {
            const int r = rows[q];
            const double e = sq43 * vp[q];
            C.lam[r] = fma(C.diag[r], e, C.lam[r]);
            for (int k = 0; k < FP_NSLOT; ++k) {
                int j = __ldg(T.src + (size_t)k * T.nrow + r);
                if ((unsigned)j >= (unsigned)N) continue;
                C.lam[j] = fma(sc.s[grp_of(k)] * __ldg(T.coef + (size_t)k * T.nrow + r), e, C.lam[j]);
            }
        }
        // direct parameter terms: g . dR^T/dp m'dot + sqrt(4pi/3) vp . ((dA/dp) c)_rows
        double mdot[3];
        for (int q = 0; q < 3; ++q) mdot[q] = sq43 * apply_row(rows[q], cst, sc, C.diag, N, T);
        DScal ds[4];
        dscal_all(A.mat, P, in.d, in.theta, in.phi, Bl, ds);
        const double ct = cos(in.theta), stt = sin(in.theta), cp = cos(in.phi), sp = sin(in.phi);
        const double dRt[9] = {-stt * cp, -stt * sp, -ct, 0.0, 0.0, 0.0, ct * cp, ct * sp, -stt};
        const double dRp[9] = {-ct * sp, ct * cp, 0.0, -cp, -sp, 0.0, -stt * sp, stt * cp, 0.0};
        for (int p = 0; p < 4; ++p) {
            double acc = 0.0;
            for (int q = 0; q < 3; ++q) {
                const int r = rows[q];
                double dr = ds[p].dl * __ldg(T.lam + r) * cst[r] + ds[p].dw * __ldg(T.wdiag + r) * cst[r];
                for (int k = 0; k < FP_NSLOT; ++k) {
                    int j = __ldg(T.src + (size_t)k * T.nrow + r);
                    if ((unsigned)j >= (unsigned)N) continue;
                    dr = fma(ds[p].s[grp_of(k)] * __ldg(T.coef + (size_t)k * T.nrow + r), cst[j], dr);
                }
                acc = fma(sq43 * vp[q], dr, acc);
            }
            if (p >= 2) {   // rotation of the output back to the lab frame: m = R^T m'
                const double* dR = p == 2 ? dRt : dRp;
                for (int k = 0; k < 3; ++k) {
                    double dm = dR[k] * mdot[0] + dR[3 + k] * mdot[1] + dR[6 + k] * mdot[2];
                    acc = fma(g[k], dm, acc);
                }
            }
            grad[p] += acc;
        }
    }
    __syncthreads();
}

// transposed stage solve: G^T zeta = e_S x lambda, zeta in C.F, starting from
// zero or (warm) from the zeta already in C.F (the previous step's, or a
// partial solution); stages Z (for the stage times) unchanged; factors
// current.  Returns the iteration count, -1 on a non-finite value, -2 when the
// iteration stalls or does not converge.
template <int S>
__device__ int adjoint_stages(Ctx<S>& C, const DevTab& T, double hs, double h_f, int maxit, Shared<S>& sh,
                              bool warm) {
    constexpr int NC = (S - 1) / 2;
    const int N = C.N, w = threadIdx.x >> 5;
    const float fscale = (float)(h_f / hs);
    if (!warm)
        for (int i = threadIdx.x; i < S * N; i += NT) C.F[i] = 0.0;
    float lm = 0.f;
    for (int i = threadIdx.x; i < N; i += NT) lm = nanmax(lm, fabsf((float)C.lam[i]));
    const float lmax = block_max(lm, sh.red);
    if (lmax == 0.f) return 0;
    if (!(lmax <= 3.0e38f)) return -1;
    float prev = 3.0e38f;
    bool last = false;
    int nflat = 0;
    for (int it = 0; it < maxit; ++it) {
        // v_i = sum_j a_ji zeta_j ; w_i = A_i^T v_i
        for (int e = threadIdx.x; e < S * N; e += NT) {
            const int i = e / N, r = e - i * N;
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < S; ++j) acc = fma(RAD<S>().a[j][i], C.F[j * N + r], acc);
            C.yb[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < S * N; e += NT) {
            const int i = e / N, r = e - i * N;
            C.aw[e] = apply_row_T(r, C.yb + i * N, sh.scj[i], C.diag, N, T);
        }
        __syncthreads();
        // rho_i = delta_iS lambda - zeta_i + h w_i  -> q = Lam^T T^T rho (FP32)
        for (int b = threadIdx.x; b < N; b += NT) {
            const int r = __ldg(C.glob + b);
            float rho[S];
#pragma unroll
            for (int i = 0; i < S; ++i) {
                double v = fma(hs, C.aw[i * N + r], -C.F[i * N + r]);
                if (i == S - 1) v += C.lam[r];
                rho[i] = (float)v;
            }
            float tr[S];           // T^T rho
#pragma unroll
            for (int k = 0; k < S; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < S; ++i) acc = fmaf((float)RAD<S>().T[i][k], rho[i], acc);
                tr[k] = acc;
            }
            // Lam^T: real gam; pairs [[alp, -bet], [bet, alp]]
            C.rr[b] = (float)RAD<S>().gam * tr[0];
#pragma unroll
            for (int p = 0; p < NC; ++p) {
                const float al = (float)RAD<S>().alp[p], be = (float)RAD<S>().bet[p];
                const float q1 = al * tr[1 + 2 * p] - be * tr[2 + 2 * p];
                const float q2 = be * tr[1 + 2 * p] + al * tr[2 + 2 * p];
                C.rc[p * N + b] = make_float2(q1, -q2);        // conjugated for the transposed complex solve
            }
        }
        __syncthreads();
        {
            constexpr int GW = Groups<S>::GW;
            const int sys = w / GW, gw = w - sys * GW;
            if (sys == 0) group_solve<float, S, GW, true>(C, C.fr, C.rr, C.zr, gw, 1);
            else if (sys <= NC)
                group_solve<float2, S, GW, true>(C, C.fc + (size_t)(sys - 1) * C.ly.fsum, C.rc + (sys - 1) * N,
                                                 C.zc + (sys - 1) * N, gw, 1 + sys);
        }
        __syncthreads();
        // zeta += T^{-T} omega (h_f / h)
        float dm = 0.f, zm = 0.f;
        for (int b = threadIdx.x; b < N; b += NT) {
            const int r = __ldg(C.glob + b);
            float om[S];
            om[0] = fscale * C.zr[b];
#pragma unroll
            for (int p = 0; p < NC; ++p) {
                float2 v = C.zc[p * N + b];
                om[1 + 2 * p] = fscale * v.x;
                om[2 + 2 * p] = -fscale * v.y;                  // conjugate back
            }
#pragma unroll
            for (int k = 0; k < S; ++k) {
                float dz = 0.f;
#pragma unroll
                for (int j = 0; j < S; ++j) dz = fmaf((float)RAD<S>().Ti[j][k], om[j], dz);
                C.F[k * N + r] += (double)dz;
                dm = nanmax(dm, fabsf(dz));
                zm = nanmax(zm, fabsf((float)C.F[k * N + r]));
            }
        }
        const float dmax = block_max(dm, sh.red);
        const float zmax = block_max(zm, sh.red);
        if (!(dmax <= 3.0e38f) || !(zmax <= 3.0e38f)) return -1;
        // increments relative to the larger of lambda and zeta (zeta can exceed
        // lambda by the conditioning of the step).  The iteration stagnates
        // when two increments in a row fail to shrink by 1 % (a single
        // non-decreasing increment is common on the way down); it is then
        // accepted once its increments are below 1e-7 of that scale, the
        // single-precision level of the factor solves
        const float scale = fmaxf(lmax, zmax);
        if (dmax <= 1e-10f * scale) return it + 1;
        nflat = (it >= 2 && dmax > 0.99f * prev) ? nflat + 1 : 0;
        if (nflat >= 2) return dmax <= 1e-7f * scale ? it + 1 : -2;   // stagnated
        prev = dmax;
        last = dmax <= 1e-7f * scale;
    }
    return last ? maxit : -2;
}

struct GArgs {
    KArgs A;
    const double* dJ;       // [n][C][K+1][2]
    double* grad;           // [n][4]
    const double* tw;       // twiddles [S_p][2]
    double ch[4][3];
    int C, K;
    double* work;           // per CTA: work_per_cta doubles
    size_t work_per_cta;
    size_t fac_doubles;     // global factors at the head of each CTA's workspace (0: in shared memory)
    int max_rec;
};

template <int S>
__global__ void __launch_bounds__(NT, 1) fp_adjoint_kernel(GArgs G) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared<S> sh;
    __shared__ double s_g[3], s_grad[4];
    const KArgs& A = G.A;
    const DevTab& T = A.tab;
    Ctx<S> C;
    const int Sp = A.drv.samples_per_period, j0 = A.S_out - Sp;
    const int Nmax = (A.L_launch + 1) * (A.L_launch + 1);
    double* ws = G.work + (size_t)blockIdx.x * G.work_per_cta;          // [fac_doubles] factors (5 stages)
    bind_smem<S, true>(C, smem, A.L_launch, sh, G.fac_doubles ? (unsigned char*)ws : nullptr);
    double* ws_steps = ws + G.fac_doubles;                              // [max_rec][FP_REC]
    double* ws_ckpt = ws_steps + (size_t)G.max_rec * FP_REC;            // [max_rec/CKPT + 1][Nmax]
    double* ws_seg = ws_ckpt + (size_t)(G.max_rec / FP_CKPT + 1) * Nmax; // [CKPT + 1][Nmax]
    double* ws_g = ws_seg + (size_t)(FP_CKPT + 1) * Nmax;                // [Sp][3]
    double* ws_Z = ws_g + (size_t)Sp * 3;                                // [CKPT][S][Nmax] stage increments

    for (int inst = blockIdx.x; inst < A.n; inst += gridDim.x) {
        const fp_instance in = A.inst[inst];
        if (!instance_ok(in, A.L_launch)) {
            if (threadIdx.x < 4) G.grad[inst * 4 + threadIdx.x] = 0.0;
            if (threadIdx.x == 0) A.status[inst] = FP_STATUS_BAD_INPUT;
            continue;
        }
        const FpParams P = setup_instance<S>(C, A, in, sh);
        const int N = C.N;
        double R[9], off[3];
        for (int k = 0; k < 9; ++k) R[k] = sh.R[k];
        for (int k = 0; k < 3; ++k) off[k] = sh.off[k];
        // (1) dJ/du_c(t_j) over the last period, as lab vectors g_j = sum_c (dJ/du_c) p_c
        for (int j = threadIdx.x; j < Sp; j += NT) {
            double gv[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c < G.C; ++c) {
                const double* dj = G.dJ + (((size_t)inst * G.C + c) * (G.K + 1)) * 2;
                double acc = 0.0;
                int q = 0;
                for (int k = 0; k <= G.K; ++k) {
                    acc = fma(dj[2 * k], G.tw[2 * q], acc);
                    acc = fma(-dj[2 * k + 1], G.tw[2 * q + 1], acc);
                    q += j;
                    if (q >= Sp) q -= Sp;
                }
                acc /= (double)Sp;
                for (int k = 0; k < 3; ++k) gv[k] = fma(acc, G.ch[c][k], gv[k]);
            }
            for (int k = 0; k < 3; ++k) ws_g[j * 3 + k] = gv[k];
        }
        __syncthreads();
        // (2) forward pass recording steps and checkpoints
        const FwdOut fo = forward_instance<S, true>(C, A, inst, P, sh, ws_steps, ws_ckpt, G.max_rec);
        int status = fo.status;
        const int nacc = fo.nsteps;
        if (threadIdx.x < 4) s_grad[threadIdx.x] = 0.0;
        for (int i = threadIdx.x; i < N; i += NT) C.lam[i] = 0.0;
        __syncthreads();
        // (3) backward sweep, segment by segment
        double sc_rep = A.tol.atol;                // replay Newton tolerance, set per segment
        // the iteration matrices of every replayed and transposed step are the
        // forward's: refactorised whenever the recorded factor point changes
        bool fac_valid = false;
        double h_f = 0.0, t_fc = 0.0;
        int fail_phase = 0, fail_step = -1;
        const int nseg = (nacc + FP_CKPT - 1) / FP_CKPT;
        for (int sg = nseg - 1; sg >= 0 && status == FP_STATUS_OK; --sg) {
            const int n0 = sg * FP_CKPT, n1 = min(nacc, n0 + FP_CKPT);
            // replay the segment from its checkpoint, keeping every state and
            // every step's stage increments
            float ym = 0.f;
            for (int i = threadIdx.x; i < N; i += NT) {
                C.y[i] = ws_ckpt[(size_t)sg * N + i]; ws_seg[i] = C.y[i];
                ym = nanmax(ym, fabsf((float)C.y[i]));
            }
            // the forward's Newton tolerance: replayed states stay within the
            // forward's own iteration error of the recorded path
            sc_rep = A.tol.atol + A.tol.rtol * (double)block_max(ym, sh.red);
            fac_valid = false;                     // the last factors belong to a later time
            double h_prev = 0.0;                   // the previous replayed step (its stages are in Z)
            for (int n = n0; n < n1; ++n) {
                const double* rs = ws_steps + (size_t)n * FP_REC;
                const double t = rs[0], hs = rs[1];
                if (!fac_valid || rs[3] != t_fc || rs[4] != h_f) {
                    refactor<S>(C, A, P, R, off, rs[3], rs[4], sh);
                    t_fc = rs[3]; h_f = rs[4]; fac_valid = true;
                }
                // start from the previous step's collocation polynomial, as the
                // forward pass did (accepted steps are contiguous)
                const bool pred = h_prev > 0.0;
                stage_scalars<S>(A, P, R, off, t, hs, pred, pred ? h_prev : 1.0, sh);
                predict_stages<S>(C, pred, sh);
                float eta = 1.f;
                NewtonResult nr = newton_stages<S>(C, T, hs, h_f, sc_rep, eta, 0.02f, 4 * A.tol.newton_max_iter, sh);
                // a stalled iteration whose last increment is already below the
                // tolerance scale is as good as the forward's accepted stages;
                // otherwise (the forward reached these stages from a better
                // predictor) retry from zero with factors made for this very step
                if (!nr.nonfinite && !nr.conv && !(nr.dmax <= (float)sc_rep)) {
                    refactor<S>(C, A, P, R, off, t, hs, sh);
                    t_fc = t; h_f = hs;
                    stage_scalars<S>(A, P, R, off, t, hs, false, 1.0, sh);
                    predict_stages<S>(C, false, sh);
                    eta = 1.f;
                    nr = newton_stages<S>(C, T, hs, h_f, sc_rep, eta, 0.02f, 4 * A.tol.newton_max_iter, sh);
                }
                if (nr.nonfinite || (!nr.conv && !(nr.dmax <= (float)sc_rep))) {
                    status = nr.nonfinite ? FP_STATUS_NONFINITE : FP_STATUS_NEWTON_FAIL;
                    fail_phase = 2; fail_step = n;
                    break;
                }
                h_prev = hs;
                double* zs = ws_Z + (size_t)(n - n0) * S * N;
                for (int e = threadIdx.x; e < S * N; e += NT) zs[e] = C.Z[e];
                for (int i = threadIdx.x; i < N; i += NT) {
                    C.y[i] += C.Z[(S - 1) * N + i];
                    ws_seg[(size_t)(n - n0 + 1) * N + i] = C.y[i];
                }
                __syncthreads();
            }
            if (status != FP_STATUS_OK) break;
            fac_valid = false;
            for (int n = n1 - 1; n >= n0; --n) {
                const double* rs = ws_steps + (size_t)n * FP_REC;
                const double t = rs[0], hs = rs[1];
                const int js = (int)rs[2];
                // readout at t + hs if this step landed on a sample of the last period
                if (js >= j0) {
                    if (threadIdx.x < 3) s_g[threadIdx.x] = ws_g[(js - j0) * 3 + threadIdx.x];
                    __syncthreads();
                    double gl[3] = {s_g[0], s_g[1], s_g[2]};
                    double grad_loc[4] = {0, 0, 0, 0};
                    readout_adjoint<S>(C, A, P, in, R, off, t + hs, gl, ws_seg + (size_t)(n - n0 + 1) * N, grad_loc, sh);
                    if (threadIdx.x == 0) for (int p = 0; p < 4; ++p) s_grad[p] += grad_loc[p];
                    __syncthreads();
                }
                // state c_n and the replayed stage increments of step n
                const double* zs = ws_Z + (size_t)(n - n0) * S * N;
                for (int i = threadIdx.x; i < N; i += NT) C.y[i] = ws_seg[(size_t)(n - n0) * N + i];
                for (int e = threadIdx.x; e < S * N; e += NT) C.Z[e] = zs[e];
                __syncthreads();
                if (!fac_valid || rs[3] != t_fc || rs[4] != h_f) {
                    refactor<S>(C, A, P, R, off, rs[3], rs[4], sh);
                    t_fc = rs[3]; h_f = rs[4]; fac_valid = true;
                }
                stage_scalars<S>(A, P, R, off, t, hs, false, 1.0, sh);
                // transposed stage solve for zeta (in F), started from the
                // previous step's zeta inside a segment (the segment replay
                // reuses F); a slow iteration with the forward's factors is
                // continued with factors made for this step
                int ai = adjoint_stages<S>(C, T, hs, h_f, 4 * A.tol.newton_max_iter, sh, n != n1 - 1);
                if (ai == -2) {
                    refactor<S>(C, A, P, R, off, t, hs, sh);
                    t_fc = t; h_f = hs;
                    stage_scalars<S>(A, P, R, off, t, hs, false, 1.0, sh);
                    ai = adjoint_stages<S>(C, T, hs, h_f, 16 * A.tol.newton_max_iter, sh, true);
                }
                if (ai < 0) {
                    status = ai == -1 ? FP_STATUS_NONFINITE : FP_STATUS_NEWTON_FAIL;
                    fail_phase = 3; fail_step = n;
                    break;
                }
                // gradient: h sum_j xi_j^T (dA_j/dp) Y_j with xi_j = sum_i a_ij zeta_i, Y_j = c_n + Z_j
                double gacc[4] = {0, 0, 0, 0};
                for (int j = 0; j < S; ++j) {
                    for (int i = threadIdx.x; i < N; i += NT) {
                        double xv = 0.0;
#pragma unroll
                        for (int k = 0; k < S; ++k) xv = fma(RAD<S>().a[k][j], C.F[k * N + i], xv);
                        C.yb[i] = xv;                                   // xi_j
                        C.aw[i] = C.y[i] + C.Z[j * N + i];              // Y_j
                    }
                    __syncthreads();
                    double beta[10];
                    bilinear(C.yb, C.aw, N, T, beta);
                    block_sum10(beta, sh.dred);
                    double Bl[3];
                    lab_field(A, off, t + RAD<S>().c[j] * hs, Bl);
                    DScal ds[4];
                    dscal_all(A.mat, P, in.d, in.theta, in.phi, Bl, ds);
                    for (int p = 0; p < 4; ++p) gacc[p] += hs * dot_dscal(ds[p], beta);
                }
                if (threadIdx.x == 0) for (int p = 0; p < 4; ++p) s_grad[p] += gacc[p];
                // lambda_n = sum_i zeta_i
                for (int i = threadIdx.x; i < N; i += NT) {
                    double v = 0.0;
#pragma unroll
                    for (int k = 0; k < S; ++k) v += C.F[k * N + i];
                    C.lam[i] = v;
                }
                __syncthreads();
            }
        }
        if (status == FP_STATUS_OK) {
            // readout at t = 0 when the schedule samples it (and it lies in the last period)
            if (sample_time(A.drv, 0) <= 0.0 && j0 == 0) {
                if (threadIdx.x < 3) s_g[threadIdx.x] = ws_g[threadIdx.x];
                for (int i = threadIdx.x; i < N; i += NT) C.y[i] = ws_ckpt[i];
                __syncthreads();
                double gl[3] = {s_g[0], s_g[1], s_g[2]};
                double grad_loc[4] = {0, 0, 0, 0};
                readout_adjoint<S>(C, A, P, in, R, off, 0.0, gl, C.y, grad_loc, sh);
                if (threadIdx.x == 0) for (int p = 0; p < 4; ++p) s_grad[p] += grad_loc[p];
                __syncthreads();
            }
            // initial state: lambda_0^T dc_0/dp by central differences of the projection
            double Bl[3];
            lab_field(A, off, 0.0, Bl);
            for (int p = 0; p < 4; ++p) {
                double val[2];
                const double base = p == 0 ? in.K : p == 1 ? in.d : p == 2 ? in.theta : in.phi;
                const double dp = p <= 1 ? 1e-5 * fmax(fabs(base), p == 0 ? 1.0 : 1e-9) : 1e-5;
                for (int sgn = 0; sgn < 2; ++sgn) {
                    const double v = base + (sgn == 0 ? dp : -dp);
                    const double K = p == 0 ? v : in.K, d = p == 1 ? v : in.d;
                    const double th = p == 2 ? v : in.theta, ph = p == 3 ? v : in.phi;
                    const FpParams Pp = fp_derive(A.mat, K, d);
                    double Rp[9], Bp[3];
                    fp_rotation(th, ph, Rp);
                    for (int r = 0; r < 3; ++r) Bp[r] = Rp[3 * r] * Bl[0] + Rp[3 * r + 1] * Bl[1] + Rp[3 * r + 2] * Bl[2];
                    initial_state<S>(C, Pp, Bp, smem, C.yb);
                    double part = 0.0;
                    for (int i = threadIdx.x; i < N; i += NT) part = fma(C.lam[i], C.yb[i], part);
                    double tmp[10] = {part, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                    block_sum10(tmp, sh.dred);
                    val[sgn] = tmp[0];
                }
                if (threadIdx.x == 0) s_grad[p] += (val[0] - val[1]) / (2.0 * dp);
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            A.status[inst] = status;
            for (int p = 0; p < 4; ++p) G.grad[inst * 4 + p] = status == FP_STATUS_OK ? s_grad[p] : 0.0;
            if (A.stats) {
                A.stats[inst * 4 + 0] = fo.nsteps; A.stats[inst * 4 + 1] = fo.nrej;
                A.stats[inst * 4 + 2] = fo.status != FP_STATUS_OK ? 1 : fail_phase;
                A.stats[inst * 4 + 3] = fail_step;
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------- host launch ----
int fp_launch_solve(int stages, const DevTab* tab, const DevBlk* blk, const fp_material* mat, const fp_drive* drv,
                    const fp_tol* tol, const fp_instance* d_inst, int n, int L_launch, double* d_m, double* d_dmdt,
                    int* d_status, int* d_stats, int num_sms, cudaStream_t st, const int* d_order, int* d_queue,
                    unsigned char* d_fac) {
    KArgs A;
    A.order = d_order;
    A.queue = d_queue;
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
    A.fac = nullptr;
    A.fac_stride = 0;
    cudaError_t e;
    if (L_launch > FP_L_SMEM) {
        // blocks of up to 2 L_launch <= 64 rows (two row slots per lane), factors in
        // this launch's global scratch, one CTA per SM (one scratch slot each)
        if (stages != 3 || !d_fac) return FP_EUNSUPPORTED;
        A.fac = d_fac;
        A.fac_stride = fp_solver_fac_bytes(3, L_launch);
        const size_t sm = fp_solver_smem_bytes(3, L_launch);
        e = cudaFuncSetAttribute(fp_solve_kernel<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        const int grid = n < num_sms ? n : num_sms;
        fp_solve_kernel<3, 2><<<grid, NT, sm, st>>>(A);
        return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
    }
    if (stages == 5) {
        // one global factor slot per CTA, up to two CTAs per SM
        if (!d_fac) return FP_EUNSUPPORTED;
        A.fac = d_fac;
        A.fac_stride = fp_solver_fac_bytes(5, L_launch);
        const size_t sm = fp_solver_smem_bytes(5, L_launch);
        e = cudaFuncSetAttribute(fp_solve_kernel<5, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp_solve_kernel<5, 1>, NT, sm) != cudaSuccess)
            per_sm = 1;
        const int slots = fp_solver_ctas_per_sm(5, L_launch);
        per_sm = per_sm < 1 ? 1 : (per_sm > slots ? slots : per_sm);
        const int cap = per_sm * num_sms;
        const int grid = n < cap ? n : cap;
        fp_solve_kernel<5, 1><<<grid, NT, sm, st>>>(A);
        return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
    }
    // stages 3: as many CTAs per SM as registers and shared memory allow
    // (one at the kernel's register budget)
    const size_t sm = make_layout<3>(L_launch).total;
    int per_sm = 0;
    cudaFuncSetAttribute(fp_solve_kernel<3, 1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    e = cudaFuncSetAttribute(fp_solve_kernel<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return FP_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp_solve_kernel<3, 1>, NT, sm) != cudaSuccess) per_sm = 1;
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    const int cap = per_sm * num_sms;
    const int grid = n < cap ? n : cap;
    fp_solve_kernel<3, 1><<<grid, NT, sm, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
}

size_t fp_adjoint_work_doubles_per_cta(int stages, int L_max, int S_p, int max_rec) {
    const size_t Nmax = (size_t)(L_max + 1) * (L_max + 1);
    const size_t d = adjoint_fac_doubles(stages, L_max) + (size_t)max_rec * FP_REC +
                     (size_t)(max_rec / FP_CKPT + 1) * Nmax + (size_t)(FP_CKPT + 1) * Nmax + (size_t)S_p * 3 +
                     (size_t)FP_CKPT * stages * Nmax;
    return (d + 1) & ~(size_t)1;                      // even: CTA slots stay 16-byte aligned
}

int fp_launch_adjoint(int stages, const DevTab* tab, const DevBlk* blk, const fp_material* mat, const fp_drive* drv,
                      const fp_tol* tol, const fp_instance* d_inst, int n, int L_launch, int k_max,
                      const double* channels, int C, const double* d_dJ, const double* d_tw, double* d_grad,
                      int* d_status, int* d_stats, double* d_work, int max_rec, int grid, cudaStream_t st) {
    GArgs G;
    KArgs& A = G.A;
    A.order = nullptr;
    A.queue = nullptr;
    A.tab = *tab;
    A.blk = *blk;
    A.mat = *mat;
    A.drv = *drv;
    A.tol = *tol;
    A.inst = d_inst;
    A.n = n;
    A.m_out = nullptr;
    A.dmdt_out = nullptr;
    A.status = d_status;
    A.stats = d_stats;
    A.S_out = drv->output_periods * drv->samples_per_period;
    A.L_launch = L_launch;
    G.dJ = d_dJ;
    G.grad = d_grad;
    G.tw = d_tw;
    for (int c = 0; c < 4; ++c)
        for (int k = 0; k < 3; ++k) G.ch[c][k] = c < C ? channels[3 * c + k] : 0.0;
    G.C = C;
    G.K = k_max;
    G.work = d_work;
    G.max_rec = max_rec;
    G.work_per_cta = fp_adjoint_work_doubles_per_cta(stages, L_launch, drv->samples_per_period, max_rec);
    G.fac_doubles = adjoint_fac_doubles(stages, L_launch);
    size_t sm = fp_adjoint_smem_bytes(stages, L_launch);
    cudaError_t e;
    if (stages == 5) {
        e = cudaFuncSetAttribute(fp_adjoint_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        fp_adjoint_kernel<5><<<grid, NT, sm, st>>>(G);
    } else {
        e = cudaFuncSetAttribute(fp_adjoint_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return FP_ECUDA;
        fp_adjoint_kernel<3><<<grid, NT, sm, st>>>(G);
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
