// Batched Fokker-Planck solver for Neel rotation (Sec. 2.1, Eq. FP-general,
// Eq. convection, Eq. mean_magmom_FP) on sm_103a.
//
// One CTA owns one instance at a time (persistent loop over instances).  The
// real-SH coefficient vector c (N = (L+1)^2 doubles) and every Radau stage
// live in shared memory; nothing is streamed from HBM per step except the
// (L1/L2-resident) closed-form coupling tables shared by all instances.
//
// Time step: 3-stage Radau IIA (order 5, L-stable), simplified Newton:
//   residual  R_i = -Z_i + h sum_j a_ij A(t + c_j h)(y + Z_j)        FP64
//   correction (Lam - h_f Abar) dW = K R,  dZ = T dW (h_f / h)         FP32
// where Abar = A(t_f + h_f) is frozen for up to refactor_every steps and the
// block-tridiagonal (in |m|) matrices Lam - h_f Abar (one real, one complex
// shift) are factorised in FP32 as explicit inverses of their Schur-complement
// diagonal blocks (block Thomas; warp-level Gauss-Jordan with partial
// pivoting).  Embedded error estimate filtered through the real factor;
// steps land on every output sample time.
#include <cuda_runtime.h>
#include <stdint.h>
#include "fp_internal.h"

#define NT 256
#define NWARP (NT / 32)
#define NLAT 12          // lateral slots SL_RX..SL_RY+1 (4) and SL_GX..SL_GY+3 (8)
#define FULLMASK 0xffffffffu

__constant__ FpRadau c_rad;
__constant__ double c_glx[FP_NGL];
__constant__ double c_glw[FP_NGL];

struct DevTab {
    const double* coef;
    const int* src;
    const int* tslot;
    const double* lam;
    const double* wdiag;
};

struct KArgs {
    DevTab tab;
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
// lateral slot index (0..11) of slot k, or -1
__host__ __device__ constexpr int lat_of(int k) {
    return (k >= SL_RX && k < SL_GZ) ? k - SL_RX : (k >= SL_GX ? k - SL_GX + 4 : -1);
}
__host__ __device__ constexpr int slot_of_lat(int q) { return q < 4 ? SL_RX + q : SL_GX + (q - 4); }

struct AScal { double s[8]; };

// ---------------------------------------------------------------- layout ----
struct Layout {
    int N, L, nmax;
    size_t y, Z, F, tmp, yb, diag, rr, rc, zr, zc, latv, fr, fc, s1r, s2r, s1c, s2c, ic, total;
};

__host__ __device__ inline int nblk(int mu, int L) { return mu == 0 ? L + 1 : 2 * (L + 1 - mu); }

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Layout make_layout(int L) {
    Layout ly;
    ly.L = L;
    ly.N = (L + 1) * (L + 1);
    ly.nmax = L >= 1 ? (2 * L > L + 1 ? 2 * L : L + 1) : 1;
    size_t fsum = 0;
    for (int mu = 0; mu <= L; ++mu) fsum += (size_t)nblk(mu, L) * nblk(mu, L);
    size_t o = 0;
    const size_t N = ly.N, nm2 = (size_t)ly.nmax * ly.nmax;
    ly.y = o;    o = al16(o + N * 8);
    ly.Z = o;    o = al16(o + 3 * N * 8);
    ly.F = o;    o = al16(o + 3 * N * 8);
    ly.tmp = o;  o = al16(o + N * 8);
    ly.yb = o;   o = al16(o + N * 8);
    ly.diag = o; o = al16(o + N * 8);
    ly.rr = o;   o = al16(o + N * 4);
    ly.rc = o;   o = al16(o + N * 8);
    ly.zr = o;   o = al16(o + N * 4);
    ly.zc = o;   o = al16(o + N * 8);
    ly.latv = o; o = al16(o + N * NLAT * 4);
    ly.fr = o;   o = al16(o + fsum * 4);
    ly.fc = o;   o = al16(o + fsum * 8);
    ly.s1r = o;  o = al16(o + nm2 * 4);
    ly.s2r = o;  o = al16(o + nm2 * 4);
    ly.s1c = o;  o = al16(o + nm2 * 8);
    ly.s2c = o;  o = al16(o + nm2 * 8);
    ly.ic = ly.fr;                                    // initial-state scratch aliases the factors
    size_t ic_end = ly.ic + (size_t)FP_NGL * (L + 1) * 8;
    ly.total = o > ic_end ? o : al16(ic_end);
    return ly;
}

size_t fp_solver_smem_bytes(int L) { return make_layout(L).total; }

// ------------------------------------------------------------- helpers ----
__device__ __forceinline__ int isqrt_i(int g) {
    int l = (int)sqrtf((float)g + 0.5f);
    while ((l + 1) * (l + 1) <= g) ++l;
    while (l * l > g) --l;
    return l;
}
__device__ __forceinline__ void glob_to_blk(int g, int& mu, int& k) {
    int l = isqrt_i(g), m = g - l * l - l;
    mu = m < 0 ? -m : m;
    k = mu == 0 ? l : 2 * (l - mu) + (m < 0 ? 1 : 0);
}
__device__ __forceinline__ int blk_to_glob(int mu, int k) {
    if (mu == 0) return k * k + k;
    int l = mu + (k >> 1), m = (k & 1) ? -mu : mu;
    return l * l + l + m;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {   // a*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

__device__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULLMASK, v, o));
    int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    __syncthreads();
    if (ln == 0) red[w] = v;
    __syncthreads();
    float r = red[0];
    for (int i = 1; i < NWARP; ++i) r = fmaxf(r, red[i]);
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

// y = A x for rows i = tid, tid+nthr, ... (FP64, matrix-free from the tables)
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

// ------------------------------------------------- warp Gauss-Jordan ------
// In-place inversion of an n x n (n <= 32) matrix S (row-major) with partial
// pivoting; lane r holds row r in registers.  The inverse is stored
// column-major (out[c * n + r] = Inv[r][c]) for conflict-free matvecs.
__device__ void warp_gj_real(const float* S, float* out, int n, int* pp) {
    const int lane = threadIdx.x & 31;
    float a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) a[j] = (lane < n && j < n) ? S[lane * n + j] : (j == lane ? 1.f : 0.f);
    bool used = lane >= n;
    int myk = -1;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k < n) {
            float v = used ? 0.f : fabsf(a[k]);
            unsigned key = (__float_as_uint(v) & ~31u) | (unsigned)lane;
            key = __reduce_max_sync(FULLMASK, key);
            int p = (int)(key & 31u);
            if (lane == 0) pp[k] = p;
            float pk = __shfl_sync(FULLMASK, a[k], p);
            float pinv = 1.f / pk;
            float f = a[k];
            bool ispiv = lane == p;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j == k) continue;
                float prj = __shfl_sync(FULLMASK, a[j], p);
                a[j] = ispiv ? prj * pinv : fmaf(-f * pinv, prj, a[j]);
            }
            a[k] = ispiv ? pinv : -f * pinv;
            if (ispiv) { used = true; myk = k; }
        }
    }
    __syncwarp();
    if (lane < n && myk >= 0 && myk < n) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < n && pp[j] < n) out[pp[j] * n + myk] = a[j];   // pp[j] >= n only for a singular block
    }
    __syncwarp();
}

__device__ void warp_gj_cplx(const float2* S, float2* out, int n, int* pp) {
    const int lane = threadIdx.x & 31;
    float2 a[32];
#pragma unroll
    for (int j = 0; j < 32; ++j)
        a[j] = (lane < n && j < n) ? S[lane * n + j] : make_float2(j == lane ? 1.f : 0.f, 0.f);
    bool used = lane >= n;
    int myk = -1;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k < n) {
            float v = used ? 0.f : fabsf(a[k].x) + fabsf(a[k].y);
            unsigned key = (__float_as_uint(v) & ~31u) | (unsigned)lane;
            key = __reduce_max_sync(FULLMASK, key);
            int p = (int)(key & 31u);
            if (lane == 0) pp[k] = p;
            float2 pk = make_float2(__shfl_sync(FULLMASK, a[k].x, p), __shfl_sync(FULLMASK, a[k].y, p));
            float d = 1.f / (pk.x * pk.x + pk.y * pk.y);
            float2 pinv = make_float2(pk.x * d, -pk.y * d);
            float2 f = a[k];
            float2 fp = cmul(f, pinv);
            bool ispiv = lane == p;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j == k) continue;
                float2 prj = make_float2(__shfl_sync(FULLMASK, a[j].x, p), __shfl_sync(FULLMASK, a[j].y, p));
                a[j] = ispiv ? cmul(prj, pinv) : cfma(make_float2(-fp.x, -fp.y), prj, a[j]);
            }
            a[k] = ispiv ? pinv : make_float2(-fp.x, -fp.y);
            if (ispiv) { used = true; myk = k; }
        }
    }
    __syncwarp();
    if (lane < n && myk >= 0 && myk < n) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < n && pp[j] < n) out[pp[j] * n + myk] = a[j];   // pp[j] >= n only for a singular block
    }
    __syncwarp();
}

// ------------------------------------------------------- per-CTA state ----
struct Ctx {
    Layout ly;
    int L, N;
    double* y; double* Z; double* F; double* tmp; double* yb; double* diag;
    float* rr; float2* rc; float* zr; float2* zc; float* latv;
    float* fr; float2* fc; float* s1r; float* s2r; float2* s1c; float2* s2c;
    int* boff; int* foff;
};

// latv[i][q] = entry of (shift - h Abar) at row i, lateral slot q (= -h Abar_ij)
__device__ void build_latv(Ctx& C, const DevTab& T, const AScal& sc, double h) {
    for (int e = threadIdx.x; e < C.N * NLAT; e += NT) {
        int i = e / NLAT, q = e - i * NLAT, k = slot_of_lat(q);
        int j = __ldg(T.src + (size_t)i * FP_NSLOT + k);
        float v = 0.f;
        if ((unsigned)j < (unsigned)C.N)
            v = (float)(-h * sc.s[grp_of(k)] * __ldg(T.coef + (size_t)i * FP_NSLOT + k));
        C.latv[e] = v;
    }
}

// Factorise (gam - h Abar) [real] and ((alp - i bet) - h Abar) [complex].
__device__ void factorize(Ctx& C, const DevTab& T, const AScal& sc, double h, int* pp) {
    const int L = C.L, N = C.N;
    const float gam = (float)c_rad.gam, alp = (float)c_rad.alp, bet = (float)c_rad.bet;
    build_latv(C, T, sc, h);
    __syncthreads();
    for (int mu = 0; mu <= L; ++mu) {
        const int n = nblk(mu, L);
        // (1) diagonal block D_mu of the shifted matrix
        for (int e = threadIdx.x; e < n * n; e += NT) { C.s1r[e] = 0.f; C.s1c[e] = make_float2(0.f, 0.f); }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += NT) {
            int g = blk_to_glob(mu, r);
            float vd = (float)(-h * C.diag[g]);
            C.s1r[r * n + r] += gam + vd;
            C.s1c[r * n + r] = make_float2(C.s1c[r * n + r].x + alp + vd, C.s1c[r * n + r].y - bet);
            const double* cf = T.coef + (size_t)g * FP_NSLOT;
            const int* sr = T.src + (size_t)g * FP_NSLOT;
#pragma unroll
            for (int k = 0; k < SL_RX; ++k) {                       // W, ZR, RZ: same |m|
                int j = __ldg(sr + k);
                if ((unsigned)j >= (unsigned)N) continue;
                int mj, kj;
                glob_to_blk(j, mj, kj);
                float v = (float)(-h * sc.s[grp_of(k)] * __ldg(cf + k));
                C.s1r[r * n + kj] += v;
                C.s1c[r * n + kj].x += v;
            }
#pragma unroll
            for (int k = SL_GZ; k < SL_GX; ++k) {                   // GZ: same |m|
                int j = __ldg(sr + k);
                if ((unsigned)j >= (unsigned)N) continue;
                int mj, kj;
                glob_to_blk(j, mj, kj);
                float v = (float)(-h * sc.s[grp_of(k)] * __ldg(cf + k));
                C.s1r[r * n + kj] += v;
                C.s1c[r * n + kj].x += v;
            }
        }
        __syncthreads();
        // Schur complement: D~ = D - C_mu X_{mu-1},  X_{mu-1} = Inv_{mu-1} B_{mu-1} in s2
        if (mu > 0) {
            const int np = nblk(mu - 1, L);
            for (int e = threadIdx.x; e < n * n; e += NT) {
                int r = e / n, c = e - r * n;
                int g = blk_to_glob(mu, r);
                float ar = 0.f;
                float2 ac = make_float2(0.f, 0.f);
                for (int q = 0; q < NLAT; ++q) {
                    int j = __ldg(T.src + (size_t)g * FP_NSLOT + slot_of_lat(q));
                    if ((unsigned)j >= (unsigned)N) continue;
                    int mj, kj;
                    glob_to_blk(j, mj, kj);
                    if (mj != mu - 1) continue;
                    float v = C.latv[g * NLAT + q];
                    ar = fmaf(v, C.s2r[kj * n + c], ar);
                    ac.x = fmaf(v, C.s2c[kj * n + c].x, ac.x);
                    ac.y = fmaf(v, C.s2c[kj * n + c].y, ac.y);
                }
                C.s1r[e] -= ar;
                C.s1c[e].x -= ac.x;
                C.s1c[e].y -= ac.y;
            }
            (void)np;
            __syncthreads();
        }
        // (2) invert the two diagonal blocks, one warp each
        const int w = threadIdx.x >> 5;
        if (w == 0) warp_gj_real(C.s1r, C.fr + C.foff[mu], n, pp);
        else if (w == 1) warp_gj_cplx(C.s1c, C.fc + C.foff[mu], n, pp + 32);
        __syncthreads();
        // (3) X_mu = Inv_mu B_mu (n x n2) for the next block
        if (mu < L) {
            const int n2 = nblk(mu + 1, L);
            const float* Ir = C.fr + C.foff[mu];
            const float2* Ic = C.fc + C.foff[mu];
            for (int e = threadIdx.x; e < n * n2; e += NT) {
                int r = e / n2, c = e - r * n2;
                int gc = blk_to_glob(mu + 1, c);
                float ar = 0.f;
                float2 ac = make_float2(0.f, 0.f);
                for (int q = 0; q < NLAT; ++q) {
                    int s = slot_of_lat(q);
                    int j = __ldg(T.src + (size_t)gc * FP_NSLOT + s);
                    if ((unsigned)j >= (unsigned)N) continue;
                    int mj, kj;
                    glob_to_blk(j, mj, kj);
                    if (mj != mu) continue;
                    int t = __ldg(T.tslot + (size_t)gc * FP_NSLOT + s);
                    // B_mu[kj][c]; no back-slot means a structurally zero entry
                    // (row (0,0) of A vanishes: conservation of mass)
                    float bval = t >= 0 ? C.latv[j * NLAT + lat_of(t)] : 0.f;
                    ar = fmaf(Ir[kj * n + r], bval, ar);            // Inv[r][kj]
                    ac = cfma(Ic[kj * n + r], make_float2(bval, 0.f), ac);
                }
                C.s2r[r * n2 + c] = ar;
                C.s2c[r * n2 + c] = ac;
            }
            __syncthreads();
        }
    }
}

// Block-Thomas solve with the explicit block inverses; rr/rc hold the right-hand
// sides in block order, the solutions end in zr/zc.  Real rows run on warps
// 0-3, complex rows on warps 4-7.
__device__ void solve_blocks(Ctx& C, const DevTab& T, bool do_cplx) {
    const int L = C.L, N = C.N;
    const int half = NT / 2;
    const bool is_c = threadIdx.x >= half;
    const int tl = is_c ? threadIdx.x - half : threadIdx.x;
    if (is_c && !do_cplx) {
        // still take part in every barrier below
    }
    for (int mu = 0; mu <= L; ++mu) {
        const int n = nblk(mu, L), bo = C.boff[mu];
        if (mu > 0) {
            const int bp = C.boff[mu - 1];
            for (int r = tl; r < n; r += half) {
                if (is_c && !do_cplx) break;
                int g = blk_to_glob(mu, r);
                float ar = 0.f;
                float2 ac = make_float2(0.f, 0.f);
                for (int q = 0; q < NLAT; ++q) {
                    int j = __ldg(T.src + (size_t)g * FP_NSLOT + slot_of_lat(q));
                    if ((unsigned)j >= (unsigned)N) continue;
                    int mj, kj;
                    glob_to_blk(j, mj, kj);
                    if (mj != mu - 1) continue;
                    float v = C.latv[g * NLAT + q];
                    if (is_c) ac = cfma(make_float2(v, 0.f), C.zc[bp + kj], ac);
                    else ar = fmaf(v, C.zr[bp + kj], ar);
                }
                if (is_c) { C.rc[bo + r].x -= ac.x; C.rc[bo + r].y -= ac.y; }
                else C.rr[bo + r] -= ar;
            }
            __syncthreads();
        }
        const int fo = C.foff[mu];
        for (int r = tl; r < n; r += half) {
            if (is_c && !do_cplx) break;
            if (is_c) {
                float2 acc = make_float2(0.f, 0.f);
                for (int c = 0; c < n; ++c) acc = cfma(C.fc[fo + c * n + r], C.rc[bo + c], acc);
                C.zc[bo + r] = acc;
            } else {
                float acc = 0.f;
                for (int c = 0; c < n; ++c) acc = fmaf(C.fr[fo + c * n + r], C.rr[bo + c], acc);
                C.zr[bo + r] = acc;
            }
        }
        __syncthreads();
    }
    for (int mu = L - 1; mu >= 0; --mu) {
        const int n = nblk(mu, L), bo = C.boff[mu], bn = C.boff[mu + 1];
        for (int r = tl; r < n; r += half) {
            if (is_c && !do_cplx) break;
            int g = blk_to_glob(mu, r);
            float ar = 0.f;
            float2 ac = make_float2(0.f, 0.f);
            for (int q = 0; q < NLAT; ++q) {
                int j = __ldg(T.src + (size_t)g * FP_NSLOT + slot_of_lat(q));
                if ((unsigned)j >= (unsigned)N) continue;
                int mj, kj;
                glob_to_blk(j, mj, kj);
                if (mj != mu + 1) continue;
                float v = C.latv[g * NLAT + q];
                if (is_c) ac = cfma(make_float2(v, 0.f), C.zc[bn + kj], ac);
                else ar = fmaf(v, C.zr[bn + kj], ar);
            }
            if (is_c) C.rc[bo + r] = ac;
            else C.rr[bo + r] = ar;
        }
        __syncthreads();
        const int fo = C.foff[mu];
        for (int r = tl; r < n; r += half) {
            if (is_c && !do_cplx) break;
            if (is_c) {
                float2 acc = make_float2(0.f, 0.f);
                for (int c = 0; c < n; ++c) acc = cfma(C.fc[fo + c * n + r], C.rc[bo + c], acc);
                C.zc[bo + r].x -= acc.x;
                C.zc[bo + r].y -= acc.y;
            } else {
                float acc = 0.f;
                for (int c = 0; c < n; ++c) acc = fmaf(C.fr[fo + c * n + r], C.rr[bo + c], acc);
                C.zr[bo + r] -= acc;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------- initial state -----
// Projection of the Boltzmann density f ~ exp(bT B.m + sigma z^2) (easy-axis
// frame) on the real SH basis.  The azimuthal integral is exact through the
// modified Bessel functions: int exp(k cos(p - pB)) cos(mu p) dp = 2 pi I_mu(k) cos(mu pB);
// the polar integral uses FP_NGL Gauss-Legendre nodes.
__device__ void initial_state(Ctx& C, const FpParams& P, const double* B) {
    const int L = C.L;
    double* E = (double*)((char*)C.y - C.ly.y + C.ly.ic);   // [FP_NGL][L+1]
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
#pragma unroll
            for (int q = 0; q < FP_NGL / 32; ++q) {
                double cur;
                if (l == mu) cur = q2[q];
                else if (l == mu + 1) cur = sqrt(2.0 * mu + 3.0) * xs[q] * q2[q];
                else {
                    double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)mu * mu));
                    double b = sqrt((((double)l - 1.0) * (l - 1.0) - (double)mu * mu) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                    cur = a * (xs[q] * q2[q] - b * q1[q]);
                }
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

__global__ void __launch_bounds__(NT, 1) fp_solve_kernel(KArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_boff[FP_L_MAX + 2], s_foff[FP_L_MAX + 2];
    __shared__ int s_pp[64];
    __shared__ float s_red[NWARP];
    __shared__ double s_R[9], s_off[3], s_dm[3];

    Ctx C;
    C.ly = make_layout(A.L_launch);
    C.y = (double*)(smem + C.ly.y);
    C.Z = (double*)(smem + C.ly.Z);
    C.F = (double*)(smem + C.ly.F);
    C.tmp = (double*)(smem + C.ly.tmp);
    C.yb = (double*)(smem + C.ly.yb);
    C.diag = (double*)(smem + C.ly.diag);
    C.rr = (float*)(smem + C.ly.rr);
    C.rc = (float2*)(smem + C.ly.rc);
    C.zr = (float*)(smem + C.ly.zr);
    C.zc = (float2*)(smem + C.ly.zc);
    C.latv = (float*)(smem + C.ly.latv);
    C.fr = (float*)(smem + C.ly.fr);
    C.fc = (float2*)(smem + C.ly.fc);
    C.s1r = (float*)(smem + C.ly.s1r);
    C.s2r = (float*)(smem + C.ly.s2r);
    C.s1c = (float2*)(smem + C.ly.s1c);
    C.s2c = (float2*)(smem + C.ly.s2c);
    C.boff = s_boff;
    C.foff = s_foff;
    const DevTab& T = A.tab;
    const double sq43 = sqrt(4.0 * 3.14159265358979323846 / 3.0);

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
        __syncthreads();
        if (threadIdx.x == 0) {
            int bo = 0, fo = 0;
            for (int mu = 0; mu <= L + 1; ++mu) {
                s_boff[mu] = bo; s_foff[mu] = fo;
                if (mu <= L) { int nb = nblk(mu, L); bo += nb; fo += nb * nb; }
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
        initial_state(C, P, B);

        const double T_s = A.drv.period / A.drv.samples_per_period;     // sample spacing = h_max
        const double rtol = A.tol.rtol, atol = A.tol.atol;
        double t = 0.0;
        double tau = 0.5 / P.D;
        double h = fmin(T_s, 0.01 * tau);
        int jn = 0, nsteps = 0, nrej = 0, nit = 0, nfac = 0, status = FP_STATUS_OK;
        bool have_pred = false, fac_valid = false, force_refac = false;
        int since_fac = 0;
        double h_f = 0.0, h_old = 0.0;

        AScal sc0 = make_scal(P, B);
        apply_A(C.y, C.tmp, sc0, C.diag, N, T);            // f0 = A(t) y, kept in tmp
        __syncthreads();

        auto write_sample = [&](int j, double tj) {
            // <m> and d<m>/dt at t_j, rotated back to the lab frame
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

        // |y|_inf for the error scale
        float ym = 0.f;
        for (int i = threadIdx.x; i < N; i += NT) ym = fmaxf(ym, fabsf((float)C.y[i]));
        double ymax = block_max(ym, s_red);
        AScal scf;

        while (jn < A.S_out) {
            if (nsteps + nrej >= A.tol.max_steps) { status = FP_STATUS_MAXSTEPS; break; }
            if (h < 1e-6 * T_s) { status = FP_STATUS_STEP_UNDERFLOW; break; }
            const double tt = sample_time(A.drv, jn);
            double hs = fmin(h, T_s);
            bool last = false;
            if (t + hs >= tt - 1e-12 * T_s) { hs = tt - t; last = true; }
            // (re)factorise the iteration matrices
            double rat = fac_valid ? hs / h_f : 0.0;
            if (!fac_valid || force_refac || rat < 0.8 || rat > 1.25 || since_fac >= A.tol.refactor_every) {
                double Bf[3];
                field_nframe(A, R, off, t + hs, Bf);
                scf = make_scal(P, Bf);
                factorize(C, T, scf, hs, s_pp);
                h_f = hs; fac_valid = true; force_refac = false; since_fac = 0; ++nfac;
            }
            AScal scj[3];
            for (int j = 0; j < 3; ++j) {
                double Bj[3];
                field_nframe(A, R, off, t + c_rad.c[j] * hs, Bj);
                scj[j] = make_scal(P, Bj);
            }
            // predictor from the previous collocation polynomial
            if (have_pred) {
                const double r = hs / h_old;
                double nd[4] = {0.0, c_rad.c[0], c_rad.c[1], c_rad.c[2]};
                double Pm[3][3];
                for (int i = 0; i < 3; ++i) {
                    double tau_i = 1.0 + c_rad.c[i] * r;
                    for (int j = 1; j < 4; ++j) {
                        double lj = 1.0;
                        for (int k = 0; k < 4; ++k)
                            if (k != j) lj *= (tau_i - nd[k]) / (nd[j] - nd[k]);
                        Pm[i][j - 1] = lj - (j == 3 ? 1.0 : 0.0);
                    }
                }
                for (int i = threadIdx.x; i < N; i += NT) {
                    double z0 = C.Z[i], z1 = C.Z[N + i], z2 = C.Z[2 * N + i];
                    for (int k = 0; k < 3; ++k) C.Z[k * N + i] = Pm[k][0] * z0 + Pm[k][1] * z1 + Pm[k][2] * z2;
                }
            } else {
                for (int i = threadIdx.x; i < 3 * N; i += NT) C.Z[i] = 0.0;
            }
            const double sc_err = atol + rtol * ymax;
            const float fscale = (float)(h_f / hs);
            bool conv = false, nonfinite = false;
            float prev = 3.0e38f;
            for (int it = 0; it < A.tol.newton_max_iter; ++it) {
                // F_j = A(t + c_j h)(y + Z_j), FP64
                for (int j = 0; j < 3; ++j) {
                    for (int i = threadIdx.x; i < N; i += NT) C.yb[i] = C.y[i] + C.Z[j * N + i];
                    __syncthreads();
                    apply_A(C.yb, C.F + j * N, scj[j], C.diag, N, T);
                    __syncthreads();
                }
                // residual and right-hand sides (block order)
                for (int i = threadIdx.x; i < N; i += NT) {
                    double f0v = C.F[i], f1v = C.F[N + i], f2v = C.F[2 * N + i];
                    float Rk[3];
                    for (int k = 0; k < 3; ++k) {
                        double Rv = -C.Z[k * N + i] + hs * (c_rad.a[k][0] * f0v + c_rad.a[k][1] * f1v + c_rad.a[k][2] * f2v);
                        Rk[k] = (float)Rv;
                    }
                    int mu, kk;
                    glob_to_blk(i, mu, kk);
                    int b = C.boff[mu] + kk;
                    float q0 = (float)c_rad.K[0][0] * Rk[0] + (float)c_rad.K[0][1] * Rk[1] + (float)c_rad.K[0][2] * Rk[2];
                    float q1 = (float)c_rad.K[1][0] * Rk[0] + (float)c_rad.K[1][1] * Rk[1] + (float)c_rad.K[1][2] * Rk[2];
                    float q2 = (float)c_rad.K[2][0] * Rk[0] + (float)c_rad.K[2][1] * Rk[1] + (float)c_rad.K[2][2] * Rk[2];
                    C.rr[b] = q0;
                    C.rc[b] = make_float2(q1, q2);
                }
                __syncthreads();
                solve_blocks(C, T, true);
                // Z += T dW (h_f / h)
                float dm = 0.f;
                for (int i = threadIdx.x; i < N; i += NT) {
                    int mu, kk;
                    glob_to_blk(i, mu, kk);
                    int b = C.boff[mu] + kk;
                    float w0 = fscale * C.zr[b], w1 = fscale * C.zc[b].x, w2 = fscale * C.zc[b].y;
                    for (int k = 0; k < 3; ++k) {
                        float dz = (float)c_rad.T[k][0] * w0 + (float)c_rad.T[k][1] * w1 + (float)c_rad.T[k][2] * w2;
                        C.Z[k * N + i] += (double)dz;
                        dm = fmaxf(dm, fabsf(dz));
                    }
                }
                float dmax = block_max(dm, s_red);
                ++nit;
                if (!(dmax < 3.0e38f)) { nonfinite = true; break; }
                if (dmax <= 0.01f * (float)sc_err) { conv = true; break; }
                if (it >= 1 && dmax > 0.99f * prev) break;
                prev = dmax;
            }
            if (nonfinite) { status = FP_STATUS_NONFINITE; break; }
            if (!conv) {
                ++nrej;
                if (since_fac == 0 && h_f == hs && hs <= 1e-6 * T_s) { status = FP_STATUS_NEWTON_FAIL; break; }
                h = hs * 0.5; have_pred = false; force_refac = true;
                __syncthreads();
                continue;
            }
            // embedded error estimate, filtered through the real factor
            for (int i = threadIdx.x; i < N; i += NT) {
                double ev = hs * c_rad.g0 * C.tmp[i] + c_rad.e[0] * C.Z[i] + c_rad.e[1] * C.Z[N + i] + c_rad.e[2] * C.Z[2 * N + i];
                int mu, kk;
                glob_to_blk(i, mu, kk);
                C.rr[C.boff[mu] + kk] = (float)ev;
            }
            __syncthreads();
            solve_blocks(C, T, false);
            float em = 0.f;
            const float escale = (float)(c_rad.gam * h_f / hs);
            for (int i = threadIdx.x; i < N; i += NT) {
                int mu, kk;
                glob_to_blk(i, mu, kk);
                em = fmaxf(em, fabsf(escale * C.zr[C.boff[mu] + kk]));
            }
            double en = (double)block_max(em, s_red) / sc_err;
            if (!(en < 1e300)) { status = FP_STATUS_NONFINITE; break; }
            double fac = en > 0.0 ? 0.9 * pow(en, -0.25) : 4.0;
            if (en <= 1.0) {
                float ymx = 0.f;
                for (int i = threadIdx.x; i < N; i += NT) {
                    C.y[i] += C.Z[2 * N + i];
                    C.tmp[i] = C.F[2 * N + i];          // f0 of the next step ~ A(t+h) y_new
                    ymx = fmaxf(ymx, fabsf((float)C.y[i]));
                }
                ymax = block_max(ymx, s_red);
                ++nsteps; ++since_fac;
                t = last ? tt : t + hs;
                if (last) { write_sample(jn, tt); ++jn; }
                double hn = hs * fmin(4.0, fmax(0.2, fac));
                if (last && hs < h) hn = fac < 1.0 ? fmin(h, hn) : h;
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
        // zero the samples that were not reached
        for (int e = jn * 3 + threadIdx.x; e < A.S_out * 3; e += NT) {
            if (A.m_out) A.m_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
            if (A.dmdt_out) A.dmdt_out[(size_t)inst * A.S_out * 3 + e] = 0.0;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------- host launch ----
int fp_launch_solve(const DevTab* tab, const fp_material* mat, const fp_drive* drv, const fp_tol* tol,
                    const fp_instance* d_inst, int n, int L_launch, double* d_m, double* d_dmdt,
                    int* d_status, int* d_stats, int grid, cudaStream_t st) {
    KArgs A;
    A.tab = *tab;
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
    size_t sm = fp_solver_smem_bytes(L_launch);
    cudaError_t e = cudaFuncSetAttribute(fp_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return FP_ECUDA;
    fp_solve_kernel<<<grid, NT, sm, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
}

int fp_upload_constants(const FpRadau* r, const double* glx, const double* glw) {
    if (cudaMemcpyToSymbol(c_rad, r, sizeof(FpRadau)) != cudaSuccess) return FP_ECUDA;
    if (cudaMemcpyToSymbol(c_glx, glx, sizeof(double) * FP_NGL) != cudaSuccess) return FP_ECUDA;
    if (cudaMemcpyToSymbol(c_glw, glw, sizeof(double) * FP_NGL) != cudaSuccess) return FP_ECUDA;
    return FP_OK;
}
