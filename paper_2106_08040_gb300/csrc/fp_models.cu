// Data-driven system-matrix models of Sec. 2.2 and the distance measures of
// Sec. 2.3 on sm_103a:
//   fp_equilibrium  -- model M0: the equilibrium mean moment m_equ/m0 =
//                      L(bT |B|) B/|B| (Eq. Langevin) and its exact time
//                      derivative at every output sample, in the layout of
//                      fp_solve_batch (so fp_signal turns it into phi_hat_D)
//   fp_m1_fit       -- model M1 (and M0): per dictionary element q, channel c
//                      and row k, a_qk = S_k conj(Phi_qk)^T / ||Phi_qk||^2 and the
//                      row error of Eq. error1 for S_model = diag(a_q) Phi_q
//   fp_nrmse        -- per-frequency and global NRMSE (eq. globalMeasure) from
//                      row errors over a frequency index set
//   fp_mixing_order / fp_freq_index_set -- Eq. mix and I_freq (host only)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include "fp_internal.h"

// ------------------------------------------------------------- Langevin ----
// L(x) = coth x - 1/x = sum_n c_n x^(2n-1), c_n = 2^(2n) B_2n / (2n)!  (B_2n the
// Bernoulli numbers), n = 1..11; below x = 0.5 the closed form cancels
// (relative error ~ 3 eps / x^2), so g = L/x and d = L' - g come from the series
// there: g = sum c_n x^(2n-2), d = sum (2n-2) c_n x^(2n-2).
#define FP_LSER_N 11
#define FP_LSER_MAX 0.5
__constant__ double c_lser[FP_LSER_N];

static void langevin_series(double* c) {
    // reduced fractions 2^(2n) B_2n / (2n)!, divided in long double
    static const long double num[FP_LSER_N] = {1.0L, -1.0L, 2.0L, -1.0L, 2.0L, -1382.0L, 4.0L, -3617.0L, 87734.0L,
                                               -349222.0L, 310732.0L};
    static const long double den[FP_LSER_N] = {3.0L, 45.0L, 945.0L, 4725.0L, 93555.0L, 638512875.0L, 18243225.0L,
                                               162820783125.0L, 38979295480125.0L, 1531329465290625.0L,
                                               13447856940643125.0L};
    for (int i = 0; i < FP_LSER_N; ++i) c[i] = (double)(num[i] / den[i]);
}

// g = L(x)/x and d = L'(x) - L(x)/x for x >= 0
__device__ __forceinline__ void langevin_gd(double x, double& g, double& d) {
    if (x < FP_LSER_MAX) {
        const double x2 = x * x;
        double gs = c_lser[FP_LSER_N - 1], ds = (2.0 * FP_LSER_N - 2.0) * c_lser[FP_LSER_N - 1];
#pragma unroll
        for (int n = FP_LSER_N - 2; n >= 0; --n) {
            gs = fma(gs, x2, c_lser[n]);
            ds = fma(ds, x2, (2.0 * n) * c_lser[n]);
        }
        g = gs;
        d = ds;
    } else {
        const double e = exp(-2.0 * x);
        const double coth = (1.0 + e) / (1.0 - e);
        const double csch2 = 4.0 * e / ((1.0 - e) * (1.0 - e));
        const double ix = 1.0 / x;
        const double L = coth - ix;
        g = L * ix;
        d = (ix * ix - csch2) - g;
    }
}

struct EqArgs {
    fp_material mat;
    fp_drive drv;
    const fp_instance* inst;
    int n, S_out;
    double* m_out;
    double* dmdt_out;
};

// one thread per (instance, sample): B = off + amp sin(w t + ph),
// dB/dt = amp w cos(w t + ph); m = L(xi) B/|B| = bT g B,
// dm/dt = bT [g dB/dt + d (Bhat . dB/dt) Bhat]   (xi = bT |B|)
__global__ void fp_equilibrium_kernel(EqArgs A) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)A.n * A.S_out) return;
    const int i = (int)(e / A.S_out), j = (int)(e - (long long)i * A.S_out);
    const fp_instance in = A.inst[i];
    double* mo = A.m_out ? A.m_out + (size_t)e * 3 : nullptr;
    double* dmo = A.dmdt_out ? A.dmdt_out + (size_t)e * 3 : nullptr;
    if (!(in.d > 0.0) || in.flags != 0) {
        for (int k = 0; k < 3; ++k) {
            if (mo) mo[k] = 0.0;
            if (dmo) dmo[k] = 0.0;
        }
        return;
    }
    const double twopi = 6.283185307179586476925286766559;
    const double t = ((double)A.drv.warmup_periods + (double)j / (double)A.drv.samples_per_period) * A.drv.period;
    double B[3], Bd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double w = twopi * A.drv.freq[k];
        double s, c;
        sincos(w * t + A.drv.phase[k], &s, &c);
        B[k] = in.h_off[k] + A.drv.amp[k] * s;
        Bd[k] = A.drv.amp[k] * w * c;
    }
    const double V = 3.14159265358979323846 * in.d * in.d * in.d / 6.0;
    const double bT = V * A.mat.Ms / (FP_KB * A.mat.T_B);
    const double nb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    double g, d;
    langevin_gd(bT * nb, g, d);
    double proj = 0.0, bh[3] = {0.0, 0.0, 0.0};
    if (nb > 0.0) {
        const double inb = 1.0 / nb;
#pragma unroll
        for (int k = 0; k < 3; ++k) bh[k] = B[k] * inb;
        proj = bh[0] * Bd[0] + bh[1] * Bd[1] + bh[2] * Bd[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (mo) mo[k] = bT * g * B[k];
        if (dmo) dmo[k] = bT * fma(d * proj, bh[k], g * Bd[k]);
    }
}

// -------------------------------------------------------------- M1 fit ----
// Columns (c, k) are contiguous in the [N][C][K1] layout, so a block takes
// FP_M1_COLS consecutive columns of one dictionary element and FP_M1_VG voxel
// groups (voxels nu = g, g + VG, ...); partial sums meet in shared memory.
#define FP_M1_COLS 64
#define FP_M1_VG 4

// pass 1: a = sum S conj(Phi) / sum |Phi|^2 and max |S| per column
__global__ void fp_m1_pass1(const double2* __restrict__ phi, const double2* __restrict__ S, int N, int CK,
                            double2* __restrict__ a, double* __restrict__ smax) {
    __shared__ double red[FP_M1_VG][FP_M1_COLS][4];
    const int col = blockIdx.x * FP_M1_COLS + (threadIdx.x % FP_M1_COLS);
    const int g = threadIdx.x / FP_M1_COLS;
    const int q = blockIdx.y;
    double sr = 0.0, si = 0.0, pp = 0.0, mx = 0.0;
    if (col < CK) {
        const double2* P = phi + (size_t)q * N * CK + col;
        const double2* Sv = S + col;
        for (int nu = g; nu < N; nu += FP_M1_VG) {
            const double2 p = __ldg(P + (size_t)nu * CK), s = __ldg(Sv + (size_t)nu * CK);
            sr = fma(s.x, p.x, fma(s.y, p.y, sr));          // S conj(Phi)
            si = fma(s.y, p.x, fma(-s.x, p.y, si));
            pp = fma(p.x, p.x, fma(p.y, p.y, pp));
            mx = fmax(mx, s.x * s.x + s.y * s.y);
        }
    }
    const int cl = threadIdx.x % FP_M1_COLS;
    red[g][cl][0] = sr; red[g][cl][1] = si; red[g][cl][2] = pp; red[g][cl][3] = mx;
    __syncthreads();
    if (g == 0 && col < CK) {
        for (int h = 1; h < FP_M1_VG; ++h) {
            sr += red[h][cl][0]; si += red[h][cl][1]; pp += red[h][cl][2]; mx = fmax(mx, red[h][cl][3]);
        }
        const double ip = pp > 0.0 ? 1.0 / pp : 0.0;
        a[(size_t)q * CK + col] = make_double2(sr * ip, si * ip);
        if (q == 0) smax[col] = sqrt(mx);
    }
}

// pass 2: eps = sqrt(sum |S - a Phi|^2 / N) / max |S|
__global__ void fp_m1_pass2(const double2* __restrict__ phi, const double2* __restrict__ S, int N, int CK,
                            const double2* __restrict__ a, const double* __restrict__ smax, double* __restrict__ eps) {
    __shared__ double red[FP_M1_VG][FP_M1_COLS];
    const int col = blockIdx.x * FP_M1_COLS + (threadIdx.x % FP_M1_COLS);
    const int g = threadIdx.x / FP_M1_COLS;
    const int q = blockIdx.y;
    double rr = 0.0;
    if (col < CK) {
        const double2 av = a[(size_t)q * CK + col];
        const double2* P = phi + (size_t)q * N * CK + col;
        const double2* Sv = S + col;
        for (int nu = g; nu < N; nu += FP_M1_VG) {
            const double2 p = __ldg(P + (size_t)nu * CK), s = __ldg(Sv + (size_t)nu * CK);
            const double dr = s.x - (av.x * p.x - av.y * p.y);
            const double di = s.y - (av.x * p.y + av.y * p.x);
            rr = fma(dr, dr, fma(di, di, rr));
        }
    }
    const int cl = threadIdx.x % FP_M1_COLS;
    red[g][cl] = rr;
    __syncthreads();
    if (g == 0 && col < CK) {
        for (int h = 1; h < FP_M1_VG; ++h) rr += red[h][cl];
        const double m = smax[col];
        eps[(size_t)q * CK + col] = m > 0.0 ? sqrt(rr / N) / m : 0.0;
    }
}

// eps_freq[k] = sqrt(mean over (angle, channel) of eps^2); global = sqrt(mean over I_freq of eps_freq^2)
__global__ void fp_nrmse_kernel(const double* __restrict__ eps, int A, int C, int K1, const int* __restrict__ ks,
                                int nk, double* __restrict__ eps_freq, double* __restrict__ eps_global) {
    __shared__ double red[256];
    double part = 0.0;
    for (int k = threadIdx.x; k < K1; k += blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < A; ++a)
            for (int c = 0; c < C; ++c) {
                const double v = eps[((size_t)a * C + c) * K1 + k];
                s = fma(v, v, s);
            }
        s /= (double)(A * C);
        if (eps_freq) eps_freq[k] = sqrt(s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        const int k = ks[i];
        double s = 0.0;
        for (int a = 0; a < A; ++a)
            for (int c = 0; c < C; ++c) {
                const double v = eps[((size_t)a * C + c) * K1 + k];
                s = fma(v, v, s);
            }
        part += s / (double)(A * C);
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *eps_global = sqrt(red[0] / (double)nk);
}

// ------------------------------------------------------------- C ABI ------
static int g_lser_device = -1;

extern "C" {

int fp_equilibrium(fp_ctx* ctx, const fp_instance* d_inst, int n, double* d_m, double* d_dmdt, void* stream) {
    if (!ctx) return fp_fail(FP_EINVAL, "fp_equilibrium: NULL ctx");
    if (n < 0) return fp_fail(FP_EINVAL, "fp_equilibrium: n < 0");
    if (n == 0) return FP_OK;
    if (!d_inst || (!d_m && !d_dmdt)) return fp_fail(FP_EINVAL, "fp_equilibrium: NULL buffer");
    if (g_lser_device != ctx->device) {
        double c[FP_LSER_N];
        langevin_series(c);
        if (cudaMemcpyToSymbol(c_lser, c, sizeof(c)) != cudaSuccess)
            return fp_fail(FP_ECUDA, "fp_equilibrium: constant upload failed");
        g_lser_device = ctx->device;
    }
    EqArgs A;
    A.mat = ctx->mat;
    A.drv = ctx->drv;
    A.inst = d_inst;
    A.n = n;
    A.S_out = ctx->drv.output_periods * ctx->drv.samples_per_period;
    A.m_out = d_m;
    A.dmdt_out = d_dmdt;
    const long long total = (long long)n * A.S_out;
    const int bs = 256;
    fp_equilibrium_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, (cudaStream_t)stream>>>(A);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_equilibrium: launch failed");
    return FP_OK;
}

int fp_m1_fit(const double* d_phi, int Q, const double* d_S, int N, int C, int K1, double* d_a, double* d_eps,
              double* d_smax, void* stream) {
    if (!d_phi || !d_S || !d_a || !d_eps || !d_smax) return fp_fail(FP_EINVAL, "fp_m1_fit: NULL buffer");
    if (Q < 0 || N < 0 || C < 1 || K1 < 1) return fp_fail(FP_EINVAL, "fp_m1_fit: bad sizes");
    if (Q == 0 || N == 0) return FP_OK;
    if (Q > 65535) return fp_fail(FP_EINVAL, "fp_m1_fit: Q=%d > 65535 dictionary elements per call", Q);
    const int CK = C * K1;
    dim3 grid((CK + FP_M1_COLS - 1) / FP_M1_COLS, Q);
    cudaStream_t st = (cudaStream_t)stream;
    fp_m1_pass1<<<grid, FP_M1_COLS * FP_M1_VG, 0, st>>>((const double2*)d_phi, (const double2*)d_S, N, CK,
                                                        (double2*)d_a, d_smax);
    fp_m1_pass2<<<grid, FP_M1_COLS * FP_M1_VG, 0, st>>>((const double2*)d_phi, (const double2*)d_S, N, CK,
                                                        (const double2*)d_a, d_smax, d_eps);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_m1_fit: launch failed");
    return FP_OK;
}

int fp_nrmse(const double* d_eps, int A, int C, int K1, const int* d_ks, int nk, double* d_eps_freq,
             double* d_eps_global, void* stream) {
    if (!d_eps || !d_ks || !d_eps_global) return fp_fail(FP_EINVAL, "fp_nrmse: NULL buffer");
    if (A < 1 || C < 1 || K1 < 1 || nk < 1) return fp_fail(FP_EINVAL, "fp_nrmse: bad sizes");
    fp_nrmse_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(d_eps, A, C, K1, d_ks, nk, d_eps_freq, d_eps_global);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_nrmse: launch failed");
    return FP_OK;
}

int fp_mixing_order(int k, int n_dens, int* mx, int* my) {
    if (n_dens < 1 || !mx || !my) return fp_fail(FP_EINVAL, "fp_mixing_order: bad argument");
    // every solution of k = m_x n + m_y (n + 1) has m_y = k (mod n): scan m_y
    // over enough periods on both sides and keep the smallest |m_x| + |m_y|
    // (then the smaller |m_x|, then m_x >= 0)
    const long long n = n_dens, kk = k;
    long long r0 = kk % n;
    if (r0 < 0) r0 += n;
    const long long span = (kk < 0 ? -kk : kk) / n + 2;
    long long best_key0 = -1, best_key1 = 0, best_key2 = 0, bx = 0, by = 0;
    for (long long j = -span; j <= span; ++j) {
        const long long yv = r0 + j * n;
        const long long rem = kk - yv * (n + 1);
        if (rem % n) continue;
        const long long xv = rem / n;
        const long long k0 = (xv < 0 ? -xv : xv) + (yv < 0 ? -yv : yv), k1 = xv < 0 ? -xv : xv, k2 = xv >= 0 ? 0 : 1;
        if (best_key0 < 0 || k0 < best_key0 || (k0 == best_key0 && (k1 < best_key1 || (k1 == best_key1 && k2 < best_key2)))) {
            best_key0 = k0; best_key1 = k1; best_key2 = k2; bx = xv; by = yv;
        }
    }
    *mx = (int)bx;
    *my = (int)by;
    return FP_OK;
}

int fp_freq_index_set(int M_x, int M_y, int n_dens, int k_limit, int* h_ks, int cap, int* count) {
    if (M_x < 0 || M_y < 0 || n_dens < 1 || !count || (cap > 0 && !h_ks))
        return fp_fail(FP_EINVAL, "fp_freq_index_set: bad argument");
    // distinct k(m_x, m_y) = m_x n + m_y (n + 1) in increasing order, without the
    // orders (0,0), (0,1), (1,0) and without k > k_limit
    int cnt = 0;
    for (int k = 0; k <= k_limit; ++k) {
        bool hit = false;
        for (int x = 0; x <= M_x && !hit; ++x) {
            const long long rem = (long long)k - (long long)x * n_dens;
            if (rem < 0 || rem % (n_dens + 1)) continue;
            const long long y = rem / (n_dens + 1);
            if (y > M_y) continue;
            if ((x == 0 && y == 0) || (x == 0 && y == 1) || (x == 1 && y == 0)) continue;
            hit = true;
        }
        if (!hit) continue;
        if (cnt < cap) h_ks[cnt] = k;
        ++cnt;
    }
    *count = cnt;
    return FP_OK;
}

}  // extern "C"
