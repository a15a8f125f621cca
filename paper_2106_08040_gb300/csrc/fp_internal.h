// Internal definitions shared by the host table builder and the CUDA kernels.
#pragma once
#include <math.h>
#include "../../include/fp.h"

#ifdef __CUDACC__
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif

#define FP_L_MAX 24          // largest supported truncation degree
#define FP_L_SMEM 16         // largest degree whose factors fit in shared memory (above: global scratch, 3 stages)
#define FP_NSLOT 19          // coupling slots per target row (see slot map below)
#define FP_NGL 128           // Gauss-Legendre nodes for the Boltzmann initial state

// Slot map of one target row (l, m) of the Galerkin matrix in the easy-axis frame:
//   0,1   W   (anisotropy damping)      sources (l-2, m), (l+2, m)
//   2,3   ZRz (anisotropy precession)   sources (l-1, -m), (l+1, -m)
//   4     Rz  (precession about n)      source  (l, -m)
//   5,6   Rx  (precession about x')     sources (l, m'), |m'| = |m| -/+ 1
//   7,8   Ry  (precession about y')     sources (l, m'), |m'| = |m| -/+ 1
//   9,10  Gz  (damping along n)         sources (l-1, m), (l+1, m)
//   11-14 Gx  (damping along x')        sources (l-/+1, m'), |m'| = |m| -/+ 1
//   15-18 Gy  (damping along y')        sources (l-/+1, m'), |m'| = |m| -/+ 1
enum { SL_W = 0, SL_ZR = 2, SL_RZ = 4, SL_RX = 5, SL_RY = 7, SL_GZ = 9, SL_GX = 11, SL_GY = 15 };

static const double FP_KB = 1.380649e-23;   // J/K (exact SI)

// Per-instance constants of Sec. 2.1 (Neel constants) and Sec. 2.2 (m0, beta).
// Fields are mu0 H in tesla, so p1, p2 multiply tesla and bT = beta/mu0.
struct FpParams {
    double D;        // 1/(2 tau)
    double p1, p2;   // gamma~, gamma~ alpha
    double p3, p4;   // 2 gamma~ K / Ms, alpha p3
    double sigma;    // K V / (kB T)
    double bT;       // V Ms / (kB T)
};

FP_HD FpParams fp_derive(const fp_material& mt, double K, double d) {
    FpParams P;
    const double pi = 3.14159265358979323846;
    double V = pi * d * d * d / 6.0;
    double gt = mt.gamma / (1.0 + mt.alpha * mt.alpha);
    double kT = FP_KB * mt.T_B;
    double tau = V * mt.Ms / (2.0 * kT * gt * mt.alpha);
    P.D = 0.5 / tau;
    P.p1 = gt;
    P.p2 = gt * mt.alpha;
    P.p3 = 2.0 * gt * K / mt.Ms;
    P.p4 = mt.alpha * P.p3;
    P.sigma = K * V / kT;
    P.bT = V * mt.Ms / kT;
    return P;
}

// Rotation taking the easy axis n(theta, phi) to z: R = R_y(-theta) R_z(-phi).
FP_HD void fp_rotation(double th, double ph, double R[9]) {
    double ct = cos(th), st = sin(th), cp = cos(ph), sp = sin(ph);
    R[0] = ct * cp; R[1] = ct * sp; R[2] = -st;
    R[3] = -sp;     R[4] = cp;      R[5] = 0.0;
    R[6] = st * cp; R[7] = st * sp; R[8] = ct;
}

// Coefficients of an s-stage Radau IIA method (s = 3, 5, 7) and of its
// simplified-Newton transformation and embedded error estimate (host-derived).
#define FP_SMAX 7
struct FpRadau {
    int s;
    double c[FP_SMAX];
    double a[FP_SMAX][FP_SMAX];
    double T[FP_SMAX][FP_SMAX];      // a^{-1} = T Lam T^{-1}
    double Ti[FP_SMAX][FP_SMAX];
    double K[FP_SMAX][FP_SMAX];      // Ti a^{-1}
    double gam;                      // real eigenvalue of a^{-1}
    double alp[3], bet[3];           // complex pairs alp +- i bet (bet > 0)
    double e[FP_SMAX], g0;           // err_pre = h g0 f(t_n, y_n) + sum_i e_i Z_i
};

// Host-built tables (device copies live in the context).
struct FpTablesHost {
    int L;               // tables cover degrees 0..L
    int N;               // (L+1)^2
    double* coef;        // [N][FP_NSLOT]
    int* src;            // [N][FP_NSLOT], -1 where no source exists
    double* lam;         // [N] l(l+1)
    double* wdiag;       // [N] diagonal of W
    int* tslot;          // [N][FP_NSLOT] slot of row src pointing back (lateral slots), else -1
};

int fp_build_tables(int L, FpTablesHost* out);     // returns 0 / FP_ENOMEM
void fp_free_tables(FpTablesHost* t);
int fp_build_radau(int s, FpRadau* r);             // returns 0 / FP_EINVAL

// Block structure of the Galerkin matrix for one degree L, rows in block order
// (blocks mu = |m| = 0..L; block 0 = (l, 0) for l = 0..L, block mu > 0 =
// (l, +mu), (l, -mu) interleaved for l = mu..L).  For every row: up to 7
// couplings inside its block (sb), up to 6 to block mu-1 (dn) and up to 6 to
// block mu+1 (up), each as (local column, scalar group, table coefficient);
// dnT gives, for each dn partner, the position in the partner's up list of the
// coupling back to this row (255 if that entry is structurally zero).
#define FP_NSB 8
#define FP_NLT 6
struct FpBlkHost {
    int L, N;
    int* glob;                 // [N] natural index of block row b
    unsigned char* sb_k;       // [N][FP_NSB]  (255 = none)
    unsigned char* sb_g;
    float* sb_cf;
    unsigned char* dn_k;       // [N][FP_NLT]
    unsigned char* dn_g;
    float* dn_cf;
    unsigned char* up_k;       // [N][FP_NLT]
    unsigned char* up_g;
    float* up_cf;
    unsigned char* dnT;        // [N][FP_NLT]
    unsigned char* upT;        // [N][FP_NLT] for each up partner: position in its dn list of the coupling back
};
int fp_build_blocks(const FpTablesHost* t, int L, FpBlkHost* out);

struct FpPair { int row, slot; };

// Device views of the tables (pointers into context-owned device memory).
#include <stdint.h>
struct DevTab {
    // slot-major ("transposed") device copies: entry (row i, slot k) at
    // k * nrow + i, so a warp over consecutive rows reads consecutive words
    const double* coef;              // [FP_NSLOT][nrow]
    const int* src;                  // [FP_NSLOT][nrow]
    const double* lam;               // [nrow]
    const double* wdiag;             // [nrow]
    const FpPair* colT;              // [FP_NCT][nrow] column view (row, slot)
    const double* coef4;             // [FP_NSLOT][nrow] coef with the G slots times alpha and the W slots
                                     // times alpha/2: A(t) x in four scalar groups (anisotropy, x', y', z')
    int nrow;                        // rows of the tables: (L_max + 1)^2
};
struct DevBlk {                      // block structure of every degree, packed
    const int* glob;
    const uint8_t* sb_k;
    const uint8_t* sb_g;
    const float* sb_cf;
    const uint8_t* dn_k;
    const uint8_t* dn_g;
    const float* dn_cf;
    const uint8_t* up_k;
    const uint8_t* up_g;
    const float* up_cf;
    const uint8_t* dnT;
    const uint8_t* upT;
    int off[FP_L_MAX + 2];           // first packed row of degree L
};

// Column view of the coupling tables (for A^T x): for column i, up to FP_NCT
// (row, slot) pairs with table[row][slot] having source i; row = -1 pads.
#define FP_NCT 24
int fp_build_columns(const FpTablesHost* t, FpPair* out);   // out: [N][FP_NCT]
void fp_build_coef4(const FpTablesHost* t, double alpha, double* out);   // out: [N][FP_NSLOT]
void fp_free_blocks(FpBlkHost* b);
void fp_gauss_legendre(int n, double* x, double* w);

// ------------------------------------------------ context and launchers ----
#include <cuda_runtime.h>
size_t fp_solver_smem_bytes(int stages, int L);
size_t fp_solver_fac_bytes(int stages, int L);     // global factor bytes per CTA (0 when they fit in shared memory)
int fp_solver_ctas_per_sm(int stages, int L);     // CTAs per SM of the solve launch (one factor slot each)
// bytes of the factor scratch a solve launch at (stages, L) needs on num_sms SMs (0: none)
size_t fp_solver_fac_scratch_bytes(int stages, int L, int num_sms);
// d_fac: factor scratch of at least fp_solver_fac_scratch_bytes(stages, L_launch, num_sms) bytes when that is nonzero
int fp_launch_solve(int stages, const DevTab* tab, const DevBlk* blk, const fp_material* mat, const fp_drive* drv,
                    const fp_tol* tol, const fp_instance* d_inst, int n, int L_launch, double* d_m, double* d_dmdt,
                    int* d_status, int* d_stats, int num_sms, cudaStream_t st, const int* d_order, int* d_queue,
                    unsigned char* d_fac);
int fp_upload_constants(const FpRadau* r3, const FpRadau* r5, const double* glx, const double* glw);
size_t fp_adjoint_smem_bytes(int stages, int L);
size_t fp_adjoint_work_doubles_per_cta(int stages, int L_max, int S_p, int max_rec);
int fp_launch_adjoint(int stages, const DevTab* tab, const DevBlk* blk, const fp_material* mat, const fp_drive* drv,
                      const fp_tol* tol, const fp_instance* d_inst, int n, int L_launch, int k_max,
                      const double* channels, int C, const double* d_dJ, const double* d_tw, double* d_grad,
                      int* d_status, int* d_stats, double* d_work, int max_rec, int grid, cudaStream_t st);

struct fp_ctx {
    fp_material mat;
    fp_drive drv;
    fp_tol tol;
    int L_max;
    int device;
    int num_sms;
    FpTablesHost host;
    double* d_coef;
    int* d_src;
    double* d_lam;
    double* d_wdiag;
    FpPair* d_colT;           // column view of the tables (adjoint)
    double* d_coef4;          // coefficients regrouped by field component (forward apply)
    DevBlk blk;               // device block structure, all degrees 2..L_max
    void* d_blk_mem;          // one allocation backing blk
    double* d_tw;             // twiddles cos/sin(2 pi q / S_p), q < S_p (fp_signal)
    unsigned char* d_fac;     // factor scratch of the solve launch (five stages or L_max > FP_L_SMEM), else NULL
    int* d_queue;             // work counter of fp_solve_batch (instances taken one at a time by the CTAs)
};

int fp_fail(int code, const char* fmt, ...);
