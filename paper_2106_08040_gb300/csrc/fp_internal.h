// Internal definitions shared by the host table builder and the CUDA kernels.
#pragma once
#include <math.h>
#include "../../include/fp.h"

#ifdef __CUDACC__
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif

#define FP_L_MAX 16          // largest degree with shared-memory factors in this build
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

// Coefficients of the 3-stage Radau IIA method and of its simplified-Newton
// transformation and embedded error estimate (derived on the host).
struct FpRadau {
    double c[3];
    double a[3][3];
    double T[3][3];      // a^{-1} = T Lam T^{-1}
    double Ti[3][3];
    double K[3][3];      // Ti a^{-1} (= Lam Ti)
    double gam, alp, bet;
    double e[3], g0;     // err_pre = h g0 f(t_n, y_n) + sum_i e_i Z_i
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
void fp_build_radau(FpRadau* r);
void fp_gauss_legendre(int n, double* x, double* w);
