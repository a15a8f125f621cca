// Model M2 of Sec. 2.2, second step: non-negative superposition weights of
// the dictionary Psi_q = diag(a_q) Phi_q (eq. psi_def) over all easy-axis
// angles (eq. LSfitM2), regularised by truncating the SVD of the stacked
// Sigma-weighted dictionary matrix M (eq. LSfitM2_alternative,
// eq. approx_low_rank).
//
//   fp_m2_gram (GPU)   the complex Gram matrix of [M | y]: every product the
//                      fit needs (M^H M, M^H y, y^H y), as one FP64 reduction
//                      over rows r = (angle, voxel, channel, frequency row)
//   fp_m2_solve (host) M^H M = V diag(s^2) V^H -> U_s^H M = diag(s_s) V_s^H and
//                      U_s^H y = diag(1/s_s) V_s^H M^H y; real and imaginary
//                      parts stacked (the weights are real); the quadratic
//                      program min 1/2 w^T Q w + f^T w, w >= 0 solved by a
//                      primal-dual interior-point method
#include <cuda_runtime.h>
#include <math.h>
#include <algorithm>
#include <cstring>
#include <vector>
#include "fp_internal.h"

#define M2_T 16            // output tile (M2_T x M2_T entries of the Gram matrix)
#define M2_R 16            // rows staged per step

struct GramArgs {
    const double2* phi;    // [A][J][N][C][K1]
    const double2* a;      // [A][J][C][K1]
    const double2* S;      // [A][N][C][K1]
    const double* smax;    // [A][C][K1]
    const int* ks;         // [nk]
    int A, J, N, C, K1, nk;
    long long R;           // rows = A N C nk
    long long rows_per_split;
    int ntile;             // tiles per side, ceil((J + 1) / M2_T)
    double2* G;            // [(J + 1)][(J + 1)]
};

// entry (r, col) of [M | y]: col < J -> sigma a Phi, col == J -> sigma S
__device__ __forceinline__ double2 m2_entry(const GramArgs& g, long long r, int col) {
    if (col > g.J) return make_double2(0.0, 0.0);
    const int kk = (int)(r % g.nk);
    long long t = r / g.nk;
    const int c = (int)(t % g.C);
    t /= g.C;
    const int nu = (int)(t % g.N);
    const int th = (int)(t / g.N);
    const int k = __ldg(g.ks + kk);
    const size_t ck = (size_t)c * g.K1 + k;
    const double m = __ldg(g.smax + (size_t)th * g.C * g.K1 + ck);
    const double sig = m > 0.0 ? 1.0 / m : 0.0;
    if (col == g.J) {
        const double2 s = __ldg(g.S + ((size_t)th * g.N + nu) * g.C * g.K1 + ck);
        return make_double2(sig * s.x, sig * s.y);
    }
    const double2 av = __ldg(g.a + ((size_t)th * g.J + col) * g.C * g.K1 + ck);
    const double2 p = __ldg(g.phi + (((size_t)th * g.J + col) * g.N + nu) * g.C * g.K1 + ck);
    return make_double2(sig * (av.x * p.x - av.y * p.y), sig * (av.x * p.y + av.y * p.x));
}

// blockIdx.x: upper-triangle tile (ti <= tj), blockIdx.y: row split.
// Thread (row u, column v) of the tile accumulates sum_r conj(M[r][i]) M[r][j].
__global__ void __launch_bounds__(M2_T * M2_T) fp_m2_gram_kernel(GramArgs g) {
    __shared__ double2 Mi[M2_R][M2_T], Mj[M2_R][M2_T];
    int ti = 0, rem = blockIdx.x;
    while (rem >= g.ntile - ti) { rem -= g.ntile - ti; ++ti; }
    const int tj = ti + rem;
    const int u = threadIdx.x / M2_T, v = threadIdx.x % M2_T;
    const int i = ti * M2_T + u, j = tj * M2_T + v;
    const long long r0 = (long long)blockIdx.y * g.rows_per_split;
    const long long r1 = min(g.R, r0 + g.rows_per_split);
    double re = 0.0, im = 0.0;
    // staging: thread (q, w) loads row r + q of columns ti*T + w and tj*T + w
    const int q = threadIdx.x % M2_R, w = threadIdx.x / M2_R;
    for (long long r = r0; r < r1; r += M2_R) {
        const long long rr = r + q;
        const bool ok = rr < r1;
        Mi[q][w] = ok ? m2_entry(g, rr, ti * M2_T + w) : make_double2(0.0, 0.0);
        Mj[q][w] = ok ? m2_entry(g, rr, tj * M2_T + w) : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int s = 0; s < M2_R; ++s) {
            const double2 x = Mi[s][u], y = Mj[s][v];
            re = fma(x.x, y.x, fma(x.y, y.y, re));      // conj(x) y
            im = fma(x.x, y.y, fma(-x.y, y.x, im));
        }
        __syncthreads();
    }
    if (i <= g.J && j <= g.J) {
        atomicAdd(&g.G[(size_t)i * (g.J + 1) + j].x, re);
        atomicAdd(&g.G[(size_t)i * (g.J + 1) + j].y, im);
    }
}

// --------------------------------------------------------- host algebra ----
// Cyclic Jacobi eigen-decomposition of a real symmetric n x n matrix (row
// major, destroyed): eigenvalues into ev, eigenvectors as the columns of V.
static void jacobi_eigen(int n, std::vector<double>& Am, std::vector<double>& ev, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                const double x = Am[(size_t)p * n + q] * Am[(size_t)p * n + q];
                tot += x;
                if (p != q) off += x;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = Am[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = Am[(size_t)p * n + p], aqq = Am[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {           // A <- A J (columns p, q)
                    const double akp = Am[(size_t)k * n + p], akq = Am[(size_t)k * n + q];
                    Am[(size_t)k * n + p] = c * akp - s * akq;
                    Am[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {           // A <- J^T A (rows p, q)
                    const double apk = Am[(size_t)p * n + k], aqk = Am[(size_t)q * n + k];
                    Am[(size_t)p * n + k] = c * apk - s * aqk;
                    Am[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    ev.resize(n);
    for (int i = 0; i < n; ++i) ev[i] = Am[(size_t)i * n + i];
}

// Cholesky solve of the SPD n x n system K x = b (K destroyed); false if not SPD
static bool cholesky_solve(int n, std::vector<double>& K, std::vector<double>& x) {
    for (int j = 0; j < n; ++j) {
        double d = K[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= K[(size_t)j * n + k] * K[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        K[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = K[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= K[(size_t)i * n + k] * K[(size_t)j * n + k];
            K[(size_t)i * n + j] = v / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double v = x[i];
        for (int k = 0; k < i; ++k) v -= K[(size_t)i * n + k] * x[k];
        x[i] = v / K[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < n; ++k) v -= K[(size_t)k * n + i] * x[k];
        x[i] = v / K[(size_t)i * n + i];
    }
    return true;
}

static void qp_polish(int n, const std::vector<double>& Q, const std::vector<double>& f, std::vector<double>& w,
                      const std::vector<double>& z);

// min 1/2 w^T Q w + f^T w, w >= 0: primal-dual interior point (Mehrotra
// predictor-corrector) on Q w + f - z = 0, w z = mu, w, z > 0
static int qp_nonneg(int n, const std::vector<double>& Q, const std::vector<double>& f, std::vector<double>& w) {
    std::vector<double> z(n), rd(n), dw(n), dz(n), K((size_t)n * n), rhs(n), dwa(n), dza(n);
    double scale = 1.0;
    for (int i = 0; i < n; ++i) scale = std::max(scale, std::max(std::fabs(Q[(size_t)i * n + i]), std::fabs(f[i])));
    w.assign(n, 1.0);
    for (int i = 0; i < n; ++i) z[i] = scale;
    auto newton = [&](const std::vector<double>& rc, std::vector<double>& ow, std::vector<double>& oz) -> bool {
        // (Q + Z/W) dw = -rd - rc/w ;  dz = (-rc - z dw) / w
        for (size_t e = 0; e < K.size(); ++e) K[e] = Q[e];
        for (int i = 0; i < n; ++i) {
            K[(size_t)i * n + i] += z[i] / w[i];
            rhs[i] = -rd[i] - rc[i] / w[i];
        }
        if (!cholesky_solve(n, K, rhs)) return false;
        for (int i = 0; i < n; ++i) {
            ow[i] = rhs[i];
            oz[i] = (-rc[i] - z[i] * rhs[i]) / w[i];
        }
        return true;
    };
    auto step_to_boundary = [&](const std::vector<double>& a, const std::vector<double>& da) {
        double s = 1.0;
        for (int i = 0; i < n; ++i)
            if (da[i] < 0.0) s = std::min(s, -a[i] / da[i]);
        return s;
    };
    std::vector<double> rc(n);
    for (int it = 0; it < 200; ++it) {
        double mu = 0.0, rdn = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = f[i] - z[i];
            for (int k = 0; k < n; ++k) v += Q[(size_t)i * n + k] * w[k];
            rd[i] = v;
            rdn = std::max(rdn, std::fabs(v));
            mu += w[i] * z[i];
        }
        mu /= n;
        if (mu <= 1e-15 * scale && rdn <= 1e-13 * scale) {
            qp_polish(n, Q, f, w, z);
            return it;
        }
        for (int i = 0; i < n; ++i) rc[i] = w[i] * z[i];                      // affine step
        if (!newton(rc, dwa, dza)) return -1;
        const double aw = step_to_boundary(w, dwa), az = step_to_boundary(z, dza);
        double mua = 0.0;
        for (int i = 0; i < n; ++i) mua += (w[i] + aw * dwa[i]) * (z[i] + az * dza[i]);
        mua /= n;
        const double sigma = std::pow(mua / mu, 3.0);
        for (int i = 0; i < n; ++i) rc[i] = w[i] * z[i] + dwa[i] * dza[i] - sigma * mu;   // corrector
        if (!newton(rc, dw, dz)) return -1;
        const double a = std::min(1.0, 0.995 * std::min(step_to_boundary(w, dw), step_to_boundary(z, dz)));
        for (int i = 0; i < n; ++i) {
            w[i] = std::max(w[i] + a * dw[i], 1e-300);
            z[i] = std::max(z[i] + a * dz[i], 1e-300);
        }
    }
    return -2;
}

static double qp_value(int n, const std::vector<double>& Q, const std::vector<double>& f, const std::vector<double>& w) {
    double v = 0.0;
    for (int i = 0; i < n; ++i) {
        double qi = 0.0;
        for (int k = 0; k < n; ++k) qi += Q[(size_t)i * n + k] * w[k];
        v += w[i] * (0.5 * qi + f[i]);
    }
    return v;
}

// Polish an interior-point solution: the components with w_i > z_i are taken
// as free, the rest as zero, and the free block solves Q_FF w_F = -f_F (no
// free component: the candidate is w = 0).  The result is kept if it is
// non-negative and does not raise the objective (interior points approach a
// degenerate optimum, where the gradient vanishes on zero weights too, only
// like sqrt(mu)).
static void qp_polish(int n, const std::vector<double>& Q, const std::vector<double>& f, std::vector<double>& w,
                      const std::vector<double>& z) {
    std::vector<int> F;
    for (int i = 0; i < n; ++i)
        if (w[i] > z[i]) F.push_back(i);
    const int m = (int)F.size();
    if (m == 0) {
        const std::vector<double> w0(n, 0.0);
        if (qp_value(n, Q, f, w0) <= qp_value(n, Q, f, w)) w = w0;
        return;
    }
    std::vector<double> K((size_t)m * m), x(m);
    for (int a = 0; a < m; ++a) {
        x[a] = -f[F[a]];
        for (int b = 0; b < m; ++b) K[(size_t)a * m + b] = Q[(size_t)F[a] * n + F[b]];
    }
    if (!cholesky_solve(m, K, x)) return;
    std::vector<double> wp(n, 0.0);
    for (int a = 0; a < m; ++a) {
        if (x[a] < 0.0) return;
        wp[F[a]] = x[a];
    }
    if (qp_value(n, Q, f, wp) <= qp_value(n, Q, f, w)) w = wp;
}

extern "C" {

long long fp_m2_gram_bytes(int J) { return (long long)(J + 1) * (J + 1) * 16; }

int fp_m2_gram(const double* d_phi, const double* d_a, const double* d_S, const double* d_smax, int A, int J, int N,
               int C, int K1, const int* d_ks, int nk, double* d_G, void* stream) {
    if (!d_phi || !d_a || !d_S || !d_smax || !d_ks || !d_G) return fp_fail(FP_EINVAL, "fp_m2_gram: NULL buffer");
    if (A < 1 || J < 1 || N < 1 || C < 1 || K1 < 1 || nk < 1) return fp_fail(FP_EINVAL, "fp_m2_gram: bad sizes");
    GramArgs g;
    g.phi = (const double2*)d_phi;
    g.a = (const double2*)d_a;
    g.S = (const double2*)d_S;
    g.smax = d_smax;
    g.ks = d_ks;
    g.A = A; g.J = J; g.N = N; g.C = C; g.K1 = K1; g.nk = nk;
    g.R = (long long)A * N * C * nk;
    g.ntile = (J + 1 + M2_T - 1) / M2_T;
    g.G = (double2*)d_G;
    const int tiles = g.ntile * (g.ntile + 1) / 2;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long splits = (4LL * sms + tiles - 1) / tiles;
    const long long max_split = (g.R + M2_R - 1) / M2_R;
    if (splits > max_split) splits = max_split;
    if (splits > 65535) splits = 65535;
    g.rows_per_split = ((g.R + splits - 1) / splits + M2_R - 1) / M2_R * M2_R;
    splits = (g.R + g.rows_per_split - 1) / g.rows_per_split;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_G, 0, (size_t)fp_m2_gram_bytes(J), st) != cudaSuccess)
        return fp_fail(FP_ECUDA, "fp_m2_gram: clearing the output failed");
    fp_m2_gram_kernel<<<dim3(tiles, (unsigned)splits), M2_T * M2_T, 0, st>>>(g);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_m2_gram: launch failed");
    return FP_OK;
}

int fp_m2_solve(const double* h_G, int J, int s_rank, double* h_w, double* h_objective, double* h_residual,
                double* h_sv) {
    if (!h_G || !h_w || J < 1) return fp_fail(FP_EINVAL, "fp_m2_solve: bad argument");
    const int J1 = J + 1;
    // Hermitian: the products are read from the upper triangle (i <= j) only
    auto G = [&](int i, int j, int part) {
        if (i <= j) return h_G[((size_t)i * J1 + j) * 2 + part];
        const double v = h_G[((size_t)j * J1 + i) * 2 + part];
        return part == 0 ? v : -v;
    };
    // Hermitian M^H M as the real symmetric [[Re, -Im], [Im, Re]] of size 2J
    const int n2 = 2 * J;
    std::vector<double> H((size_t)n2 * n2), ev, V;
    for (int i = 0; i < J; ++i)
        for (int j = 0; j < J; ++j) {
            const double re = G(i, j, 0), im = G(i, j, 1);
            H[(size_t)i * n2 + j] = re;
            H[(size_t)(i + J) * n2 + (j + J)] = re;
            H[(size_t)i * n2 + (j + J)] = -im;
            H[(size_t)(i + J) * n2 + j] = im;
        }
    jacobi_eigen(n2, H, ev, V);
    std::vector<int> order(n2);
    for (int i = 0; i < n2; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
    // complex orthonormal eigenvectors v = x + i y, one per eigenvalue pair
    std::vector<double> vr, vi, lam;
    for (int o = 0; o < n2 && (int)lam.size() < J; ++o) {
        const int col = order[o];
        std::vector<double> xr(J), xi(J);
        for (int i = 0; i < J; ++i) { xr[i] = V[(size_t)i * n2 + col]; xi[i] = V[(size_t)(i + J) * n2 + col]; }
        for (size_t q = 0; q < lam.size(); ++q) {       // remove components along chosen vectors
            double pr = 0.0, pi = 0.0;                  // <v_q, x> = sum conj(v_q) x
            for (int i = 0; i < J; ++i) {
                const double ar = vr[q * J + i], ai = vi[q * J + i];
                pr += ar * xr[i] + ai * xi[i];
                pi += ar * xi[i] - ai * xr[i];
            }
            for (int i = 0; i < J; ++i) {
                const double ar = vr[q * J + i], ai = vi[q * J + i];
                xr[i] -= pr * ar - pi * ai;
                xi[i] -= pr * ai + pi * ar;
            }
        }
        double nrm = 0.0;
        for (int i = 0; i < J; ++i) nrm += xr[i] * xr[i] + xi[i] * xi[i];
        if (nrm < 0.25) continue;                       // the partner i v of a chosen vector
        nrm = 1.0 / std::sqrt(nrm);
        for (int i = 0; i < J; ++i) { vr.push_back(xr[i] * nrm); vi.push_back(xi[i] * nrm); }
        lam.push_back(std::max(ev[col], 0.0));
    }
    const int nv = (int)lam.size();
    if (h_sv)
        for (int k = 0; k < J; ++k) h_sv[k] = k < nv ? std::sqrt(lam[k]) : 0.0;
    // reduced problem: rows diag(s) V^H (M columns) and diag(1/s) V^H M^H y (data)
    const double smax = nv > 0 ? std::sqrt(lam[0]) : 0.0;
    int s = (s_rank > 0 && s_rank < nv) ? s_rank : nv;
    while (s > 0 && !(std::sqrt(lam[s - 1]) > 1e-13 * smax)) --s;     // drop numerically zero directions
    std::vector<double> Gr((size_t)2 * s * J), hr(2 * s);
    for (int k = 0; k < s; ++k) {
        const double sk = std::sqrt(lam[k]);
        double br = 0.0, bi = 0.0;                      // (V^H M^H y)_k
        for (int i = 0; i < J; ++i) {
            const double ar = vr[k * J + i], ai = vi[k * J + i];      // conj(v_ik) (M^H y)_i
            const double yr = G(i, J, 0), yi = G(i, J, 1);
            br += ar * yr + ai * yi;
            bi += ar * yi - ai * yr;
            Gr[(size_t)k * J + i] = sk * ar;             // s_k conj(v_ik)
            Gr[(size_t)(s + k) * J + i] = -sk * ai;
        }
        hr[k] = br / sk;
        hr[s + k] = bi / sk;
    }
    std::vector<double> Q((size_t)J * J, 0.0), f(J, 0.0), w;
    for (int r = 0; r < 2 * s; ++r)
        for (int i = 0; i < J; ++i) {
            const double gi = Gr[(size_t)r * J + i];
            f[i] -= gi * hr[r];
            for (int j = 0; j < J; ++j) Q[(size_t)i * J + j] += gi * Gr[(size_t)r * J + j];
        }
    // weights of dictionary columns that are zero in the truncated problem
    // (Q_ii = |column i|^2 = 0, hence f_i = 0) leave the objective unchanged:
    // they are set to 0 and the QP runs over the others
    double qmax = 0.0;
    for (int i = 0; i < J; ++i) qmax = std::max(qmax, Q[(size_t)i * J + i]);
    std::vector<int> act;
    for (int i = 0; i < J; ++i)
        if (Q[(size_t)i * J + i] > 1e-24 * qmax) act.push_back(i);
    const int na = (int)act.size();
    w.assign(J, 0.0);
    if (na > 0) {
        std::vector<double> Qa((size_t)na * na), fa(na), wa;
        for (int a = 0; a < na; ++a) {
            fa[a] = f[act[a]];
            for (int b = 0; b < na; ++b) Qa[(size_t)a * na + b] = Q[(size_t)act[a] * J + act[b]];
        }
        const int its = qp_nonneg(na, Qa, fa, wa);
        if (its < 0)
            return fp_fail(FP_EUNSUPPORTED, "fp_m2_solve: interior-point iteration did not converge (%d)", its);
        for (int a = 0; a < na; ++a) w[act[a]] = wa[a];
    }
    double obj = 0.0;                                    // ||Gr w - hr||^2
    for (int r = 0; r < 2 * s; ++r) {
        double v = -hr[r];
        for (int i = 0; i < J; ++i) v += Gr[(size_t)r * J + i] * w[i];
        obj += v * v;
    }
    for (int i = 0; i < J; ++i) h_w[i] = w[i];
    if (h_objective) *h_objective = obj;
    if (h_residual) {                                    // ||M w - y||^2 from the Gram matrix
        double r2 = G(J, J, 0);
        for (int i = 0; i < J; ++i) {
            r2 -= 2.0 * w[i] * G(i, J, 0);
            for (int j = 0; j < J; ++j) r2 += w[i] * w[j] * G(i, j, 0);
        }
        *h_residual = r2 > 0.0 ? r2 : 0.0;
    }
    return s;
}

}  // extern "C"
