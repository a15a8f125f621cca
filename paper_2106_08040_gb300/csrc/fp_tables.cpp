// Closed-form coupling coefficients of the Fokker-Planck operator (Sec. 2.1,
// Eq. FP-general with the drift of Eq. convection) in a real spherical-harmonic
// basis, easy-axis frame (n = z).  Host code, FP64.
//
// Basis: Y_{l,0} = Q_l^0(z); Y_{l,m} = sqrt2 Q_l^m cos(m p); Y_{l,-m} = sqrt2 Q_l^m sin(m p)
// (orthonormal, no Condon-Shortley phase), flat index l*l + l + m.
//
// With R = m x grad (rotation generators) and M_k = multiplication by m_k, the
// operator of dc/dt = A c is
//   A = -D Lap - p3 M_z R_z - (p4/2) W - sum_k p1 B_k R_k - sum_k p2 B_k G_k
// where, for u = m_k and w = (n.m)^2 = z^2 (identities on the sphere:
// Lap m_k = -2 m_k, Lap w = -6 w + 2, div(f grad u) = (Lap(uf) - u Lap f + f Lap u)/2):
//   G_k Y_l = -(l+2) Proj_{l+1}(m_k Y_l) + (l-1) Proj_{l-1}(m_k Y_l)
//   W Y_l   = sum_{l'=l,l+-2} [ (l(l+1) - l'(l'+1))/2 - 3 ] Proj_{l'}(w Y_l) + Y_l
// Precession: div((H x m) f) = H . R f, and div((n.m)(n x m) f) = (n.m)(n.R) f.
//
// Closed forms used:
//   z Y_{l,m} = a(l,|m|) Y_{l+1,m} + a(l-1,|m|) Y_{l-1,m},
//       a(l, mu) = sqrt(((l+1)^2 - mu^2) / ((2l+1)(2l+3)))
//   R_z Y_{l,m} = -m Y_{l,-m} (m > 0), R_z Y_{l,-m} = m Y_{l,m}
//   R_x, R_y from the angular-momentum ladder operators of the complex basis
//       (L+- Y^m = sqrt((l -+ m)(l +- m + 1)) Y^{m+-1}, R = i L), transformed
//       to the real basis per degree l;
//   x = [M_z, R_y]-form: M_x = M_z R_y - R_y M_z, M_y = R_x M_z - M_z R_x
//       (since R_y z = -x, R_x z = y).
#include <complex>
#include <map>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include "fp_internal.h"

namespace {

typedef std::map<std::pair<int, int>, double> SpMat;   // (target, source) -> value

inline int gi(int l, int m) { return l * l + l + m; }
inline void lm_of(int i, int& l, int& m) {
    l = (int)std::floor(std::sqrt((double)i) + 1e-9);
    while ((l + 1) * (l + 1) <= i) ++l;
    while (l * l > i) --l;
    m = i - l * l - l;
}

double a_coef(int l, int mu) {
    if (l < 0 || l < mu) return 0.0;
    return std::sqrt((double)((l + 1) * (l + 1) - mu * mu) / (double)((2 * l + 1) * (2 * l + 3)));
}

// multiplication by z, degrees 0..Lmax (targets may reach Lmax+1)
SpMat build_Mz(int Lmax) {
    SpMat M;
    for (int l = 0; l <= Lmax; ++l)
        for (int m = -l; m <= l; ++m) {
            int mu = std::abs(m);
            double up = a_coef(l, mu), dn = a_coef(l - 1, mu);
            if (up != 0.0) M[{gi(l + 1, m), gi(l, m)}] = up;
            if (l - 1 >= mu && dn != 0.0) M[{gi(l - 1, m), gi(l, m)}] = dn;
        }
    return M;
}

SpMat build_Rz(int Lmax) {
    SpMat R;
    for (int l = 0; l <= Lmax; ++l)
        for (int m = 1; m <= l; ++m) {
            R[{gi(l, -m), gi(l, m)}] = -(double)m;
            R[{gi(l, m), gi(l, -m)}] = (double)m;
        }
    return R;
}

// R_x and R_y in the real basis, per degree l, via the complex ladder operators.
void build_Rxy(int Lmax, SpMat& Rx, SpMat& Ry) {
    typedef std::complex<double> cd;
    const cd I(0.0, 1.0);
    const double s2 = std::sqrt(2.0);
    for (int l = 0; l <= Lmax; ++l) {
        int n = 2 * l + 1;
        auto ci = [l](int m) { return m + l; };            // complex index
        std::vector<cd> Rxc(n * n, 0.0), Ryc(n * n, 0.0);  // [target][source]
        for (int m = -l; m <= l; ++m) {
            if (m + 1 <= l) {
                double lp = std::sqrt((double)(l - m) * (l + m + 1));
                Rxc[ci(m + 1) * n + ci(m)] += I * 0.5 * lp;
                Ryc[ci(m + 1) * n + ci(m)] += 0.5 * lp;
            }
            if (m - 1 >= -l) {
                double lm = std::sqrt((double)(l + m) * (l - m + 1));
                Rxc[ci(m - 1) * n + ci(m)] += I * 0.5 * lm;
                Ryc[ci(m - 1) * n + ci(m)] += -0.5 * lm;
            }
        }
        // U[a][m]: real function a = sum_m U[a][m] Y^m (complex, CS phase)
        std::vector<cd> U(n * n, 0.0);
        U[ci(0) * n + ci(0)] = 1.0;
        for (int mu = 1; mu <= l; ++mu) {
            double sg = (mu % 2) ? -1.0 : 1.0;
            U[ci(mu) * n + ci(mu)] = sg / s2;
            U[ci(mu) * n + ci(-mu)] = 1.0 / s2;
            U[ci(-mu) * n + ci(mu)] = sg / (s2 * I);
            U[ci(-mu) * n + ci(-mu)] = -1.0 / (s2 * I);
        }
        // R Y_a = sum_m U[a][m] sum_m' Rc[m'][m] Y^m', Y^m' = sum_b conj(U[b][m']) Y_b
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                cd sx = 0.0, sy = 0.0;
                for (int m = 0; m < n; ++m) {
                    if (U[a * n + m] == cd(0.0)) continue;
                    for (int mp = 0; mp < n; ++mp) {
                        cd v = std::conj(U[b * n + mp]) * U[a * n + m];
                        sx += v * Rxc[mp * n + m];
                        sy += v * Ryc[mp * n + m];
                    }
                }
                int ta = gi(l, b - l), so = gi(l, a - l);   // target b, source a
                if (std::abs(sx) > 1e-13) Rx[{ta, so}] = sx.real();
                if (std::abs(sy) > 1e-13) Ry[{ta, so}] = sy.real();
            }
    }
}

SpMat matmul(const SpMat& A, const SpMat& B) {      // (A B)[t][s] = sum_k A[t][k] B[k][s]
    std::map<int, std::vector<std::pair<int, double>>> Bcol;   // k -> (s, val) rows of B by k
    for (auto& e : B) Bcol[e.first.first].push_back({e.first.second, e.second});
    SpMat C;
    for (auto& e : A) {
        auto it = Bcol.find(e.first.second);
        if (it == Bcol.end()) continue;
        for (auto& bs : it->second) C[{e.first.first, bs.first}] += e.second * bs.second;
    }
    return C;
}

SpMat sub(const SpMat& A, const SpMat& B) {
    SpMat C = A;
    for (auto& e : B) C[e.first] -= e.second;
    return C;
}

}  // namespace

int fp_build_tables(int L, FpTablesHost* out) {
    const int N = (L + 1) * (L + 1);
    std::memset(out, 0, sizeof(*out));
    out->L = L;
    out->N = N;
    out->coef = (double*)std::calloc((size_t)N * FP_NSLOT, sizeof(double));
    out->src = (int*)std::malloc((size_t)N * FP_NSLOT * sizeof(int));
    out->lam = (double*)std::calloc(N, sizeof(double));
    out->wdiag = (double*)std::calloc(N, sizeof(double));
    out->tslot = (int*)std::malloc((size_t)N * FP_NSLOT * sizeof(int));
    if (!out->coef || !out->src || !out->lam || !out->wdiag || !out->tslot) { fp_free_tables(out); return FP_ENOMEM; }
    for (int i = 0; i < N * FP_NSLOT; ++i) { out->src[i] = -1; out->tslot[i] = -1; }

    SpMat Mz = build_Mz(L + 1);
    SpMat Rz = build_Rz(L + 1);
    SpMat Rx, Ry;
    build_Rxy(L + 1, Rx, Ry);
    SpMat Mx = sub(matmul(Mz, Ry), matmul(Ry, Mz));
    SpMat My = sub(matmul(Rx, Mz), matmul(Mz, Rx));
    SpMat Mz2 = matmul(Mz, Mz);
    SpMat ZRz = matmul(Mz, Rz);

    auto in_range = [N](int t, int s) { return t < N && s < N; };
    auto put = [&](int t, int slot, int s, double v) {
        out->coef[t * FP_NSLOT + slot] = v;
        out->src[t * FP_NSLOT + slot] = s;
    };
    for (int t = 0; t < N; ++t) {
        int l, m;
        lm_of(t, l, m);
        out->lam[t] = (double)l * (l + 1);
    }
    // W (anisotropy damping) from z^2
    for (auto& e : Mz2) {
        int t = e.first.first, s = e.first.second;
        if (!in_range(t, s)) continue;
        int lt, mt, ls, ms;
        lm_of(t, lt, mt); lm_of(s, ls, ms);
        double f = 0.5 * ((double)ls * (ls + 1) - (double)lt * (lt + 1)) - 3.0;
        double v = e.second * f;
        if (lt == ls) out->wdiag[t] = v + 1.0;
        else if (lt == ls + 2) put(t, SL_W + 0, s, v);
        else if (lt == ls - 2) put(t, SL_W + 1, s, v);
    }
    for (auto& e : ZRz) {
        int t = e.first.first, s = e.first.second;
        if (!in_range(t, s) || e.second == 0.0) continue;
        int lt, mt, ls, ms;
        lm_of(t, lt, mt); lm_of(s, ls, ms);
        put(t, lt == ls + 1 ? SL_ZR + 0 : SL_ZR + 1, s, e.second);
    }
    for (auto& e : Rz) {
        int t = e.first.first, s = e.first.second;
        if (in_range(t, s)) put(t, SL_RZ, s, e.second);
    }
    auto put_lat = [&](const SpMat& R, int base) {       // same-l, |m| +- 1
        for (auto& e : R) {
            int t = e.first.first, s = e.first.second;
            if (!in_range(t, s) || std::fabs(e.second) < 1e-15) continue;
            int lt, mt, ls, ms;
            lm_of(t, lt, mt); lm_of(s, ls, ms);
            put(t, base + (std::abs(ms) < std::abs(mt) ? 0 : 1), s, e.second);
        }
    };
    put_lat(Rx, SL_RX);
    put_lat(Ry, SL_RY);
    auto put_G = [&](const SpMat& M, int base, bool same_m) {
        for (auto& e : M) {
            int t = e.first.first, s = e.first.second;
            if (!in_range(t, s) || std::fabs(e.second) < 1e-15) continue;
            int lt, mt, ls, ms;
            lm_of(t, lt, mt); lm_of(s, ls, ms);
            double f = (lt == ls + 1) ? -(double)(ls + 2) : (double)(ls - 1);
            if (f == 0.0) continue;
            int slot;
            if (same_m) slot = base + (lt == ls + 1 ? 0 : 1);          // source l-1 / l+1
            else slot = base + 2 * (lt == ls + 1 ? 0 : 1) + (std::abs(ms) < std::abs(mt) ? 0 : 1);
            put(t, slot, s, e.second * f);
        }
    };
    put_G(Mz, SL_GZ, true);
    put_G(Mx, SL_GX, false);
    put_G(My, SL_GY, false);
    // transpose slot of every lateral (|m| +- 1) coupling: the slot of row `src`
    // whose source is the present row (the coupling pattern is symmetric)
    for (int t = 0; t < N; ++t)
        for (int k = SL_RX; k < FP_NSLOT; ++k) {
            if (k >= SL_GZ && k < SL_GX) continue;
            int s = out->src[t * FP_NSLOT + k];
            if (s < 0) continue;
            for (int k2 = SL_RX; k2 < FP_NSLOT; ++k2)
                if (out->src[s * FP_NSLOT + k2] == t) { out->tslot[t * FP_NSLOT + k] = k2; break; }
        }
    return FP_OK;
}

void fp_free_tables(FpTablesHost* t) {
    std::free(t->coef); std::free(t->src); std::free(t->lam); std::free(t->wdiag); std::free(t->tslot);
    t->coef = nullptr; t->src = nullptr; t->lam = nullptr; t->wdiag = nullptr; t->tslot = nullptr;
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
void fp_gauss_legendre(int n, double* x, double* w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ---- block structure for one degree L (rows in block order) ---------------
namespace {
inline int slot_group(int k) {     // W, ZR, RZ, RX, RY, GZ, GX, GY
    return k < 2 ? 0 : k < 4 ? 1 : k < 5 ? 2 : k < 7 ? 3 : k < 9 ? 4 : k < 11 ? 5 : k < 15 ? 6 : 7;
}
inline int nblock(int mu, int L) { return mu == 0 ? L + 1 : 2 * (L + 1 - mu); }
}  // namespace

int fp_build_blocks(const FpTablesHost* t, int L, FpBlkHost* out) {
    std::memset(out, 0, sizeof(*out));
    if (L > t->L) return FP_EINVAL;
    const int N = (L + 1) * (L + 1);
    out->L = L;
    out->N = N;
    out->glob = (int*)std::malloc(sizeof(int) * N);
    out->sb_k = (unsigned char*)std::malloc((size_t)N * FP_NSB);
    out->sb_g = (unsigned char*)std::calloc((size_t)N * FP_NSB, 1);
    out->sb_cf = (float*)std::calloc((size_t)N * FP_NSB, sizeof(float));
    out->dn_k = (unsigned char*)std::malloc((size_t)N * FP_NLT);
    out->dn_g = (unsigned char*)std::calloc((size_t)N * FP_NLT, 1);
    out->dn_cf = (float*)std::calloc((size_t)N * FP_NLT, sizeof(float));
    out->up_k = (unsigned char*)std::malloc((size_t)N * FP_NLT);
    out->up_g = (unsigned char*)std::calloc((size_t)N * FP_NLT, 1);
    out->up_cf = (float*)std::calloc((size_t)N * FP_NLT, sizeof(float));
    out->dnT = (unsigned char*)std::malloc((size_t)N * FP_NLT);
    out->upT = (unsigned char*)std::malloc((size_t)N * FP_NLT);
    if (!out->glob || !out->sb_k || !out->sb_g || !out->sb_cf || !out->dn_k || !out->dn_g || !out->dn_cf ||
        !out->up_k || !out->up_g || !out->up_cf || !out->dnT || !out->upT) {
        fp_free_blocks(out);
        return FP_ENOMEM;
    }
    std::memset(out->sb_k, 255, (size_t)N * FP_NSB);
    std::memset(out->dn_k, 255, (size_t)N * FP_NLT);
    std::memset(out->up_k, 255, (size_t)N * FP_NLT);
    std::memset(out->dnT, 255, (size_t)N * FP_NLT);
    std::memset(out->upT, 255, (size_t)N * FP_NLT);
    std::vector<int> boff(L + 2, 0), blk_of(N), loc_of(N), brow(N);
    for (int mu = 0; mu <= L; ++mu) boff[mu + 1] = boff[mu] + nblock(mu, L);
    for (int g = 0; g < N; ++g) {
        int l, m;
        lm_of(g, l, m);
        int mu = std::abs(m), k = mu == 0 ? l : 2 * (l - mu) + (m < 0 ? 1 : 0);
        blk_of[g] = mu;
        loc_of[g] = k;
        brow[g] = boff[mu] + k;
        out->glob[boff[mu] + k] = g;
    }
    for (int g = 0; g < N; ++g) {
        const int b = brow[g], mu = blk_of[g];
        int nsb = 0, ndn = 0, nup = 0;
        for (int k = 0; k < FP_NSLOT; ++k) {
            int j = t->src[g * FP_NSLOT + k];
            if (j < 0 || j >= N) continue;
            double cf = t->coef[g * FP_NSLOT + k];
            if (cf == 0.0) continue;
            int mj = blk_of[j];
            unsigned char kj = (unsigned char)loc_of[j], gr = (unsigned char)slot_group(k);
            if (mj == mu) {
                out->sb_k[b * FP_NSB + nsb] = kj; out->sb_g[b * FP_NSB + nsb] = gr;
                out->sb_cf[b * FP_NSB + nsb] = (float)cf; ++nsb;
            } else if (mj == mu - 1) {
                out->dn_k[b * FP_NLT + ndn] = kj; out->dn_g[b * FP_NLT + ndn] = gr;
                out->dn_cf[b * FP_NLT + ndn] = (float)cf; ++ndn;
            } else if (mj == mu + 1) {
                out->up_k[b * FP_NLT + nup] = kj; out->up_g[b * FP_NLT + nup] = gr;
                out->up_cf[b * FP_NLT + nup] = (float)cf; ++nup;
            }
            if (nsb > FP_NSB || ndn > FP_NLT || nup > FP_NLT) { fp_free_blocks(out); return FP_EINVAL; }
        }
    }
    // make the dn/up patterns mutually symmetric: row (0,0) of A vanishes (mass
    // conservation) while its column does not, so add explicit zero couplings
    // where only the reverse direction exists (the transposed solve needs them)
    auto add_if_missing = [&](unsigned char* kl, unsigned char* gl, float* cl, int row, int kloc) -> bool {
        for (int q = 0; q < FP_NLT; ++q)
            if (kl[row * FP_NLT + q] == kloc) return true;
        for (int q = 0; q < FP_NLT; ++q)
            if (kl[row * FP_NLT + q] == 255) {
                kl[row * FP_NLT + q] = (unsigned char)kloc; gl[row * FP_NLT + q] = 0; cl[row * FP_NLT + q] = 0.f;
                return true;
            }
        return false;
    };
    for (int b = 0; b < N; ++b) {
        int g = out->glob[b], mu = blk_of[g];
        for (int p = 0; p < FP_NLT; ++p) {
            int kd = out->dn_k[b * FP_NLT + p];
            if (kd != 255 && !add_if_missing(out->up_k, out->up_g, out->up_cf, boff[mu - 1] + kd, loc_of[g])) {
                fp_free_blocks(out); return FP_EINVAL;
            }
            int ku = out->up_k[b * FP_NLT + p];
            if (ku != 255 && !add_if_missing(out->dn_k, out->dn_g, out->dn_cf, boff[mu + 1] + ku, loc_of[g])) {
                fp_free_blocks(out); return FP_EINVAL;
            }
        }
    }
    // back pointers: for dn partner p of row b, the slot of the partner's up list that points to b
    for (int b = 0; b < N; ++b) {
        int g = out->glob[b], mu = blk_of[g];
        for (int p = 0; p < FP_NLT; ++p) {
            int kj = out->dn_k[b * FP_NLT + p];
            if (kj == 255) continue;
            int bp = boff[mu - 1] + kj;
            for (int q = 0; q < FP_NLT; ++q)
                if (out->up_k[bp * FP_NLT + q] == loc_of[g]) { out->dnT[b * FP_NLT + p] = (unsigned char)q; break; }
        }
        for (int p = 0; p < FP_NLT; ++p) {
            int ku = out->up_k[b * FP_NLT + p];
            if (ku == 255) continue;
            int bp = boff[mu + 1] + ku;
            for (int q = 0; q < FP_NLT; ++q)
                if (out->dn_k[bp * FP_NLT + q] == loc_of[g]) { out->upT[b * FP_NLT + p] = (unsigned char)q; break; }
        }
    }
    return FP_OK;
}

int fp_build_columns(const FpTablesHost* t, FpPair* out) {
    const int N = t->N;
    std::vector<int> cnt(N, 0);
    for (int i = 0; i < N * FP_NCT; ++i) out[i] = FpPair{-1, 0};
    for (int r = 0; r < N; ++r)
        for (int k = 0; k < FP_NSLOT; ++k) {
            int j = t->src[r * FP_NSLOT + k];
            if (j < 0 || j >= N) continue;
            if (cnt[j] >= FP_NCT) return FP_EINVAL;
            out[j * FP_NCT + cnt[j]++] = FpPair{r, k};
        }
    return FP_OK;
}

// The forward apply groups the slots by the scalar that multiplies them:
// -(p4/2) W - p3 M_zR_z = -p3 (M_zR_z + (alpha/2) W) and, per easy-axis-frame
// field component k, -p1 B_k R_k - p2 B_k G_k = -p1 B_k (R_k + alpha G_k)
// (p4 = alpha p3, p2 = alpha p1, Sec. 2.1), so the W and G coefficients are
// stored pre-multiplied by alpha/2 and alpha.
void fp_build_coef4(const FpTablesHost* t, double alpha, double* out) {
    for (int r = 0; r < t->N; ++r)
        for (int k = 0; k < FP_NSLOT; ++k) {
            const double f = k < SL_ZR ? 0.5 * alpha : k >= SL_GZ ? alpha : 1.0;
            out[r * FP_NSLOT + k] = f * t->coef[r * FP_NSLOT + k];
        }
}

void fp_free_blocks(FpBlkHost* b) {
    std::free(b->glob); std::free(b->sb_k); std::free(b->sb_g); std::free(b->sb_cf);
    std::free(b->dn_k); std::free(b->dn_g); std::free(b->dn_cf);
    std::free(b->up_k); std::free(b->up_g); std::free(b->up_cf); std::free(b->dnT); std::free(b->upT);
    std::memset(b, 0, sizeof(*b));
}
