// Radau IIA collocation constants (s = 3, 5, 7) derived on the host from the
// collocation definition, plus the transformation that decouples the
// simplified-Newton system and an embedded error formula.
//
//   nodes   c_i: zeros of d^{s-1}/dx^{s-1} [x^{s-1} (x - 1)^s]  (right Radau points)
//   a_ij  = int_0^{c_i} l_j(x) dx,  l_j the Lagrange basis on the nodes
//   a^{-1} = T Lam T^{-1},  Lam = diag(gam, [[alp_q, bet_q], [-bet_q, alp_q]] ...)
//   K     = T^{-1} a^{-1}
//   embedded formula of order s with an explicit stage at t_n of weight
//   g0 = 1/gam: sum_{i>=0} bh_i c_i^{q-1} = 1/q (q = 1..s), c_0 = 0;
//   err_pre = h g0 f(t_n, y_n) + sum_i e_i Z_i with e = (bh - b)^T a^{-1}.
#include <algorithm>
#include <complex>
#include <cmath>
#include <cstring>
#include <vector>
#include "fp_internal.h"

namespace {
typedef std::complex<double> cd;
typedef std::vector<double> Poly;     // ascending coefficients

Poly pmul(const Poly& a, const Poly& b) {
    Poly r(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
    return r;
}
Poly pder(const Poly& a) {
    Poly r(a.size() > 1 ? a.size() - 1 : 1, 0.0);
    for (size_t i = 1; i < a.size(); ++i) r[i - 1] = a[i] * (double)i;
    return r;
}
template <class T> T peval(const Poly& a, T x) {
    T r = 0.0;
    for (size_t i = a.size(); i-- > 0;) r = r * x + a[i];
    return r;
}
// all roots of a real polynomial (Durand-Kerner), then Newton polish
std::vector<cd> proots(const Poly& p) {
    int n = (int)p.size() - 1;
    Poly q = p;
    for (auto& v : q) v /= p[n];
    std::vector<cd> z(n);
    cd seed(0.4, 0.9);
    for (int i = 0; i < n; ++i) z[i] = std::pow(seed, i);
    for (int it = 0; it < 2000; ++it) {
        double mx = 0.0;
        for (int i = 0; i < n; ++i) {
            cd den = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (z[i] - z[j]);
            cd dz = peval(q, z[i]) / den;
            z[i] -= dz;
            mx = std::max(mx, std::abs(dz));
        }
        if (mx < 1e-15) break;
    }
    Poly dq = pder(q);
    for (auto& r : z)
        for (int it = 0; it < 5; ++it) {
            cd d = peval(dq, r);
            if (std::abs(d) == 0.0) break;
            r -= peval(q, r) / d;
        }
    return z;
}
// Gauss-Jordan inverse with partial pivoting (n <= 7)
template <class T> void ginv(int n, const T* A, T* B) {
    T M[7][14];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i * n + j] : (j - n == i ? T(1.0) : T(0.0));
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(M[i][k]) > std::abs(M[p][k])) p = i;
        for (int j = 0; j < 2 * n; ++j) std::swap(M[k][j], M[p][j]);
        T pv = M[k][k];
        for (int j = 0; j < 2 * n; ++j) M[k][j] /= pv;
        for (int i = 0; i < n; ++i)
            if (i != k) {
                T f = M[i][k];
                for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[k][j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) B[i * n + j] = M[i][j + n];
}
}  // namespace

int fp_build_radau(int s, FpRadau* r) {
    if (s != 3 && s != 5 && s != 7) return FP_EINVAL;
    std::memset(r, 0, sizeof(*r));
    r->s = s;
    // nodes
    Poly x1 = {0.0, 1.0}, xm1 = {-1.0, 1.0}, p = {1.0};
    for (int i = 0; i < s - 1; ++i) p = pmul(p, x1);
    for (int i = 0; i < s; ++i) p = pmul(p, xm1);
    for (int i = 0; i < s - 1; ++i) p = pder(p);
    std::vector<cd> z = proots(p);
    std::vector<double> c(s);
    for (int i = 0; i < s; ++i) c[i] = z[i].real();
    std::sort(c.begin(), c.end());
    c[s - 1] = 1.0;
    for (int i = 0; i < s; ++i) {                      // Newton polish on the real line
        if (i == s - 1) break;
        for (int it = 0; it < 5; ++it) {
            double d = peval(pder(p), c[i]);
            if (d == 0.0) break;
            c[i] -= peval(p, c[i]) / d;
        }
    }
    for (int i = 0; i < s; ++i) r->c[i] = c[i];
    // a_ij
    std::vector<double> a(s * s), ai(s * s);
    for (int j = 0; j < s; ++j) {
        Poly l = {1.0};
        for (int k = 0; k < s; ++k)
            if (k != j) l = pmul(l, Poly{-c[k] / (c[j] - c[k]), 1.0 / (c[j] - c[k])});
        Poly I(l.size() + 1, 0.0);
        for (size_t k = 0; k < l.size(); ++k) I[k + 1] = l[k] / (double)(k + 1);
        for (int i = 0; i < s; ++i) a[i * s + j] = peval(I, c[i]);
    }
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) r->a[i][j] = a[i * s + j];
    ginv(s, a.data(), ai.data());
    // eigenvalues of a^{-1} from its characteristic polynomial (Faddeev-LeVerrier)
    std::vector<double> M(s * s, 0.0), AM(s * s), coef(s + 1, 0.0);
    coef[s] = 1.0;
    for (int k = 1; k <= s; ++k) {
        // M_k = A M_{k-1} + c_{s-k+1} I ; c_{s-k} = -tr(A M_k)/k
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) {
                double v = 0.0;
                for (int q = 0; q < s; ++q) v += ai[i * s + q] * M[q * s + j];
                AM[i * s + j] = v;
            }
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) M[i * s + j] = AM[i * s + j] + (i == j ? coef[s - k + 1] : 0.0);
        double tr = 0.0;
        for (int i = 0; i < s; ++i)
            for (int q = 0; q < s; ++q) tr += ai[i * s + q] * M[q * s + i];
        coef[s - k] = -tr / k;
    }
    std::vector<cd> lam = proots(Poly(coef.begin(), coef.end()));
    // refine eigenpairs by inverse iteration
    auto eigvec = [&](cd& l, std::vector<cd>& v) {
        v.assign(s, cd(1.0, 0.3));
        std::vector<cd> Ms(s * s), Mi(s * s);
        for (int it = 0; it < 6; ++it) {
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < s; ++j) Ms[i * s + j] = ai[i * s + j] - (i == j ? l * (1.0 + 1e-13) : cd(0.0));
            ginv(s, Ms.data(), Mi.data());
            std::vector<cd> w(s, 0.0);
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < s; ++j) w[i] += Mi[i * s + j] * v[j];
            int km = 0;
            for (int i = 1; i < s; ++i)
                if (std::abs(w[i]) > std::abs(w[km])) km = i;
            cd nrm = w[km];
            for (int i = 0; i < s; ++i) v[i] = w[i] / nrm;
            cd av = 0.0;
            for (int j = 0; j < s; ++j) av += ai[km * s + j] * v[j];
            l = av / v[km];
        }
    };
    int ir = 0;
    for (int i = 1; i < s; ++i)
        if (std::fabs(lam[i].imag()) < std::fabs(lam[ir].imag())) ir = i;
    cd g = cd(lam[ir].real(), 0.0);
    std::vector<cd> v;
    eigvec(g, v);
    r->gam = g.real();
    for (int i = 0; i < s; ++i) r->T[i][0] = v[i].real();
    std::vector<cd> pos;
    for (int i = 0; i < s; ++i)
        if (i != ir && lam[i].imag() > 0) pos.push_back(lam[i]);
    std::sort(pos.begin(), pos.end(), [](cd x, cd y) { return x.real() < y.real(); });
    for (int q = 0; q < (int)pos.size(); ++q) {
        cd l = pos[q];
        eigvec(l, v);
        r->alp[q] = l.real();
        r->bet[q] = l.imag();
        for (int i = 0; i < s; ++i) {
            r->T[i][1 + 2 * q] = v[i].real();
            r->T[i][2 + 2 * q] = v[i].imag();
        }
    }
    std::vector<double> T(s * s), Ti(s * s);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) T[i * s + j] = r->T[i][j];
    ginv(s, T.data(), Ti.data());
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) {
            r->Ti[i][j] = Ti[i * s + j];
            double k = 0.0;
            for (int q = 0; q < s; ++q) k += Ti[i * s + q] * ai[q * s + j];
            r->K[i][j] = k;
        }
    // embedded formula
    r->g0 = 1.0 / r->gam;
    std::vector<double> V(s * s), Vi(s * s), rhs(s), bh(s, 0.0);
    for (int q = 0; q < s; ++q) {
        rhs[q] = 1.0 / (q + 1) - (q == 0 ? r->g0 : 0.0);
        for (int i = 0; i < s; ++i) V[q * s + i] = std::pow(c[i], q);
    }
    ginv(s, V.data(), Vi.data());
    for (int i = 0; i < s; ++i)
        for (int q = 0; q < s; ++q) bh[i] += Vi[i * s + q] * rhs[q];
    for (int j = 0; j < s; ++j) {
        double e = 0.0;
        for (int i = 0; i < s; ++i) e += (bh[i] - a[(s - 1) * s + i]) * ai[i * s + j];
        r->e[j] = e;
    }
    return FP_OK;
}
