// Hierarchic basis tables (host, FP64), computed once per order p.
//
// Polynomials in the four barycentric variables are held as maps from packed
// exponents to coefficients.  Integrals over the element use the classical
// simplex formula  (1/|T|) int_T lam^a = 3! a0! a1! a2! a3! / (|a| + 3)!.
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>

#include "rve_internal.h"

namespace rve {
namespace {

using Exp = std::array<int, 4>;
using Poly = std::map<Exp, double>;

Poly mono(int a, int b = -1, int c = -1) {
    Exp e{0, 0, 0, 0};
    if (a >= 0) e[a]++;
    if (b >= 0) e[b]++;
    if (c >= 0) e[c]++;
    return Poly{{e, 1.0}};
}
Poly constant(double v) { return Poly{{Exp{0, 0, 0, 0}, v}}; }

Poly mul(const Poly& x, const Poly& y) {
    Poly r;
    for (auto& [ex, cx] : x)
        for (auto& [ey, cy] : y) {
            Exp e{ex[0] + ey[0], ex[1] + ey[1], ex[2] + ey[2], ex[3] + ey[3]};
            r[e] += cx * cy;
        }
    return r;
}
Poly add(const Poly& x, const Poly& y, double sy = 1.0) {
    Poly r = x;
    for (auto& [e, c] : y) r[e] += sy * c;
    return r;
}
// derivative with respect to lam_a treating the four variables as independent
Poly dlam(const Poly& x, int a) {
    Poly r;
    for (auto& [e, c] : x)
        if (e[a] > 0) {
            Exp f = e;
            f[a]--;
            r[f] += c * e[a];
        }
    return r;
}
// d/dxi_k with xi_k = lam_k (k = 1..3) and lam_0 = 1 - xi_1 - xi_2 - xi_3
Poly dxi(const Poly& x, int k) { return add(dlam(x, k + 1), dlam(x, 0), -1.0); }

double fact(int n) {
    double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}
double mean(const Poly& x) {
    double s = 0;
    for (auto& [e, c] : x) {
        int deg = e[0] + e[1] + e[2] + e[3];
        s += c * 6.0 * fact(e[0]) * fact(e[1]) * fact(e[2]) * fact(e[3]) / fact(deg + 3);
    }
    return s;
}

std::vector<Poly> hierarchic(int p) {
    static const int edges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    static const int faces[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    std::vector<Poly> f;
    for (int a = 0; a < 4; ++a) f.push_back(mono(a));
    if (p >= 2)
        for (auto& e : edges) f.push_back(mono(e[0], e[1]));
    if (p >= 3) {
        for (auto& e : edges) f.push_back(mul(mono(e[0], e[1]), add(mono(e[1]), mono(e[0]), -1.0)));
        for (auto& t : faces) f.push_back(mono(t[0], t[1], t[2]));
    }
    return f;
}

// monomial spanning set of P_q in (lam_1, lam_2, lam_3), constant first
std::vector<Poly> spanning(int q) {
    std::vector<Poly> s{constant(1.0)};
    if (q >= 1)
        for (int a = 1; a <= 3; ++a) s.push_back(mono(a));
    if (q >= 2)
        for (int a = 1; a <= 3; ++a)
            for (int b = a; b <= 3; ++b) s.push_back(mono(a, b));
    return s;
}

Basis make_basis(int p) {
    Basis B;
    B.p = p;
    auto phi = hierarchic(p);
    B.ne = (int)phi.size();
    auto mu = spanning(p - 1);
    const int nm = (int)mu.size();
    B.nm = nm;
    // Gram matrix and its Cholesky factor: psi = L^{-1} mu is orthonormal
    std::vector<double> G(nm * nm), L(nm * nm, 0.0);
    for (int i = 0; i < nm; ++i)
        for (int j = 0; j < nm; ++j) G[i * nm + j] = mean(mul(mu[i], mu[j]));
    for (int j = 0; j < nm; ++j) {
        double s = G[j * nm + j];
        for (int k = 0; k < j; ++k) s -= L[j * nm + k] * L[j * nm + k];
        if (s <= 0) throw std::runtime_error("basis Gram matrix not SPD");
        L[j * nm + j] = std::sqrt(s);
        for (int i = j + 1; i < nm; ++i) {
            double t = G[i * nm + j];
            for (int k = 0; k < j; ++k) t -= L[i * nm + k] * L[j * nm + k];
            L[i * nm + j] = t / L[j * nm + j];
        }
    }
    // projections onto mu, then forward substitution with L gives psi-coefficients
    B.A.assign(3 * nm * B.ne, 0.0);
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < B.ne; ++j) {
            Poly g = dxi(phi[j], k);
            std::vector<double> proj(nm), c(nm);
            for (int n = 0; n < nm; ++n) proj[n] = mean(mul(g, mu[n]));
            for (int m = 0; m < nm; ++m) {
                double t = proj[m];
                for (int n = 0; n < m; ++n) t -= L[m * nm + n] * c[n];
                c[m] = t / L[m * nm + m];
            }
            for (int m = 0; m < nm; ++m) B.A[(k * nm + m) * B.ne + j] = c[m];
        }
    return B;
}

}  // namespace

const Basis& basis(int p) {
    static Basis tables[3];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int q = 1; q <= 3; ++q) tables[q - 1] = make_basis(q);
    });
    if (p < 1 || p > 3) throw std::runtime_error("p out of range");
    return tables[p - 1];
}

}  // namespace rve
