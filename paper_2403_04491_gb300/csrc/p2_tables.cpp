// P2 reference tables (see p2_tables.h). Polynomials in the barycentric coordinates are kept as
// maps from exponent vectors to coefficients; every integral is a sum of moments.
#include "p2_tables.h"

#include <array>
#include <map>
#include <mutex>
#include <stdexcept>
#include <vector>

namespace knp {

namespace {

using Expo = std::array<int, 4>;
using Poly = std::map<Expo, double>;

double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// int over the unit-measure m-simplex of prod lambda_a^{e_a}
double moment(int m, const Expo& e) {
    double num = factorial(m);
    int s = 0;
    for (int k : e) {
        num *= factorial(k);
        s += k;
    }
    return num / factorial(m + s);
}

double integral(int m, const Poly& p) {
    double s = 0.0;
    for (const auto& [e, c] : p) s += c * moment(m, e);
    return s;
}

Poly mul(const Poly& p, const Poly& q) {
    Poly r;
    for (const auto& [ea, ca] : p)
        for (const auto& [eb, cb] : q) {
            Expo e;
            for (int k = 0; k < 4; ++k) e[k] = ea[k] + eb[k];
            r[e] += ca * cb;
        }
    return r;
}

Poly d_lambda(const Poly& p, int a) {
    Poly r;
    for (const auto& [e, c] : p)
        if (e[a] > 0) {
            Expo f = e;
            f[a] -= 1;
            r[f] += c * e[a];
        }
    return r;
}

Expo unit(int a) {
    Expo e{0, 0, 0, 0};
    e[a] = 1;
    return e;
}

Expo unit2(int a, int b) {
    Expo e{0, 0, 0, 0};
    e[a] += 1;
    e[b] += 1;
    return e;
}

// P2 basis of an m-simplex: vertices, then edges (a < b) in lexicographic order
std::vector<Poly> basis(int m) {
    std::vector<Poly> B;
    for (int a = 0; a <= m; ++a) B.push_back(Poly{{unit2(a, a), 2.0}, {unit(a), -1.0}});
    for (int a = 0; a <= m; ++a)
        for (int b = a + 1; b <= m; ++b) B.push_back(Poly{{unit2(a, b), 4.0}});
    return B;
}

// index of a monomial of degree <= 2 among 1, lambda_0..lambda_d, lambda_x lambda_y (x <= y)
int monomial_index(int d, const Expo& e) {
    int deg = 0;
    for (int k : e) deg += k;
    if (deg == 0) return 0;
    if (deg == 1) {
        for (int x = 0; x <= d; ++x)
            if (e[x]) return 1 + x;
    }
    int q = 1 + (d + 1);
    for (int x = 0; x <= d; ++x)
        for (int y = x; y <= d; ++y) {
            if ((x == y && e[x] == 2) || (x != y && e[x] == 1 && e[y] == 1)) return q;
            ++q;
        }
    throw std::logic_error("monomial of degree > 2");
}

void build(int d, P2Ref& R) {
    R.d = d;
    const std::vector<Poly> B = basis(d), Bf = basis(d - 1);
    R.npe = (int)B.size();
    R.nfn = (int)Bf.size();
    R.nmom = 1 + (d + 1) + (d + 1) * (d + 2) / 2;
    for (int j = 0; j < R.npe; ++j)
        for (int l = 0; l < R.npe; ++l) {
            R.mass[j][l] = integral(d, mul(B[j], B[l]));
            for (int a = 0; a <= d; ++a)
                for (int b = 0; b <= d; ++b) R.stiff[j][l][a][b] = integral(d, mul(d_lambda(B[j], a), d_lambda(B[l], b)));
        }
    for (int c = 0; c < R.nfn; ++c)
        for (int j = 0; j < R.nfn; ++j) {
            R.fmass[c][j] = integral(d - 1, mul(Bf[c], Bf[j]));
            for (int l = 0; l < R.nfn; ++l) R.ftriple[c][j][l] = integral(d - 1, mul(mul(Bf[c], Bf[j]), Bf[l]));
        }
    // moment matrix: row q is the monomial, column c the basis function
    std::vector<Expo> monos;
    monos.push_back(Expo{0, 0, 0, 0});
    for (int x = 0; x <= d; ++x) monos.push_back(unit(x));
    for (int x = 0; x <= d; ++x)
        for (int y = x; y <= d; ++y) monos.push_back(unit2(x, y));
    for (int q = 0; q < R.nmom; ++q)
        for (int c = 0; c < R.npe; ++c) R.mom[q][c] = integral(d, mul(B[c], Poly{{monos[q], 1.0}}));
    // off-diagonal pairs and their terms
    int p = 0, t = 0;
    for (int j = 0; j < R.npe; ++j)
        for (int l = j + 1; l < R.npe; ++l) {
            R.pj[p] = j;
            R.pl[p] = l;
            R.tptr[p] = t;
            for (int a = 0; a <= d; ++a) {
                const Poly Dj = d_lambda(B[j], a);
                if (Dj.empty()) continue;
                for (int b = 0; b <= d; ++b) {
                    const Poly Dl = d_lambda(B[l], b);
                    if (Dl.empty()) continue;
                    for (const auto& [e, c] : mul(Dj, Dl)) {
                        if (c == 0.0) continue;
                        if (t >= P2_NTERM_MAX) throw std::logic_error("P2 term table too small");
                        R.terms[t++] = P2Term{a, b, monomial_index(d, e), c};
                    }
                }
            }
            ++p;
        }
    R.npairs = p;
    R.tptr[p] = t;
    R.nterms = t;
}

}  // namespace

const P2Ref& p2_ref(int d) {
    static P2Ref tables[2];
    static std::once_flag once[2];
    if (d != 2 && d != 3) throw std::invalid_argument("P2 tables exist for d = 2 and 3");
    std::call_once(once[d - 2], [d] { build(d, tables[d - 2]); });
    return tables[d - 2];
}

const P2Dev& p2_dev(int d) {
    static P2Dev tables[2];
    static std::once_flag once[2];
    const P2Ref& R = p2_ref(d);
    std::call_once(once[d - 2], [&R, d] {
        P2Dev& T = tables[d - 2];
        T = P2Dev{};
        T.npe = R.npe;
        T.nfn = R.nfn;
        T.nmom = R.nmom;
        T.npairs = R.npairs;
        for (int p = 0; p <= R.npairs; ++p) T.tptr[p] = R.tptr[p];
        for (int t = 0; t < R.nterms; ++t) {
            T.tabq[t] = R.terms[t].a | (R.terms[t].b << 2) | (R.terms[t].q << 4);
            T.tcoef[t] = R.terms[t].coef;
        }
        for (int q = 0; q < P2_NMOM_MAX; ++q)
            for (int c = 0; c < P2_NPE_MAX; ++c) T.mom[q][c] = R.mom[q][c];
        for (int i = 0; i < P2_NFN_MAX; ++i)
            for (int j = 0; j < P2_NFN_MAX; ++j) {
                T.fmass[i][j] = R.fmass[i][j];
                for (int l = 0; l < P2_NFN_MAX; ++l) T.ftriple[i][j][l] = R.ftriple[i][j][l];
            }
    });
    return tables[d - 2];
}

}  // namespace knp
