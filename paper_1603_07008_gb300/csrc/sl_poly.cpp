// sl_poly.cpp -- exact construction of the update matrices A(alpha), B(alpha)
// (Sec. II-A, update rule) as polynomials in alpha, on the host.
//
//   A_jl(alpha) = (2j+1)/2 int_{2alpha-1}^{1}  P_j(xi) P_l(xi - 2 alpha)     dxi
//   B_jl(alpha) = (2j+1)/2 int_{-1}^{2alpha-1} P_j(xi) P_l(xi + 2 - 2 alpha) dxi
//
// The target cell's polynomial is the source polynomial translated by
// sigma + alpha cells: on xi in [2alpha-1, 1] it is source cell i-sigma at
// xi - 2alpha, on [-1, 2alpha-1] source cell i-sigma-1 at xi + 2 - 2alpha;
// projecting onto P_j with eq. (cj) gives the integrals above.  The
// integrands are polynomials in (xi, alpha), so the integrals are computed
// symbolically in exact rational arithmetic and each coefficient is rounded
// once to FP64.  The result is re-expanded around alpha = 1/2, where Horner's
// rule keeps the rounding error at a few ulps for every degree up to 3.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sl_internal.cuh"

namespace sl {
namespace {

using i128 = __int128;

i128 gcd128(i128 a, i128 b)
{
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
        i128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

struct Q {
    i128 p = 0, q = 1;
    Q() = default;
    Q(long long v) : p(v), q(1) {}
    Q(i128 a, i128 b) : p(a), q(b) { norm(); }
    void norm()
    {
        if (q < 0) {
            p = -p;
            q = -q;
        }
        i128 g = gcd128(p, q);
        if (g > 1) {
            p /= g;
            q /= g;
        }
        if (p == 0) q = 1;
    }
    Q operator+(const Q& o) const { return Q(p * o.q + o.p * q, q * o.q); }
    Q operator-(const Q& o) const { return Q(p * o.q - o.p * q, q * o.q); }
    Q operator*(const Q& o) const { return Q(p * o.p, q * o.q); }
    Q operator/(const Q& o) const { return Q(p * o.q, q * o.p); }
    double to_double() const
    {
        // |p|, q < 2^53 here, so both convert exactly and the division is
        // the single rounding.
        return double((long long)p) / double((long long)q);
    }
};

constexpr int D = 2 * kMaxK + 3;   // max degree + headroom in each variable

// bivariate polynomial sum c[i][k] xi^i alpha^k
struct P2 {
    Q c[D][D];
};

P2 mul(const P2& x, const P2& y)
{
    P2 r;
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) {
            if (x.c[i][k].p == 0) continue;
            for (int j = 0; i + j < D; ++j)
                for (int l = 0; k + l < D; ++l) {
                    if (y.c[j][l].p == 0) continue;
                    r.c[i + j][k + l] = r.c[i + j][k + l] + x.c[i][k] * y.c[j][l];
                }
        }
    return r;
}

// Legendre P_n as univariate coefficients (three-term recurrence).
std::vector<Q> legendre_coeffs(int n)
{
    std::vector<Q> p0(D), p1(D);
    p0[0] = Q(1);
    if (n == 0) return p0;
    p1[1] = Q(1);
    for (int m = 1; m < n; ++m) {
        std::vector<Q> p2(D);
        for (int i = 0; i + 1 < D; ++i) p2[i + 1] = p2[i + 1] + Q(2 * m + 1) * p1[i];
        for (int i = 0; i < D; ++i) p2[i] = p2[i] - Q(m) * p0[i];
        for (int i = 0; i < D; ++i) p2[i] = p2[i] / Q(m + 1);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// P_n(xi + c1 alpha + c0) as a bivariate polynomial.
P2 legendre_shifted(int n, long long c1, long long c0)
{
    std::vector<Q> pc = legendre_coeffs(n);
    P2 lin;
    lin.c[1][0] = Q(1);
    lin.c[0][1] = Q(c1);
    lin.c[0][0] = Q(c0);
    P2 pw;
    pw.c[0][0] = Q(1);
    P2 r;
    for (int b = 0; b <= n; ++b) {
        for (int i = 0; i < D; ++i)
            for (int k = 0; k < D; ++k) r.c[i][k] = r.c[i][k] + pc[b] * pw.c[i][k];
        pw = mul(pw, lin);
    }
    return r;
}

// F(xi, alpha) evaluated at xi = u1 alpha + u0, a polynomial in alpha.
std::vector<Q> eval_at_linear(const P2& F, long long u1, long long u0)
{
    std::vector<Q> res(D);
    P2 lin;
    lin.c[0][1] = Q(u1);
    lin.c[0][0] = Q(u0);
    P2 pw;
    pw.c[0][0] = Q(1);
    for (int i = 0; i < D; ++i) {
        // add F.c[i][*] * (u1 alpha + u0)^i; pw holds the power in its xi^0 row
        for (int k = 0; k < D; ++k) {
            if (F.c[i][k].p == 0) continue;
            for (int l = 0; k + l < D; ++l) res[k + l] = res[k + l] + F.c[i][k] * pw.c[0][l];
        }
        pw = mul(pw, lin);
    }
    return res;
}

// (2j+1)/2 * int_{lower}^{upper} P_j(xi) P_l(xi + c1 alpha + c0) dxi
// with lower = l1 alpha + l0, upper = u1 alpha + u0.
std::vector<Q> entry(int j, int l, long long c1, long long c0, long long l1, long long l0,
                     long long u1, long long u0)
{
    std::vector<Q> pj = legendre_coeffs(j);
    P2 Pj;
    for (int i = 0; i < D; ++i) Pj.c[i][0] = pj[i];
    P2 R = mul(Pj, legendre_shifted(l, c1, c0));
    P2 F;   // antiderivative in xi
    for (int i = 0; i + 1 < D; ++i)
        for (int k = 0; k < D; ++k) F.c[i + 1][k] = R.c[i][k] / Q(i + 1);
    std::vector<Q> up = eval_at_linear(F, u1, u0), lo = eval_at_linear(F, l1, l0);
    std::vector<Q> r(D);
    for (int k = 0; k < D; ++k) r[k] = (up[k] - lo[k]) * Q(i128(2 * j + 1), i128(2));
    return r;
}

// Re-expand sum_k c_k alpha^k around alpha = 1/2: alpha = t + 1/2.
std::vector<Q> centre(const std::vector<Q>& c)
{
    std::vector<Q> r(D);
    // (t + 1/2)^k = sum_s C(k,s) t^s (1/2)^(k-s)
    for (int k = 0; k < D; ++k) {
        if (c[k].p == 0) continue;
        long long binom = 1;
        for (int s = 0; s <= k; ++s) {
            if (s > 0) binom = binom * (k - s + 1) / s;
            const i128 den = i128(1) << (k - s);
            r[s] = r[s] + c[k] * Q(i128(binom), den);
        }
    }
    return r;
}

}  // namespace

void build_poly_table(int K, PolyTab* out)
{
    std::memset(out, 0, sizeof(PolyTab));
    const int O = K + 1;
    for (int j = 0; j < O; ++j)
        for (int l = 0; l < O; ++l) {
            // A: P_l(xi - 2 alpha) over [2 alpha - 1, 1]
            std::vector<Q> a = centre(entry(j, l, -2, 0, 2, -1, 0, 1));
            // B: P_l(xi + 2 - 2 alpha) over [-1, 2 alpha - 1]
            std::vector<Q> b = centre(entry(j, l, -2, 2, 0, -1, 2, -1));
            for (int p = 0; p <= kMaxPolyDeg; ++p) {
                out->a[j][l][p] = a[p].to_double();
                out->b[j][l][p] = b[p].to_double();
            }
            for (int p = kMaxPolyDeg + 1; p < D; ++p) {
                if (a[p].p != 0 || b[p].p != 0) std::abort();   // degree bound violated
            }
        }
}

}  // namespace sl
