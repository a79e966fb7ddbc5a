/*
 * sl_oracle.c -- plain, slow CPU FP64 oracle for the semi-Lagrangian
 * discontinuous Galerkin (sLdG) projection sweep of
 *   L. Einkemmer, "A mixed precision semi-Lagrangian algorithm and its
 *   performance on accelerators", HPCS 2016 (arXiv:1603.07008).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; the two
 * meet only in the seeded input descriptions (grid, initial-condition terms,
 * field samples) that both receive as plain numbers.
 *
 * Everything here is written straight from the paper's definitions, in FP64,
 * with plain loops and no blocking or fusion:
 *   - Legendre modal basis on each cell, coefficients by eq. (cj)      (Sec. II-A)
 *   - translation of the piecewise polynomial by the exact solution of
 *     eq. (advection) followed by the L2 projection back onto the
 *     piecewise polynomials                                            (Sec. II, II-A)
 *   - the resulting update c' = A c[i*] + B c[i*+1] with matrices that
 *     depend only on the fractional part of the shift                  (Sec. II-A, update rule)
 *   - mass = sum of the cell means times the cell volume               (Sec. II-A, III-A)
 *
 * Readings of the paper taken here (the paper is one-dimensional and terse):
 *   - shift in cells s = a*dt/h = sigma + alpha, sigma = floor(s),
 *     alpha = s - sigma in [0,1); if the FP64 subtraction yields 1 the
 *     shift is taken as sigma+1, alpha = 0.  Source cells are i-sigma
 *     (matrix A) and i-sigma-1 (matrix B), periodic in every dimension.
 *   - alpha == 0 is an exact copy (A = I, B = 0).
 *   - d dimensions: tensor-product Legendre basis; a sweep along one
 *     dimension applies the 1D update to every fibre of coefficients that
 *     varies only in that dimension's index.  The shift is constant along
 *     a line and may depend on one orthogonal cell coordinate.
 *
 * Array layout: cells in row-major order with dimension 0 fastest; inside a
 * cell the o^d coefficients with multi-index (j_0..j_{d-1}) at
 * J = sum_m j_m o^m (j_0 fastest).  o = k+1.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * rounding of every sum follows the order written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDIM 6
#define OR_MAXK 3
#define OR_MAXQ 64

/* Planted mistakes for the test that checks the pins (tests/): with
 * or_mutation = m > 0 one plausible error of the kind a reader could make
 * (a wrong sign, index, factor or operand order) replaces the correct
 * statement at the place marked MUTATION m, so that the test can show that
 * some pin fails for each of them.  0, the default, is the oracle itself. */
static int or_mutation = 0;
void or_set_mutation(int m) { or_mutation = m; }
int or_get_mutation(void) { return or_mutation; }

/* ------------------------------------------------------------------ */
/* Legendre polynomials and Gauss-Legendre quadrature                  */
/* ------------------------------------------------------------------ */

/* P_j(x) by the three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
double or_legendre(int j, double x)
{
    if (j == 0) return 1.0;
    double pm1 = 1.0, p = x;
    for (int n = 1; n < j; ++n) {
        double pn1 = ((2.0 * n + 1.0) * x * p - n * pm1) / (or_mutation == 1 ? (double)n : n + 1.0);   /* MUTATION 1 */
        pm1 = p;
        p = pn1;
    }
    return p;
}

/* n-point Gauss-Legendre rule on [-1,1]: nodes are the roots of P_n found by
 * Newton's method from the usual cosine guess; weights 2/((1-x^2) P_n'(x)^2).
 * Nodes are returned in increasing order.  Returns 0 on success. */
int or_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1 || n > OR_MAXQ) return -1;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 1; m < n; ++m) {
                double p2 = ((2.0 * m + 1.0) * z * p1 - m * p0) / (m + 1.0);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute the derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int m = 1; m < n; ++m) {
            double p2 = ((2.0 * m + 1.0) * z * p1 - m * p0) / (m + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        /* the guess for i runs from the largest root down */
        x[n - 1 - i] = z;
        w[n - 1 - i] = or_mutation == 2 ? 2.0 / ((1.0 - z * z) * fabs(dp))                /* MUTATION 2 */
                                        : 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Shift decomposition and the projection matrices A(alpha), B(alpha)   */
/* ------------------------------------------------------------------ */

/* s = sigma + alpha with sigma = floor(s), alpha in [0,1). */
void or_shift_split(double s, int64_t* sigma, double* alpha)
{
    double f = or_mutation == 3 ? trunc(s) : floor(s);   /* MUTATION 3 */
    double a = s - f;
    int64_t sg = (int64_t)f;
    if (a >= 1.0 && or_mutation != 19) { sg += 1; a = 0.0; }   /* MUTATION 19 */
    *sigma = sg;
    *alpha = a;
}

/* A_jl = (2j+1)/2 * int_{2a-1}^{1}  P_j(xi) P_l(xi - 2a)     dxi
 * B_jl = (2j+1)/2 * int_{-1}^{2a-1} P_j(xi) P_l(xi + 2 - 2a) dxi
 * The new polynomial on cell i is the old one translated by s cells; on the
 * part xi in [2a-1,1] of the target cell it is the polynomial of source cell
 * i-sigma at local coordinate xi-2a, on [-1,2a-1] the polynomial of cell
 * i-sigma-1 at xi+2-2a.  Projecting onto P_j (eq. (cj)) gives the two sums
 * of the update rule.  Both integrands have degree <= 2k, so (k+2)-point
 * Gauss-Legendre on each sub-interval is exact.  Row-major o x o output. */
int or_ab_matrices(int k, double alpha, double* A, double* B)
{
    if (k < 0 || k > OR_MAXK || !(alpha >= 0.0) || !(alpha < 1.0)) return -1;
    const int o = k + 1;
    if (alpha == 0.0 && or_mutation != 16) {   /* MUTATION 16 */
        for (int j = 0; j < o; ++j)
            for (int l = 0; l < o; ++l) {
                A[j * o + l] = (j == l) ? 1.0 : 0.0;
                B[j * o + l] = 0.0;
            }
        return 0;
    }
    const int nq = k + 2;
    double t[OR_MAXQ], w[OR_MAXQ];
    or_gauss_legendre(nq, t, w);
    for (int j = 0; j < o; ++j) {
        for (int l = 0; l < o; ++l) {
            double sa = 0.0, sb = 0.0;
            for (int q = 0; q < nq; ++q) {
                /* [-1,1] -> [2a-1, 1]: xi = (1-a) t + a, dxi = (1-a) dt */
                double xi = (1.0 - alpha) * t[q] + alpha;
                sa += (1.0 - alpha) * w[q] * or_legendre(j, xi) *
                      or_legendre(l, or_mutation == 4 ? xi + 2.0 * alpha : xi - 2.0 * alpha);   /* MUTATION 4 */
                /* [-1,1] -> [-1, 2a-1]: eta = a t + a - 1, deta = a dt */
                double eta = alpha * t[q] + alpha - 1.0;
                sb += alpha * w[q] * or_legendre(j, eta) *
                      or_legendre(l, or_mutation == 5 ? eta - 2.0 + 2.0 * alpha : eta + 2.0 - 2.0 * alpha);   /* MUTATION 5 */
            }
            A[j * o + l] = (or_mutation == 6 ? 1.0 : 0.5) * (2.0 * j + 1.0) * sa;   /* MUTATION 6 */
            B[j * o + l] = 0.5 * (2.0 * j + 1.0) * sb;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid helpers                                                        */
/* ------------------------------------------------------------------ */

static int check_grid(int ndim, const int64_t* n, int k)
{
    if (ndim < 1 || ndim > OR_MAXDIM) return -1;
    if (k < 0 || k > OR_MAXK) return -1;
    for (int m = 0; m < ndim; ++m)
        if (n[m] < 1) return -1;
    return 0;
}

static int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

static int64_t pmod(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

/* cell multi-index of flat cell index c (dimension 0 fastest) */
static void cell_index(int ndim, const int64_t* n, int64_t c, int64_t* idx)
{
    for (int m = 0; m < ndim; ++m) {
        idx[m] = c % n[m];
        c /= n[m];
    }
}

/* ------------------------------------------------------------------ */
/* One sweep along dimension `dim`                                     */
/* ------------------------------------------------------------------ */

/* shifts: shift_dim < 0 -> one shift for every line (shifts[0]);
 *         otherwise shifts[i] for the line whose coordinate along
 *         shift_dim is i (shift_dim != dim).  Shifts are in cells. */
int or_sweep(int ndim, const int64_t* n, int k, int dim, int shift_dim,
             const double* shifts, const double* u, double* out)
{
    if (check_grid(ndim, n, k)) return -1;
    if (dim < 0 || dim >= ndim) return -1;
    if (shift_dim >= ndim || shift_dim == dim) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim);
    int64_t cells = 1, cstride = 1;
    for (int m = 0; m < ndim; ++m) cells *= n[m];
    for (int m = 0; m < dim; ++m) cstride *= n[m];
    const int64_t nclass = shift_dim < 0 ? 1 : n[shift_dim];

    /* per shift class: sigma and the matrices */
    int64_t* sig = (int64_t*)malloc(sizeof(int64_t) * nclass);
    double* AB = (double*)malloc(sizeof(double) * 2 * o * o * nclass);
    if (!sig || !AB) { free(sig); free(AB); return -2; }
    for (int64_t c = 0; c < nclass; ++c) {
        double alpha;
        if (!isfinite(shifts[c])) { free(sig); free(AB); return -1; }
        or_shift_split(shifts[c], &sig[c], &alpha);
        or_ab_matrices(k, alpha, AB + 2 * o * o * c, AB + 2 * o * o * c + o * o);
    }

    int64_t idx[OR_MAXDIM];
    for (int64_t c = 0; c < cells; ++c) {
        cell_index(ndim, n, c, idx);
        int64_t cls = shift_dim < 0 ? 0 : idx[shift_dim];
        const double* A = AB + 2 * o * o * cls;
        const double* B = A + o * o;
        int64_t ia = pmod(or_mutation == 10 ? idx[dim] + sig[cls] : idx[dim] - sig[cls], n[dim]);   /* MUTATION 10 */
        int64_t ib = pmod(or_mutation == 9 ? ia + 1 : ia - 1, n[dim]);                               /* MUTATION 9 */
        int64_t ca = c + (ia - idx[dim]) * cstride;
        int64_t cb = c + (ib - idx[dim]) * cstride;
        for (int64_t J = 0; J < ncoef; ++J) {
            int jm = (int)((J / ostride) % o);
            int64_t Jbase = J - jm * ostride;
            double acc = 0.0;
            for (int l = 0; l < o; ++l) {
                const int e = or_mutation == 7 ? l * o + jm : jm * o + l;          /* MUTATION 7 */
                const double* Aa = or_mutation == 8 ? B : A;                       /* MUTATION 8 */
                const double* Bb = or_mutation == 8 ? A : B;
                acc += Aa[e] * u[ca * ncoef + Jbase + l * ostride];
                if (or_mutation != 11) acc += Bb[e] * u[cb * ncoef + Jbase + l * ostride];   /* MUTATION 11 */
            }
            out[c * ncoef + J] = acc;
        }
    }
    free(sig);
    free(AB);
    return 0;
}

/* Brute-force sweep for small grids: it never forms A or B.  For each target
 * cell it evaluates the translated piecewise polynomial at nq Gauss nodes on
 * each side of the single source-cell boundary inside the cell, locating the
 * source cell from the translated coordinate itself, and projects onto P_j
 * (eq. (cj)).  Same arguments and layout as or_sweep. */
int or_bruteforce_sweep(int ndim, const int64_t* n, int k, int dim, int shift_dim,
                        const double* shifts, int nq, const double* u, double* out)
{
    if (check_grid(ndim, n, k)) return -1;
    if (dim < 0 || dim >= ndim || shift_dim >= ndim || shift_dim == dim) return -1;
    if (nq < 1 || nq > OR_MAXQ) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim);
    int64_t cells = 1, cstride = 1;
    for (int m = 0; m < ndim; ++m) cells *= n[m];
    for (int m = 0; m < dim; ++m) cstride *= n[m];
    const int64_t N = n[dim];
    double t[OR_MAXQ], w[OR_MAXQ];
    or_gauss_legendre(nq, t, w);

    int64_t idx[OR_MAXDIM];
    for (int64_t c = 0; c < cells; ++c) {
        cell_index(ndim, n, c, idx);
        double s = shift_dim < 0 ? shifts[0] : shifts[idx[shift_dim]];
        /* target cell in cell units: y in [i, i+1]; its preimage under the
         * translation is [i - s, i + 1 - s].  Break point where the preimage
         * crosses an integer. */
        double y0 = (double)idx[dim] - s;
        double yb = floor(y0 + 1.0);            /* integer in (y0, y0+1] */
        double xib = 2.0 * (yb - y0) - (or_mutation == 17 ? 0.0 : 1.0);   /* local coordinate of the break; MUTATION 17 */
        if (xib > 1.0) xib = 1.0;
        if (xib < -1.0) xib = -1.0;
        for (int64_t J = 0; J < ncoef; ++J) {
            int jm = (int)((J / ostride) % o);
            int64_t Jbase = J - jm * ostride;
            double acc = 0.0;
            for (int part = 0; part < 2; ++part) {
                double a = part == 0 ? -1.0 : xib;
                double b = part == 0 ? xib : 1.0;
                double half = 0.5 * (b - a);
                if (half <= 0.0) continue;
                for (int q = 0; q < nq; ++q) {
                    double xi = half * t[q] + 0.5 * (a + b);
                    double y = y0 + 0.5 * (xi + 1.0);  /* preimage point, cell units */
                    double fy = floor(y);
                    int64_t src = pmod((int64_t)fy, N);
                    double xs = 2.0 * (y - fy) - 1.0;  /* local coordinate in the source cell */
                    int64_t cs = c + (src - idx[dim]) * cstride;
                    double val = 0.0;
                    for (int l = 0; l < o; ++l)
                        val += u[cs * ncoef + Jbase + l * ostride] * or_legendre(l, xs);
                    acc += half * w[q] * val * or_legendre(jm, xi);
                }
            }
            out[c * ncoef + J] = 0.5 * (2.0 * jm + 1.0) * acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Nodal-in-velocity x-sweep                                           */
/* ------------------------------------------------------------------ */

/* The x-sweep along `dim` with the velocity taken at the o Gauss-Legendre
 * nodes eta_q of every cell of the paired v-dimension `vdim`, instead of one
 * velocity per v-cell (reading of the multi-dimensional term v d_x f, whose
 * velocity varies inside a v-cell).  For every target cell and every fibre of
 * coefficients that varies in (j_dim, j_vdim) only:
 *   1. values at the nodes: U_q(l) = sum_jv c_{l,jv} P_jv(eta_q);
 *   2. the update rule of Sec. II-A at node q, with the shift in cells
 *      s_{j,q} = (vlo + (j + 1/2 + eta_q / 2) hv) * tau_over_h, j the v-cell;
 *   3. back to coefficients with the o-point Gauss rule (eq. (cj) along v):
 *      c'_{jx,jv} = (2 jv + 1) / 2 * sum_q w_q P_jv(eta_q) U'_q(jx).
 * Same layout as or_sweep.  Returns 0, or -1 for bad arguments. */
static double node_shift(double vlo, double hv, double tau_over_h, int64_t j, double eta)
{
    const double half = or_mutation == 20 ? 1.0 : 0.5;      /* MUTATION 20 */
    return (vlo + ((double)j + 0.5 + half * eta) * hv) * tau_over_h;
}

/* Node q's part of the new coefficients of one cell (steps 1-3 above for
 * node q), added to out: ua and ub are the o^ndim coefficients of the cells
 * i - sigma_q and i - sigma_q - 1, A and B the node's matrices. */
static void nodal_node(int o, int64_t ncoef, int64_t ostride, int64_t vstride, int q, const double* eta,
                       const double* w, const double* A, const double* B, const double* ua, const double* ub,
                       double* out)
{
    const int qe = or_mutation == 22 ? o - 1 - q : q;     /* MUTATION 22 */
    for (int64_t base = 0; base < ncoef; ++base) {
        if ((base / ostride) % o != 0 || (base / vstride) % o != 0) continue;
        double Ua[OR_MAXK + 1], Ub[OR_MAXK + 1];
        for (int l = 0; l < o; ++l) {
            Ua[l] = 0.0;
            Ub[l] = 0.0;
            for (int jv = 0; jv < o; ++jv) {
                const double p = or_legendre(jv, eta[qe]);
                Ua[l] += ua[base + l * ostride + jv * vstride] * p;
                Ub[l] += ub[base + l * ostride + jv * vstride] * p;
            }
        }
        for (int jx = 0; jx < o; ++jx) {
            double up = 0.0;
            for (int l = 0; l < o; ++l) up += A[jx * o + l] * Ua[l] + B[jx * o + l] * Ub[l];
            for (int jv = 0; jv < o; ++jv) {
                const double norm = or_mutation == 21 ? (2.0 * jv + 1.0) : 0.5 * (2.0 * jv + 1.0);   /* MUTATION 21 */
                out[base + jx * ostride + jv * vstride] += norm * w[q] * or_legendre(jv, eta[q]) * up;
            }
        }
    }
}

static int nodal_args_ok(int ndim, int k, int dim, int vdim, double vlo, double hv, double tau_over_h)
{
    if (ndim < 2 || ndim > OR_MAXDIM || k < 0 || k > OR_MAXK) return 0;
    if (dim < 0 || dim >= ndim || vdim < 0 || vdim >= ndim || vdim == dim) return 0;
    return isfinite(vlo) && isfinite(hv) && isfinite(tau_over_h) && hv > 0.0;
}

int or_sweep_nodal(int ndim, const int64_t* n, int k, int dim, int vdim, double vlo, double hv,
                   double tau_over_h, const double* u, double* out)
{
    if (check_grid(ndim, n, k)) return -1;
    if (!nodal_args_ok(ndim, k, dim, vdim, vlo, hv, tau_over_h)) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim), vstride = ipow(o, vdim);
    int64_t cells = 1, cstride = 1;
    for (int m = 0; m < ndim; ++m) cells *= n[m];
    for (int m = 0; m < dim; ++m) cstride *= n[m];
    double eta[OR_MAXK + 1], w[OR_MAXK + 1];
    or_gauss_legendre(o, eta, w);

    /* per (v-cell, node): sigma and the matrices */
    const int64_t nclass = n[vdim] * o;
    int64_t* sig = (int64_t*)malloc(sizeof(int64_t) * nclass);
    double* AB = (double*)malloc(sizeof(double) * 2 * o * o * nclass);
    if (!sig || !AB) { free(sig); free(AB); return -2; }
    for (int64_t j = 0; j < n[vdim]; ++j)
        for (int q = 0; q < o; ++q) {
            const int64_t cls = j * o + q;
            double alpha;
            or_shift_split(node_shift(vlo, hv, tau_over_h, j, eta[q]), &sig[cls], &alpha);
            or_ab_matrices(k, alpha, AB + 2 * o * o * cls, AB + 2 * o * o * cls + o * o);
        }

    int64_t idx[OR_MAXDIM];
    for (int64_t c = 0; c < cells; ++c) {
        cell_index(ndim, n, c, idx);
        for (int64_t J = 0; J < ncoef; ++J) out[c * ncoef + J] = 0.0;
        for (int q = 0; q < o; ++q) {
            const int64_t cls = idx[vdim] * o + q;
            const double* A = AB + 2 * o * o * cls;
            const double* B = A + o * o;
            const int64_t ia = pmod(idx[dim] - sig[cls], n[dim]);
            const int64_t ib = pmod(ia - 1, n[dim]);
            const int64_t ca = c + (ia - idx[dim]) * cstride;
            const int64_t cb = c + (ib - idx[dim]) * cstride;
            nodal_node(o, ncoef, ostride, vstride, q, eta, w, A, B, u + ca * ncoef, u + cb * ncoef, out + c * ncoef);
        }
    }
    free(sig);
    free(AB);
    return 0;
}

/* The integer parts sigma_q of the o node shifts of v-cell j, as
 * or_sweep_nodal forms them (its step 2). */
int or_node_sigma(int k, double vlo, double hv, double tau_over_h, int64_t j, int64_t* sig)
{
    if (k < 0 || k > OR_MAXK || !isfinite(vlo) || !isfinite(hv) || !isfinite(tau_over_h) || !(hv > 0.0))
        return -1;
    const int o = k + 1;
    double eta[OR_MAXK + 1], w[OR_MAXK + 1], alpha;
    or_gauss_legendre(o, eta, w);
    for (int q = 0; q < o; ++q) or_shift_split(node_shift(vlo, hv, tau_over_h, j, eta[q]), &sig[q], &alpha);
    return 0;
}

/* The new coefficients of one cell of v-cell j in the nodal x-sweep along
 * dim: ua[q] and ub[q] point to the o^ndim coefficients of its source cells
 * i - sigma_q and i - sigma_q - 1 (sigma_q from or_node_sigma).  The
 * arithmetic of or_sweep_nodal, so the result is the same bits; it lets the
 * dependency cones of sampled cells of a large grid (sample_after) include
 * nodal sweeps. */
int or_apply_cell_nodal(int ndim, int k, int dim, int vdim, double vlo, double hv, double tau_over_h, int64_t j,
                        const double* const* ua, const double* const* ub, double* out)
{
    if (!nodal_args_ok(ndim, k, dim, vdim, vlo, hv, tau_over_h)) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim), vstride = ipow(o, vdim);
    double eta[OR_MAXK + 1], w[OR_MAXK + 1];
    or_gauss_legendre(o, eta, w);
    for (int64_t J = 0; J < ncoef; ++J) out[J] = 0.0;
    for (int q = 0; q < o; ++q) {
        int64_t sg;
        double alpha, A[(OR_MAXK + 1) * (OR_MAXK + 1)], B[(OR_MAXK + 1) * (OR_MAXK + 1)];
        or_shift_split(node_shift(vlo, hv, tau_over_h, j, eta[q]), &sg, &alpha);
        or_ab_matrices(k, alpha, A, B);
        nodal_node(o, ncoef, ostride, vstride, q, eta, w, A, B, ua[q], ub[q], out);
    }
    return 0;
}

/* The same sweep without A or B: at each node the translated piecewise
 * polynomial in x (values U_q of step 1) is projected onto P_jx by an
 * nq-point Gauss rule on each side of the source-cell boundary, as in
 * or_bruteforce_sweep; steps 1 and 3 as in or_sweep_nodal. */
int or_bruteforce_nodal(int ndim, const int64_t* n, int k, int dim, int vdim, double vlo, double hv,
                        double tau_over_h, int nq, const double* u, double* out)
{
    if (check_grid(ndim, n, k)) return -1;
    if (ndim < 2 || dim < 0 || dim >= ndim || vdim < 0 || vdim >= ndim || vdim == dim) return -1;
    if (nq < 1 || nq > OR_MAXQ || !(hv > 0.0)) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim), vstride = ipow(o, vdim);
    int64_t cells = 1, cstride = 1;
    for (int m = 0; m < ndim; ++m) cells *= n[m];
    for (int m = 0; m < dim; ++m) cstride *= n[m];
    const int64_t N = n[dim];
    double eta[OR_MAXK + 1], w[OR_MAXK + 1], t[OR_MAXQ], tw[OR_MAXQ];
    or_gauss_legendre(o, eta, w);
    or_gauss_legendre(nq, t, tw);

    int64_t idx[OR_MAXDIM];
    for (int64_t c = 0; c < cells; ++c) {
        cell_index(ndim, n, c, idx);
        for (int64_t J = 0; J < ncoef; ++J) out[c * ncoef + J] = 0.0;
        for (int q = 0; q < o; ++q) {
            const double s = (vlo + ((double)idx[vdim] + 0.5 + 0.5 * eta[q]) * hv) * tau_over_h;
            const double y0 = (double)idx[dim] - s;
            const double yb = floor(y0 + 1.0);
            double xib = 2.0 * (yb - y0) - 1.0;
            if (xib > 1.0) xib = 1.0;
            if (xib < -1.0) xib = -1.0;
            for (int64_t base = 0; base < ncoef; ++base) {
                if ((base / ostride) % o != 0 || (base / vstride) % o != 0) continue;
                for (int jx = 0; jx < o; ++jx) {
                    double acc = 0.0;
                    for (int part = 0; part < 2; ++part) {
                        const double a = part == 0 ? -1.0 : xib;
                        const double b = part == 0 ? xib : 1.0;
                        const double half = 0.5 * (b - a);
                        if (half <= 0.0) continue;
                        for (int r = 0; r < nq; ++r) {
                            const double xi = half * t[r] + 0.5 * (a + b);
                            const double y = y0 + 0.5 * (xi + 1.0);
                            const double fy = floor(y);
                            const int64_t src = pmod((int64_t)fy, N);
                            const double xs = 2.0 * (y - fy) - 1.0;
                            const int64_t cs = c + (src - idx[dim]) * cstride;
                            double val = 0.0;
                            for (int l = 0; l < o; ++l)
                                for (int jv = 0; jv < o; ++jv)
                                    val += u[cs * ncoef + base + l * ostride + jv * vstride] *
                                           or_legendre(l, xs) * or_legendre(jv, eta[q]);
                            acc += half * tw[r] * val * or_legendre(jx, xi);
                        }
                    }
                    const double up = 0.5 * (2.0 * jx + 1.0) * acc;
                    for (int jv = 0; jv < o; ++jv)
                        out[c * ncoef + base + jx * ostride + jv * vstride] +=
                            0.5 * (2.0 * jv + 1.0) * w[q] * or_legendre(jv, eta[q]) * up;
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Initial projection, eq. (cj)                                        */
/* ------------------------------------------------------------------ */

/* One factor of a separable initial condition:
 *   g(x) = exp(-gamma (x - mu)^2) * cos(kappa x + phi)
 * params = {gamma, mu, kappa, phi}. */
static double factor_eval(const double* prm, double x)
{
    double d = x - prm[1];
    return exp(-prm[0] * d * d) * cos(prm[2] * x + prm[3]);
}

/* 1D projection of one factor onto cell i of a dimension with lower end lo
 * and width h:  c_j = (2j+1)/2 * sum_q w_q g(x_i + h t_q / 2) P_j(t_q). */
static void factor_project(const double* prm, double lo, double h, int64_t i, int k,
                           int nq, const double* t, const double* w, double* cj)
{
    double xc = lo + ((double)i + 0.5) * h;
    for (int j = 0; j <= k; ++j) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q)
            acc += w[q] * factor_eval(prm, xc + (or_mutation == 14 ? h : 0.5 * h) * t[q]) *   /* MUTATION 14 */
                   or_legendre(j, t[q]);
        cj[j] = (or_mutation == 13 ? 1.0 : 0.5) * (2.0 * j + 1.0) * acc;   /* MUTATION 13 */
    }
}

/* u0(x) = sum_t weight[t] * prod_m g_{t,m}(x_m); params[(t*ndim + m)*4 + 0..3].
 * The projection of a product onto the tensor-product basis with a
 * tensor-product Gauss rule factorises into 1D projections, which is what is
 * computed here.  Writes the coefficients of the cells listed in `cells`
 * (flat indices; ncells of them) into out[ncells][o^d]; cells == NULL means
 * all cells in order. */
int or_project(int ndim, const int64_t* n, const double* lo, const double* hi, int k,
               int nq, int nterms, const double* weight, const double* params,
               const int64_t* cells, int64_t ncells, double* out)
{
    if (check_grid(ndim, n, k)) return -1;
    if (nq < 1 || nq > OR_MAXQ || nterms < 0) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    int64_t total = 1;
    for (int m = 0; m < ndim; ++m) total *= n[m];
    if (cells == NULL) ncells = total;
    double t[OR_MAXQ], w[OR_MAXQ];
    or_gauss_legendre(nq, t, w);
    double h[OR_MAXDIM];
    for (int m = 0; m < ndim; ++m) h[m] = (hi[m] - lo[m]) / (double)n[m];

    int64_t idx[OR_MAXDIM];
    int jidx[OR_MAXDIM];
    double p[OR_MAXDIM][OR_MAXK + 1];
    for (int64_t s = 0; s < ncells; ++s) {
        int64_t c = cells ? cells[s] : s;
        if (c < 0 || c >= total) return -1;
        cell_index(ndim, n, c, idx);
        double* dst = out + s * ncoef;
        for (int64_t J = 0; J < ncoef; ++J) dst[J] = 0.0;
        for (int tt = 0; tt < nterms; ++tt) {
            for (int m = 0; m < ndim; ++m)
                factor_project(params + (tt * ndim + m) * 4, lo[m], h[m], idx[m], k, nq, t, w, p[m]);
            for (int64_t J = 0; J < ncoef; ++J) {
                int64_t r = J;
                for (int m = 0; m < ndim; ++m) { jidx[or_mutation == 15 ? ndim - 1 - m : m] = (int)(r % o); r /= o; }   /* MUTATION 15 */
                double prod = weight[tt];
                for (int m = 0; m < ndim; ++m) prod *= p[m][jidx[m]];
                dst[J] += prod;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Mass                                                                */
/* ------------------------------------------------------------------ */

/* M = (prod_m h_m) * sum_i c_{i;0..0}: c0 is the cell mean (Sec. II-A), so the
 * mass of cell i is its volume times c0. */
double or_mass(int ndim, const int64_t* n, const double* lo, const double* hi, int k,
               const double* u)
{
    if (check_grid(ndim, n, k)) return NAN;
    const int64_t ncoef = ipow(k + 1, ndim);
    int64_t cells = 1;
    double vol = 1.0;
    for (int m = 0; m < ndim; ++m) {
        cells *= n[m];
        vol *= (hi[m] - lo[m]) / (double)n[m];
    }
    double s = 0.0;
    for (int64_t c = 0; c < cells; ++c) s += u[c * ncoef];
    return or_mutation == 12 ? s : vol * s;   /* MUTATION 12 */
}

/* ------------------------------------------------------------------ */
/* Per-cell pieces for evaluating sampled cells of large grids          */
/* ------------------------------------------------------------------ */

/* New coefficients of one cell from its two source cells along `dim`:
 * out_J = sum_l A[j_dim][l] ua[J(l)] + B[j_dim][l] ub[J(l)]. */
int or_apply_cell(int ndim, int k, int dim, const double* A, const double* B,
                  const double* ua, const double* ub, double* out)
{
    if (ndim < 1 || ndim > OR_MAXDIM || k < 0 || k > OR_MAXK || dim < 0 || dim >= ndim) return -1;
    const int o = k + 1;
    const int64_t ncoef = ipow(o, ndim);
    const int64_t ostride = ipow(o, dim);
    for (int64_t J = 0; J < ncoef; ++J) {
        int jm = (int)((J / ostride) % o);
        int64_t Jbase = J - jm * ostride;
        double acc = 0.0;
        for (int l = 0; l < o; ++l) {
            acc += A[jm * o + l] * (or_mutation == 18 ? ub : ua)[Jbase + l * ostride];   /* MUTATION 18 */
            acc += B[jm * o + l] * (or_mutation == 18 ? ua : ub)[Jbase + l * ostride];
        }
        out[J] = acc;
    }
    return 0;
}
