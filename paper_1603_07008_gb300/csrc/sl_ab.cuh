// sl_ab.cuh -- shift decomposition and construction of A(alpha), B(alpha)
// for one shift class (Sec. II-A, update rule), shared by the single-problem
// and the batched table kernels.
#pragma once

#include "sl_internal.cuh"

namespace sl {

// Shift in cells of class c: from an array, from the cell-centre velocity of
// a v-dimension, v = lo + (c + 1/2) hv, or from field samples; then a * tau / h.
// Each product and quotient is rounded once in the order written (no
// contraction), so the shift does not depend on the compiler.
__device__ __forceinline__ double shift_of(const ShiftSource& src, int c)
{
    if (src.kind == 0) return src.data[c];
    if (src.kind == 1) {
        const double v = __dadd_rn(src.lo, __dmul_rn(double(c) + 0.5, src.hv));
        return __ddiv_rn(__dmul_rn(v, src.tau), src.h);
    }
    return __ddiv_rn(__dmul_rn(src.data[c], src.tau), src.h);
}

// s = sigma + alpha, sigma = floor(s), alpha = s - sigma (alpha rounding to 1
// moves to the next integer), sigma reduced into [0, N).  The entries of A and
// B are the exact polynomials of the projection integrals, stored centred at
// alpha = 1/2 and evaluated by Horner's rule; alpha = 0 is the exact identity.
// Writes class c's record (padded to 16 bytes) in FP64 and FP32.  The degree
// is a template parameter so that the loops unroll.
template <int K>
__device__ __forceinline__ void ab_class_k(double s, uint32_t N, const PolyTab& tab, int c,
                                           int32_t* __restrict__ sigma, double* __restrict__ alpha,
                                           double* __restrict__ ab64, float* __restrict__ ab32)
{
    const double f = floor(s);
    double a = s - f;
    long long sg = (long long)f;
    if (a >= 1.0) {
        sg += 1;
        a = 0.0;
    }
    long long r = sg % (long long)N;
    if (r < 0) r += N;
    sigma[c] = int32_t(r);
    alpha[c] = a;

    constexpr int O = K + 1;
    constexpr int deg = 2 * K + 1;
    const double t = a - 0.5;
    double* m64 = ab64 + size_t(c) * ab_stride64(O);
    float* m32 = ab32 + size_t(c) * ab_stride32(O);
#pragma unroll
    for (int j = 0; j < O; ++j) {
#pragma unroll
        for (int l = 0; l < O; ++l) {
            double va, vb;
            if (a == 0.0) {
                va = (j == l) ? 1.0 : 0.0;
                vb = 0.0;
            } else {
                va = tab.a[j][l][deg];
                vb = tab.b[j][l][deg];
#pragma unroll
                for (int p = deg - 1; p >= 0; --p) {
                    va = fma(va, t, tab.a[j][l][p]);
                    vb = fma(vb, t, tab.b[j][l][p]);
                }
            }
            m64[j * O + l] = va;
            m64[O * O + j * O + l] = vb;
            m32[j * O + l] = __double2float_rn(va);
            m32[O * O + j * O + l] = __double2float_rn(vb);
        }
    }
}

__device__ __forceinline__ void ab_class(int K, double s, uint32_t N, const PolyTab& tab, int c,
                                         int32_t* __restrict__ sigma, double* __restrict__ alpha,
                                         double* __restrict__ ab64, float* __restrict__ ab32)
{
    switch (K) {
    case 0: ab_class_k<0>(s, N, tab, c, sigma, alpha, ab64, ab32); break;
    case 1: ab_class_k<1>(s, N, tab, c, sigma, alpha, ab64, ab32); break;
    case 2: ab_class_k<2>(s, N, tab, c, sigma, alpha, ab64, ab32); break;
    default: ab_class_k<3>(s, N, tab, c, sigma, alpha, ab64, ab32); break;
    }
}

}  // namespace sl
