// sl_sweep.cuh -- the sLdG projection-sweep kernels for sm_103a.
//
// Every target cell i of a line gets, for every fibre of coefficients that
// varies only in the sweep dimension's index j,
//     c'_j = sum_l A_jl(alpha) c_{i-sigma, l} + B_jl(alpha) c_{i-sigma-1, l}
// (Sec. II-A, update rule).  The work is one load and one store per degree of
// freedom against 4o-1 flops (Sec. II-A), so the kernels are HBM-bound on
// CUDA cores; no tensor cores are involved.
//
// Launch shapes:
//   * unit stride (sweep along dimension 0): one thread per target cell and
//     group of FT fibres; consecutive threads on consecutive cells of a line,
//     so every plane access of a warp is one coalesced segment.  The second
//     source cell (i-sigma-1) is the first source cell of the neighbouring
//     lane, so its load is served by L1.
//   * strided (sweep along dimension m > 0): one thread per line (consecutive
//     threads on consecutive inner indices, again coalesced), walking along
//     the sweep dimension.  The source cell i-sigma of one target is the
//     source cell i-sigma-1 of the next, so every source value is read once.
//     Either the walk keeps U cells of loads in flight in registers
//     (k_sweep_strided), or it streams its rows P rows ahead through a
//     per-thread cp.async ring in shared memory (k_sweep_strided_async).
//
// A thread's fibre group either contains the fibre of the cell mean (group 0)
// or not; the two cases are separate instantiations of the kernel body, so
// the mean's special handling costs nothing elsewhere.  The all-FP32 store
// (M_F32ALL) has no FP64 mean: every group is computed as an FP32 group.  The last group of a
// cell may be partial; its missing fibres repeat the last valid one, whose
// values are then computed and stored twice by the same thread.
//
// Precision (split store): the cell mean c_{0..0} lives in an FP64 plane.
// Its row is computed in the form
//     c'_0 = a_0 + alpha (b_0 - a_0) + sum_{l>=1} A_0l (a_l - b_l),
// which uses the exact identities A_00 + B_00 = 1 and B_0l = -A_0l (l >= 1)
// of the projection, so the sum over a line telescopes and mass is conserved
// to FP64 rounding (Sec. II-A, III-A).  The donor part is FP64; in the
// low-precision stores the sum is formed as FP64 differences of per-cell FP32
// sums (see combine), which still telescope exactly.  The other rows of the
// mean's fibre use B_j0 = -A_j0 for their l = 0 term; everything else is
// computed in the arithmetic type of the mode (FP64, or FP32 for the mixed
// modes).
#pragma once

#include "sl_internal.cuh"

namespace sl {

template <int MODE>
struct St;
template <>
struct St<M_FP64> {
    using T = double;
    using R = double;
    static constexpr bool scaled = false;
    static constexpr bool mean64 = true;   // the cell mean has its own FP64 plane
};
template <>
struct St<M_F32> {
    using T = float;
    using R = float;
    static constexpr bool scaled = false;
    static constexpr bool mean64 = true;
};
// every coefficient, the mean included, in FP32 planes with FP32 arithmetic
template <>
struct St<M_F32ALL> {
    using T = float;
    using R = float;
    static constexpr bool scaled = false;
    static constexpr bool mean64 = false;
};
// the general split stores, whose planes the coefficient map places (only
// the codec instantiates this; their sweeps are in sl_sweep_split.cu)
template <>
struct St<M_SPLIT2> {
    using T = float;
    using R = float;
    static constexpr bool scaled = false;
    static constexpr bool mean64 = true;
};
template <>
struct St<M_BF16> {
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool scaled = true;
    static constexpr bool mean64 = true;
};
template <>
struct St<M_FP16> {
    using T = __half;
    using R = float;
    static constexpr bool scaled = true;
    static constexpr bool mean64 = true;
};

__device__ __forceinline__ double ld_raw(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_raw(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_raw(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_raw(const __half* p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ void st_raw(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_raw(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_raw(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_raw(__half* p, float v) { *p = __float2half_rn(v); }

// Per-cell power-of-two scale of the scaled modes: with mx = f 2^e,
// f in [0.5, 1), s = 2^e, so every stored value v/s lies in (-1, 1) and the
// largest in magnitude in [0.5, 1).  Zero, subnormal and non-finite maxima get
// s = 1.  Multiplying by s or 1/s is exact.
__device__ __forceinline__ void pow2_scale(float mx, float& s, float& inv)
{
    uint32_t E = (__float_as_uint(mx) >> 23) & 0xffu;
    if (E == 0u || E == 255u) {
        s = 1.0f;
        inv = 1.0f;
        return;
    }
    if (E > 252u) E = 252u;
    s = __uint_as_float((E + 1u) << 23);
    inv = __uint_as_float((253u - E) << 23);
}

// Conversions between IEEE 754 binary32 and binary64 done on the integer
// pipe, without branches.  GB300's FP64 pipe (which also executes the F2F
// conversions) runs at a small fraction of the FP32 rate, and the mean row of
// the low-precision stores would otherwise spend three of its seven FP64-pipe
// instructions on conversions.  For every input outside the binary32
// subnormal range both return exactly what the conversion instructions
// return (float to double is exact; double to float rounds to nearest, ties
// to even, overflowing to infinity; zeros, infinities and NaN keep their
// kind and sign).  Subnormal binary32 values (inputs of f2d_fast, results of
// d2f_fast, all below 1.2e-38 in magnitude) are not reproduced: f2d_fast maps
// them to values below 2^-126 and d2f_fast flushes such results to a signed
// zero.  Both are fixed functions of their input, which is all the mean row
// needs for its sums to telescope.
//
// binary32 -> binary64: sign kept, exponent rebiased by 1023 - 127 = 896,
// the 23 fraction bits placed at the top of the 52-bit fraction.
__device__ __forceinline__ double f2d_fast(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t a = u & 0x7fffffffu;
    uint32_t hi = (a >> 3) + 0x38000000u;                       // exponent + 896, fraction >> 3
    hi = a >= 0x7f800000u ? (0x7ff00000u | ((a >> 3) & 0xfffffu)) : hi;   // inf, NaN
    hi = a == 0u ? 0u : hi;
    return __hiloint2double(int(hi | (u & 0x80000000u)), int(u << 29));
}

// binary64 -> binary32 of (neg ? -x : x), rounded to nearest even: the top
// 23 of the 52 fraction bits are kept and the other 29 decide the rounding;
// a carry out of the fraction moves into the exponent, which is the correct
// result, including the overflow of the largest values to infinity.
__device__ __forceinline__ float d2f_fast(double x, bool neg)
{
    const uint32_t hi = uint32_t(__double2hiint(x)) ^ (neg ? 0x80000000u : 0u);
    const uint32_t lo = uint32_t(__double2loint(x));
    const uint32_t s = hi & 0x80000000u;
    const uint32_t a = hi & 0x7fffffffu;                        // |x|, high word
    const uint32_t m = ((a & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t r = lo & 0x1fffffffu;
    const uint32_t up = (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
    uint32_t f = (((a >> 20) - 896u) << 23 | m) + up;           // normal range
    f = a >= 0x47f00000u ? 0x7f800000u : f;                     // |x| >= 2^128: infinity
    f = a >= 0x7ff00000u && (((a & 0xfffffu) | lo) != 0u) ? (0x7fc00000u | m) : f;   // NaN
    f = a < 0x38100000u ? 0u : f;                               // |x| < 2^-126: zero
    return __uint_as_float(f | s);
}

// The same two conversions with a branch around the normal-range case
// (values of the mean row nearly always are), the other cases handled by the
// branch-free forms, so the results are the same bits.
__device__ __forceinline__ double f2d_branch(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const uint32_t hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
        return __hiloint2double(int(hi), int(u << 29));
    }
    return f2d_fast(x);
}
__device__ __forceinline__ float d2f_branch(double x, bool neg)
{
    const uint32_t hi = uint32_t(__double2hiint(x)) ^ (neg ? 0x80000000u : 0u);
    const uint32_t lo = uint32_t(__double2loint(x));
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u < 254u) {
        const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t r = lo & 0x1fffffffu;
        const uint32_t f = ((hi & 0x80000000u) | ((e - 896u) << 23) | m) +
                           ((r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u);
        return __uint_as_float(f);
    }
    return d2f_fast(x, neg);
}

// f2d_fast(a) - f2d_fast(b) for binary32 a, b.  When both are normal and
// their exponents differ by at most 28, the difference of the two 24-bit
// significands aligned to the smaller exponent has fewer than 53 bits, so it
// is exact in binary64 (the FP64 subtraction would return it unrounded) and is
// assembled here on the integer pipe; otherwise the FP64 subtraction forms it.
// Either way the bits are those of the FP64 subtraction.
__device__ __forceinline__ double sub_widened(float a, float b)
{
    const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
    const uint32_t ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu;
    const uint32_t lo = min(ea, eb);
    if (ea - 1u >= 254u || eb - 1u >= 254u || max(ea, eb) - lo > 28u) return f2d_fast(a) - f2d_fast(b);
    const int64_t ma = int64_t((ua & 0x7fffffu) | 0x800000u) << (ea - lo);
    const int64_t mb = int64_t((ub & 0x7fffffu) | 0x800000u) << (eb - lo);
    const int64_t r = ((ua >> 31) ? -ma : ma) - ((ub >> 31) ? -mb : mb);   // times 2^(lo - 150)
    if (r == 0) return 0.0;
    const uint64_t m = uint64_t(r < 0 ? -r : r);   // below 2^53
    const int lz = __clzll(int64_t(m));            // at least 11
    const uint64_t frac = (m << (lz - 11)) & 0xfffffffffffffull;
    const uint64_t bexp = uint64_t(int(lo) - 150 + (63 - lz) + 1023);
    return __longlong_as_double(int64_t((r < 0 ? 0x8000000000000000ull : 0ull) | (bexp << 52) | frac));
}

// New mean of a cell in the low-precision stores (conservation form, see
// combine) from the source means ma (cell i - sigma), mb (i - sigma - 1) and
// their per-cell FP32 sums ga = G(a), gb = G(b); dm = fl32(ma - mb) for the
// l = 0 term of the other rows: three FP64-pipe instructions when the
// difference of the widened sums is formed on the integer pipe (sub_widened),
// four with the FP64 subtraction.
// Forms of the mean row, picked per kernel by measurement; all give the same
// bits.  CV_FLAT: branch-free conversions, the difference of the widened sums
// on the integer pipe (sub_widened); CV_BRANCH: the branching conversions,
// sub_widened; CV_FP64SUB: branch-free conversions, the difference by the
// FP64 subtraction (for kernels whose integer pipe is the busier one).
enum : int { CV_FLAT = 0, CV_BRANCH = 1, CV_FP64SUB = 2 };

template <int CV = CV_FLAT>
__device__ __forceinline__ double mean_row_lp(double alpha, double ma, double mb, float ga, float gb, float& dm)
{
    const double t = mb - ma;
    if constexpr (CV == CV_BRANCH) {
        dm = d2f_branch(t, true);
        return fma(alpha, t, ma) + sub_widened(ga, gb);
    } else if constexpr (CV == CV_FP64SUB) {
        dm = d2f_fast(t, true);
        return fma(alpha, t, ma) + (f2d_fast(ga) - f2d_fast(gb));
    } else {
        dm = d2f_fast(t, true);
        return fma(alpha, t, ma) + sub_widened(ga, gb);
    }
}

template <int K, int MODE, int FT>
struct CellVals {
    typename St<MODE>::R v[FT][K + 1];   // v[0][0] of the mean's group is unused: the mean is in m
    double m;
};

// Per-thread copy of the matrices of one shift class.
template <int K, int MODE>
struct Mats {
    using R = typename St<MODE>::R;
    static constexpr int O = K + 1;
    R a[O][O], b[O][O];
    double a0[O];   // row 0 of A in FP64 (mean row)
    double aj0[O];  // column 0 of A in FP64 (l = 0 term of the mean's fibre)
    double alpha;

    template <bool MEAN>
    __device__ __forceinline__ void load(const ShiftTable& t, uint32_t cls)
    {
        // one class record, read with 16-byte vector loads
        if constexpr (sizeof(R) == 8) {
            constexpr int S = ab_stride64(O);
            const double2* p = reinterpret_cast<const double2*>(t.ab64 + size_t(cls) * S);
            double v[S];
#pragma unroll
            for (int q = 0; q < S / 2; ++q) {
                const double2 x = __ldg(p + q);
                v[2 * q] = x.x;
                v[2 * q + 1] = x.y;
            }
#pragma unroll
            for (int j = 0; j < O; ++j)
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    a[j][l] = v[j * O + l];
                    b[j][l] = v[O * O + j * O + l];
                }
        } else {
            constexpr int S = ab_stride32(O);
            const float4* p = reinterpret_cast<const float4*>(t.ab32 + size_t(cls) * S);
            float v[S];
#pragma unroll
            for (int q = 0; q < S / 4; ++q) {
                const float4 x = __ldg(p + q);
                v[4 * q] = x.x;
                v[4 * q + 1] = x.y;
                v[4 * q + 2] = x.z;
                v[4 * q + 3] = x.w;
            }
#pragma unroll
            for (int j = 0; j < O; ++j)
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    a[j][l] = v[j * O + l];
                    b[j][l] = v[O * O + j * O + l];
                }
        }
        if constexpr (MEAN) {
            const double* m64 = t.ab64 + size_t(cls) * ab_stride64(O);
#pragma unroll
            for (int l = 0; l < O; ++l) {
                a0[l] = __ldg(m64 + l);
                aj0[l] = __ldg(m64 + l * O);
            }
            alpha = __ldg(t.alpha + cls);
        }
    }
};

// New values of one target cell from its source cells a (= i - sigma) and
// b (= i - sigma - 1).  With MEAN, fibre 0 of the group is the mean's fibre.
// CV: the conversion form of the mean row (see mean_row_lp).
template <int K, int MODE, int FT, bool MEAN, int CV = CV_FLAT>
__device__ __forceinline__ void combine(const Mats<K, MODE>& M, const CellVals<K, MODE, FT>& a,
                                        const CellVals<K, MODE, FT>& b,
                                        CellVals<K, MODE, FT>& out)
{
    using R = typename St<MODE>::R;
    constexpr int O = K + 1;
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        if (MEAN && u == 0) {
            if constexpr (sizeof(R) == 8) {
                double d = a.m + M.alpha * (b.m - a.m);
#pragma unroll
                for (int l = 1; l < O; ++l) d += M.a0[l] * (a.v[0][l] - b.v[0][l]);
                out.m = d;
                const double dm = a.m - b.m;
#pragma unroll
                for (int j = 1; j < O; ++j) {
                    R acc = R(M.aj0[j] * dm);
#pragma unroll
                    for (int l = 1; l < O; ++l) {
                        acc = fma(M.a[j][l], a.v[0][l], acc);
                        acc = fma(M.b[j][l], b.v[0][l], acc);
                    }
                    out.v[0][j] = acc;
                }
            } else {
                // Low-precision stores: the higher coefficients enter the mean
                // row through G(c) = sum_{l>=1} fl32(A_0l c_l), a function of
                // one cell (the matrices are fixed along a line), so the FP64
                // differences G(a) - G(b) telescope exactly over the line and
                // the mass stays conserved to FP64 rounding; only the donor
                // part a_0 + alpha (b_0 - a_0) and the differences use the
                // (slow) FP64 pipe.  The l = 0 term of the other rows uses
                // a_0 - b_0 rounded once to FP32.
                float ga = 0.0f, gb = 0.0f;
#pragma unroll
                for (int l = 1; l < O; ++l) {
                    ga = fmaf(M.a[0][l], a.v[0][l], ga);
                    gb = fmaf(M.a[0][l], b.v[0][l], gb);
                }
                float dm;
                out.m = mean_row_lp<CV>(M.alpha, a.m, b.m, ga, gb, dm);
#pragma unroll
                for (int j = 1; j < O; ++j) {
                    R acc = M.a[j][0] * dm;
#pragma unroll
                    for (int l = 1; l < O; ++l) {
                        acc = fma(M.a[j][l], a.v[0][l], acc);
                        acc = fma(M.b[j][l], b.v[0][l], acc);
                    }
                    out.v[0][j] = acc;
                }
            }
            out.v[0][0] = 0;
        } else {
#pragma unroll
            for (int j = 0; j < O; ++j) {
                R acc = R(0);
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    acc = fma(M.a[j][l], a.v[u][l], acc);
                    acc = fma(M.b[j][l], b.v[u][l], acc);
                }
                out.v[u][j] = acc;
            }
        }
    }
}

// Base coefficient index of fibre f along a sweep whose fibre stride is
// ostride = o^dim: the fibre holds J = jb + l * ostride, l = 0..k.
__device__ __forceinline__ int fibre_base(int f, int O, int ostride)
{
    return (f / ostride) * (O * ostride) + (f % ostride);
}

// Fibre bases of a group, the missing fibres of a partial last group
// repeating its last valid fibre.
template <int FT>
__device__ __forceinline__ void group_bases(int fbase, int nfib, int O, int ostride, int (&jb)[FT])
{
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        int f = fbase + u;
        if (f >= nfib) f = nfib - 1;
        jb[u] = fibre_base(f, O, ostride);
    }
}

// Per-thread pointers to the FT*(k+1) values of a group, offset by a base
// cell; a cell at `off` cells from the base is p[u][l][off].
template <int K, int MODE, int FT, bool MEAN>
struct GroupPtrs {
    using T = typename St<MODE>::T;
    static constexpr int O = K + 1;
    const T* s[FT][O];
    T* d[FT][O];
    const double* sm;
    double* dm;

    __device__ __forceinline__ void init(const Planes& src, const Planes& dst, int64_t pstride,
                                         const int (&jb)[FT], int ostride, uint32_t base)
    {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0) {
                    sm = src.mean + base;
                    dm = dst.mean + base;
                    s[0][0] = nullptr;
                    d[0][0] = nullptr;
                } else {
                    const int J = jb[u] + l * ostride;
                    s[u][l] = plane_ptr<T>(src.hi, pstride, J) + base;
                    d[u][l] = plane_ptr_w<T>(dst.hi, pstride, J) + base;
                }
            }
    }

    __device__ __forceinline__ void load(uint32_t off, CellVals<K, MODE, FT>& cv) const
    {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0) {
                    cv.m = __ldg(sm + off);
                    cv.v[0][0] = 0;
                } else {
                    cv.v[u][l] = ld_raw(s[u][l] + off);
                }
            }
    }

    __device__ __forceinline__ void store(uint32_t off, const CellVals<K, MODE, FT>& cv) const
    {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0)
                    dm[off] = cv.m;
                else
                    st_raw(d[u][l] + off, cv.v[u][l]);
            }
    }
};

// Addresses formed per access (for the unit-stride kernel, whose threads
// touch every value only two or three times, and for the scaled stores, whose
// threads hold every fibre of a cell, too many values for a pointer table).
// The scaled modes apply the cell's scale on load and the new scale (the
// cell-wide maximum) on store.
template <int K, int MODE, int FT, bool MEAN>
__device__ __forceinline__ void load_cell(const Planes& p, int64_t pstride, uint32_t c,
                                          const int (&jb)[FT], int ostride,
                                          CellVals<K, MODE, FT>& cv)
{
    using T = typename St<MODE>::T;
    constexpr int O = K + 1;
    float s = 1.0f;
    if constexpr (St<MODE>::scaled) s = __ldg(p.scale + c);
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if (MEAN && u == 0 && l == 0) {
                cv.m = __ldg(p.mean + c);
                cv.v[0][0] = 0;
            } else {
                const int J = jb[u] + l * ostride;
                auto v = ld_raw(plane_ptr<T>(p.hi, pstride, J) + c);
                if constexpr (St<MODE>::scaled) v *= s;
                cv.v[u][l] = v;
            }
        }
}

template <int K, int MODE, int FT, bool MEAN>
__device__ __forceinline__ void store_cell(const Planes& p, int64_t pstride, uint32_t c,
                                           const int (&jb)[FT], int ostride,
                                           const CellVals<K, MODE, FT>& cv)
{
    using T = typename St<MODE>::T;
    using R = typename St<MODE>::R;
    constexpr int O = K + 1;
    R inv = R(1);
    if constexpr (St<MODE>::scaled) {
        float mx = 0.0f;
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) mx = fmaxf(mx, fabsf(cv.v[u][l]));
        float s;
        pow2_scale(mx, s, inv);
        p.scale[c] = s;
    }
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if (MEAN && u == 0 && l == 0) {
                p.mean[c] = cv.m;
            } else {
                const int J = jb[u] + l * ostride;
                R v = cv.v[u][l];
                if constexpr (St<MODE>::scaled) v *= inv;
                st_raw(plane_ptr_w<T>(p.hi, pstride, J) + c, v);
            }
        }
}

__device__ __forceinline__ uint32_t shift_class(const SweepArgs& a, uint32_t inner_idx,
                                                uint32_t outer_idx)
{
    if (a.cls_src == 0) return 0;
    const uint32_t x = a.cls_src == 1 ? inner_idx : outer_idx;
    return a.fdClsMod.mod(a.fdCls.div(x));
}

// ---------------------------------------------------------------- unit stride

template <int K, int MODE, int FT, bool MEAN, int CV = CV_FLAT>
__device__ __forceinline__ void unit_body(const SweepArgs& a, uint32_t c, uint32_t ca, uint32_t cb,
                                          uint32_t cls, int fbase)
{
    constexpr int O = K + 1;
    int jb[FT];
    if constexpr (St<MODE>::scaled) {
#pragma unroll
        for (int u = 0; u < FT; ++u) jb[u] = u * O;   // fibre stride 1 along dimension 0
    } else {
        group_bases<FT>(fbase, a.nfib, O, 1, jb);
    }
    Mats<K, MODE> M;
    M.template load<MEAN>(a.tab, cls);
    CellVals<K, MODE, FT> va, vb, out;
    load_cell<K, MODE, FT, MEAN>(a.src, a.pstride, ca, jb, 1, va);
    load_cell<K, MODE, FT, MEAN>(a.src, a.pstride, cb, jb, 1, vb);
    combine<K, MODE, FT, MEAN, CV>(M, va, vb, out);
    store_cell<K, MODE, FT, MEAN>(a.dst, a.pstride, c, jb, 1, out);
}

// Target cell c of a sweep along dimension 0, fibres fbase .. fbase+FT-1.
template <int K, int MODE, int FT, int CV = CV_FLAT>
__device__ __forceinline__ void unit_cell(const SweepArgs& a, uint32_t c, int fbase)
{
    const uint32_t line = a.fdN.div(c);
    const uint32_t i = c - line * a.N;
    const uint32_t cls = shift_class(a, 0, line);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    int32_t ia = int32_t(i) - sig;
    ia += ia < 0 ? int32_t(a.N) : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? int32_t(a.N) : 0;
    const uint32_t ca = c - i + uint32_t(ia);
    const uint32_t cb = c - i + uint32_t(ib);
    if (St<MODE>::scaled || (St<MODE>::mean64 && fbase == 0))
        unit_body<K, MODE, FT, true, CV>(a, c, ca, cb, cls, fbase);
    else
        unit_body<K, MODE, FT, false, CV>(a, c, ca, cb, cls, fbase);
}

// Grid of the sweeps along dimension 0 over `tiles` blocks of cells and nfg
// fibre groups.  Blocks are dispatched in the order of their linear index
// (x fastest).  With gfast (the kernels' GF) the fibre group is x and the
// tile y (the kernels loop over tiles y, y + gridDim.y, ...), so that the
// blocks of the mean's group, which load the FP64 pipe, run beside the other
// groups' instead of all of them first: chosen where the mean's group alone
// would need more than half the FP64 pipe at the memory's rate (unit_gfast).
// Otherwise the tile is x and the group y, so that the blocks in flight read
// few planes.
inline dim3 unit_grid(uint32_t tiles, int nfg, int gfast)
{
    if (tiles < 1) tiles = 1;
    if (gfast) return dim3(uint32_t(nfg), tiles < 65535u ? tiles : 65535u);
    return dim3(tiles, uint32_t(nfg));
}
// In the mixed FP32 store the mean's group takes three FP64-pipe instructions
// per cell and moves 2 (8 + elem (ft o - 1)) bytes per cell: more than half of
// GB300's FP64 issue rate (2 per clock per SM) at the copy bandwidth below 64
// bytes.  (In the FP64 store every group loads the FP64 pipe alike.)  Only
// for a few groups (the 2D store: the mean's group is a third or a half of
// the launch): with the 27 one-fibre groups of the 4D store at k = 2 the
// blocks in flight then read all 81 planes at once, and dimension 0 measured
// 5% slower than group by group.
inline int unit_gfast(int nfg, int ft, int O, int elem)
{
    return nfg > 1 && nfg <= 4 && 2 * (8 + elem * (ft * O - 1)) < 64 ? 1 : 0;
}

// Sweep along dimension 0: one thread per target cell and fibre group (GF:
// see unit_grid).
template <int K, int MODE, int FT, bool GF>
__global__ void __launch_bounds__(256) k_sweep_unit(const SweepArgs a)
{
    if constexpr (GF) {
        const int fbase = int(blockIdx.x) * FT;
        for (uint32_t t = blockIdx.y; t * blockDim.x < a.cells; t += gridDim.y) {
            const uint32_t c = t * blockDim.x + threadIdx.x;
            if (c >= a.cells) break;
            unit_cell<K, MODE, FT>(a, c, fbase);
        }
    } else {
        const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
        if (c >= a.cells) return;
        unit_cell<K, MODE, FT>(a, c, int(blockIdx.y) * FT);
    }
}

// ---------------------------------------------------------------- unit stride, 128-bit vectors

// V = 16 / sizeof(element) consecutive elements of a plane as 16-byte loads
// and stores (p must be 16-byte aligned).
template <typename T, int NV>
__device__ __forceinline__ void ld_vec(const T* p, T* x)
{
    if constexpr (sizeof(T) == 4) {
        static_assert(NV % 4 == 0, "float vectors");
#pragma unroll
        for (int q = 0; q < NV / 4; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p) + q);
            x[4 * q] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        }
    } else {
        static_assert(NV % 2 == 0, "double vectors");
#pragma unroll
        for (int q = 0; q < NV / 2; ++q) {
            const double2 v = __ldg(reinterpret_cast<const double2*>(p) + q);
            x[2 * q] = v.x;
            x[2 * q + 1] = v.y;
        }
    }
}

template <typename T, int NV>
__device__ __forceinline__ void st_vec(T* p, const T* x)
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < NV / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < NV / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(x[2 * q], x[2 * q + 1]);
    }
}

// w[j] = x[r + j], j = 0..V, for a runtime r in [0, V), by a select network
// on the bits of r (no divergence, no local-memory indexing).
template <typename R, int V>
__device__ __forceinline__ void window(const R (&x)[2 * V], int r, R (&w)[V + 1])
{
    static_assert(V == 2 || V == 4, "vector widths");
    if constexpr (V == 2) {
#pragma unroll
        for (int j = 0; j <= V; ++j) w[j] = (r & 1) ? x[j + 1] : x[j];
    } else {
        R y[V + 3];
#pragma unroll
        for (int j = 0; j < V + 3; ++j) y[j] = (r & 1) ? x[j + 1] : x[j];
#pragma unroll
        for (int j = 0; j <= V; ++j) w[j] = (r & 2) ? y[j + 2] : y[j];
    }
}

// Cells c0 .. c0+V-1 of one line (V | n_0, so they share the line and its
// shift).  Their sources are the V+1 consecutive cells b0 = i0-sigma-1 ..
// i0-sigma+V-1 of the periodic line, which lie in two consecutive aligned
// V-vectors of the line's ring of n_0/V vectors: loaded as 16-byte vectors,
// the window is cut out by `window`, the V targets are stored as vectors.
template <int K, int MODE, int FT, bool MEAN>
__device__ __forceinline__ void unit_vec_body(const SweepArgs& a, uint32_t c0, uint32_t i0,
                                              uint32_t cls, int fbase)
{
    using T = typename St<MODE>::T;
    using R = typename St<MODE>::R;
    static_assert(!St<MODE>::scaled, "vector form of the unscaled stores");
    constexpr int V = 16 / sizeof(T);
    constexpr int O = K + 1;
    const int32_t N = int32_t(a.N);
    const uint32_t ls = c0 - i0;   // first cell of the line
    const int32_t sig = __ldg(a.tab.sigma + cls);
    int32_t b0 = int32_t(i0) - sig - 1;
    b0 += b0 < 0 ? N : 0;
    b0 += b0 < 0 ? N : 0;
    const int32_t q1 = b0 & ~(V - 1);
    const int r = int(b0 - q1);
    int32_t q2 = q1 + V;
    q2 -= q2 >= N ? N : 0;

    int jb[FT];
    group_bases<FT>(fbase, a.nfib, O, 1, jb);
    Mats<K, MODE> M;
    M.template load<MEAN>(a.tab, cls);

    R w[FT][O][V + 1];
    double wm[V + 1];
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if (MEAN && u == 0 && l == 0) {
                double x[2 * V];
                ld_vec<double, V>(a.src.mean + ls + q1, x);
                ld_vec<double, V>(a.src.mean + ls + q2, x + V);
                window<double, V>(x, r, wm);
            } else {
                const T* p = plane_ptr<T>(a.src.hi, a.pstride, jb[u] + l) + ls;
                T x[2 * V];
                ld_vec<T, V>(p + q1, x);
                ld_vec<T, V>(p + q2, x + V);
                window<R, V>(x, r, w[u][l]);
            }
        }
    R o[FT][O][V];
    double om[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        CellVals<K, MODE, FT> ca, cb, out;
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                ca.v[u][l] = w[u][l][v + 1];
                cb.v[u][l] = w[u][l][v];
            }
        if constexpr (MEAN) {
            ca.m = wm[v + 1];
            cb.m = wm[v];
        }
        combine<K, MODE, FT, MEAN>(M, ca, cb, out);
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) o[u][l][v] = out.v[u][l];
        if constexpr (MEAN) om[v] = out.m;
    }
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if (MEAN && u == 0 && l == 0)
                st_vec<double, V>(a.dst.mean + c0, om);
            else
                st_vec<T, V>(plane_ptr_w<T>(a.dst.hi, a.pstride, jb[u] + l) + c0, o[u][l]);
        }
}

// Sweep along dimension 0 with 16-byte vectors: one thread per V consecutive
// target cells and fibre group (see unit_grid); needs n_0 divisible by V.
template <int K, int MODE, int FT, bool GF>
__global__ void __launch_bounds__(256) k_sweep_unit_vec(const SweepArgs a)
{
    constexpr int V = 16 / sizeof(typename St<MODE>::T);
    auto body = [&](uint32_t c0, int fbase) {
        const uint32_t line = a.fdN.div(c0);
        const uint32_t i0 = c0 - line * a.N;
        const uint32_t cls = shift_class(a, 0, line);
        if (St<MODE>::mean64 && fbase == 0)
            unit_vec_body<K, MODE, FT, true>(a, c0, i0, cls, fbase);
        else
            unit_vec_body<K, MODE, FT, false>(a, c0, i0, cls, fbase);
    };
    if constexpr (GF) {
        const int fbase = int(blockIdx.x) * FT;
        for (uint32_t t = blockIdx.y; t * blockDim.x * V < a.cells; t += gridDim.y) {
            const uint32_t c0 = (t * blockDim.x + threadIdx.x) * V;
            if (c0 >= a.cells) break;
            body(c0, fbase);
        }
    } else {
        const uint32_t c0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
        if (c0 >= a.cells) return;
        body(c0, int(blockIdx.y) * FT);
    }
}

// ---------------------------------------------------------------- strided

struct LineSetup {
    uint32_t base;    // cell at i = 0 of the line
    uint32_t cls;
    int32_t sig;
    uint32_t i0, i1;  // target cells of this thread's chunk
    int fbase;
    bool active;
};

// The thread's line (an (outer, inner) pair), its shift class, and the
// target cells of chunk `chunk` of it.
__device__ __forceinline__ LineSetup line_setup(const SweepArgs& a, uint32_t line, uint32_t grp,
                                                uint32_t chunk, int FT)
{
    LineSetup L{};
    L.active = false;
    if (line >= a.lines) return L;
    L.fbase = int(grp) * FT;
    const uint32_t outer = a.fdInner.div(line);
    const uint32_t inn = line - outer * a.inner;
    L.base = outer * a.N * a.inner + inn;
    L.cls = shift_class(a, inn, outer);
    L.sig = __ldg(a.tab.sigma + L.cls);
    L.i0 = chunk * a.chunk;
    L.i1 = L.i0 + a.chunk;
    if (L.i1 > a.N) L.i1 = a.N;
    L.active = L.i0 < L.i1;
    return L;
}

__device__ __forceinline__ LineSetup line_setup_grid(const SweepArgs& a, int FT)
{
    return line_setup(a, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y % uint32_t(a.nfg),
                      blockIdx.y / uint32_t(a.nfg), FT);
}

// The walk's mean row uses the branching conversions (measured: about 10%
// faster than the branch-free form along dimensions > 0 of the 4D store).
template <int K, int MODE, int FT, int U, bool MEAN>
__device__ __forceinline__ void strided_body(const SweepArgs& a, const LineSetup& L)
{
    constexpr int O = K + 1;
    constexpr bool SC = St<MODE>::scaled;
    int jb[FT];
    if constexpr (SC) {
#pragma unroll
        for (int u = 0; u < FT; ++u) jb[u] = fibre_base(u, O, a.ostride);
    } else {
        group_bases<FT>(L.fbase, a.nfib, O, a.ostride, jb);
    }
    Mats<K, MODE> M;
    M.template load<MEAN>(a.tab, L.cls);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;

    GroupPtrs<K, MODE, FT, MEAN> P;
    if constexpr (!SC) P.init(a.src, a.dst, a.pstride, jb, a.ostride, L.base);
    auto load_row = [&](int32_t row, CellVals<K, MODE, FT>& cv) {
        if constexpr (SC)
            load_cell<K, MODE, FT, true>(a.src, a.pstride, L.base + uint32_t(row) * a.inner, jb,
                                         a.ostride, cv);
        else
            P.load(uint32_t(row) * a.inner, cv);
    };
    auto store_row = [&](uint32_t i, const CellVals<K, MODE, FT>& cv) {
        if constexpr (SC)
            store_cell<K, MODE, FT, true>(a.dst, a.pstride, L.base + i * a.inner, jb, a.ostride, cv);
        else
            P.store(i * a.inner, cv);
    };

    CellVals<K, MODE, FT> prev;
    load_row(ib, prev);
    uint32_t i = L.i0;
    if constexpr (U > 1) {
        for (; i + U <= L.i1; i += U) {
            CellVals<K, MODE, FT> cur[U];
#pragma unroll
            for (int s = 0; s < U; ++s) {
                int32_t x = ia + s;
                x -= x >= N ? N : 0;
                load_row(x, cur[s]);
            }
#pragma unroll
            for (int s = 0; s < U; ++s) {
                CellVals<K, MODE, FT> out;
                combine<K, MODE, FT, MEAN, CV_BRANCH>(M, cur[s], s == 0 ? prev : cur[s - 1], out);
                store_row(i + s, out);
            }
            prev = cur[U - 1];
            ia += U;
            ia -= ia >= N ? N : 0;
        }
    }
    for (; i < L.i1; ++i) {
        CellVals<K, MODE, FT> cur, out;
        load_row(ia, cur);
        combine<K, MODE, FT, MEAN, CV_BRANCH>(M, cur, prev, out);
        store_row(i, out);
        prev = cur;
        ++ia;
        if (ia == N) ia = 0;
    }
}

template <int K, int MODE, int FT, int U>
__device__ __forceinline__ void strided_line(const SweepArgs& a, const LineSetup& L)
{
    if (St<MODE>::scaled || (St<MODE>::mean64 && L.fbase == 0))
        strided_body<K, MODE, FT, U, true>(a, L);
    else
        strided_body<K, MODE, FT, U, false>(a, L);
}

// Sweep along dimension m > 0: one thread per line (and fibre group and
// chunk of the line, blockIdx.y = chunk * nfg + group), walking the target
// cells of its chunk U cells per step with the loads of a step issued first.
template <int K, int MODE, int FT, int U>
__global__ void __launch_bounds__(128) k_sweep_strided(const SweepArgs a)
{
    const LineSetup L = line_setup_grid(a, FT);
    if (!L.active) return;
    strided_line<K, MODE, FT, U>(a, L);
}

// ---------------------------------------------------------------- scaled stores, cooperative

// The scaled stores need the maximum over every coefficient of a new cell.
// When a cell has too many fibres for one thread's registers, G threads share
// it: a block holds 32 cells or lines (threadIdx.x) times G fibre groups of
// NF/G fibres (threadIdx.y).  Each thread computes its fibres, writes its
// local maximum to shared memory, and after one block barrier every thread of
// the cell reads the G maxima and encodes its values with the common scale.
// The strided form alternates two shared buffers, so one barrier per row
// suffices: a thread can only overwrite a buffer after every thread has
// passed the next barrier, i.e. has finished reading it.  All threads of a
// block walk the same rows (the chunk is per block), and threads past the
// last line or cell still take part in every barrier.

template <int K, int MODE, int FG>
__device__ __forceinline__ void coop_combine(const Mats<K, MODE>& M, const CellVals<K, MODE, FG>& a,
                                             const CellVals<K, MODE, FG>& b, bool mean,
                                             CellVals<K, MODE, FG>& out)
{
    if (mean)
        combine<K, MODE, FG, true>(M, a, b, out);
    else
        combine<K, MODE, FG, false>(M, a, b, out);
}

template <int K, int MODE, int FG>
__device__ __forceinline__ void coop_load(const Planes& p, int64_t pstride, uint32_t c,
                                          const int (&jb)[FG], int ostride, bool mean,
                                          CellVals<K, MODE, FG>& cv)
{
    if (mean)
        load_cell<K, MODE, FG, true>(p, pstride, c, jb, ostride, cv);
    else
        load_cell<K, MODE, FG, false>(p, pstride, c, jb, ostride, cv);
}

// Encode and store with the scale 1/inv; group 0 also stores the mean and s.
template <int K, int MODE, int FG>
__device__ __forceinline__ void coop_store(const Planes& p, int64_t pstride, uint32_t c,
                                           const int (&jb)[FG], int ostride, bool mean, float s,
                                           float inv, const CellVals<K, MODE, FG>& cv)
{
    using T = typename St<MODE>::T;
    constexpr int O = K + 1;
#pragma unroll
    for (int u = 0; u < FG; ++u)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if (mean && u == 0 && l == 0) {
                p.mean[c] = cv.m;
                p.scale[c] = s;
            } else {
                st_raw(plane_ptr_w<T>(p.hi, pstride, jb[u] + l * ostride) + c, cv.v[u][l] * inv);
            }
        }
}

template <int K, int MODE, int FG>
__device__ __forceinline__ float local_max(const CellVals<K, MODE, FG>& cv)
{
    float mx = 0.0f;
#pragma unroll
    for (int u = 0; u < FG; ++u)
#pragma unroll
        for (int l = 0; l < K + 1; ++l) mx = fmaxf(mx, fabsf(cv.v[u][l]));   // v[0][0] of the mean group is 0
    return mx;
}

template <int K, int MODE, int NF, int G>
__global__ void __launch_bounds__(32 * G) k_sweep_unit_coop(const SweepArgs a)
{
    static_assert(St<MODE>::scaled && NF % G == 0, "cooperative scaled sweep");
    constexpr int FG = NF / G;
    constexpr int O = K + 1;
    __shared__ float smax[G][32];
    const int lane = threadIdx.x, g = threadIdx.y;
    const uint32_t c = blockIdx.x * 32 + lane;
    const bool active = c < a.cells;
    const bool mean = g == 0;
    const uint32_t cc = active ? c : 0;
    const uint32_t line = a.fdN.div(cc);
    const uint32_t i = cc - line * a.N;
    const uint32_t cls = shift_class(a, 0, line);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    int32_t ia = int32_t(i) - sig;
    ia += ia < 0 ? int32_t(a.N) : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? int32_t(a.N) : 0;
    int jb[FG];
#pragma unroll
    for (int u = 0; u < FG; ++u) jb[u] = (g * FG + u) * O;   // fibre stride 1 along dimension 0
    Mats<K, MODE> M;
    M.template load<true>(a.tab, cls);
    CellVals<K, MODE, FG> va, vb, out;
    if (active) {
        coop_load<K, MODE, FG>(a.src, a.pstride, cc - i + uint32_t(ia), jb, 1, mean, va);
        coop_load<K, MODE, FG>(a.src, a.pstride, cc - i + uint32_t(ib), jb, 1, mean, vb);
        coop_combine<K, MODE, FG>(M, va, vb, mean, out);
        smax[g][lane] = local_max<K, MODE, FG>(out);
    }
    __syncthreads();
    if (!active) return;
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < G; ++q) mx = fmaxf(mx, smax[q][lane]);
    float s, inv;
    pow2_scale(mx, s, inv);
    coop_store<K, MODE, FG>(a.dst, a.pstride, c, jb, 1, mean, s, inv, out);
}

template <int K, int MODE, int NF, int G>
__global__ void __launch_bounds__(32 * G) k_sweep_strided_coop(const SweepArgs a)
{
    static_assert(St<MODE>::scaled && NF % G == 0, "cooperative scaled sweep");
    constexpr int FG = NF / G;
    constexpr int O = K + 1;
    __shared__ float smax[2][G][32];
    const int lane = threadIdx.x, g = threadIdx.y;
    const uint32_t line = blockIdx.x * 32 + lane;
    const bool active = line < a.lines;
    const bool mean = g == 0;
    const LineSetup L = line_setup(a, active ? line : 0, 0, blockIdx.y, 1);
    if (!L.active) return;   // the chunk is empty for the whole block
    int jb[FG];
#pragma unroll
    for (int u = 0; u < FG; ++u) jb[u] = fibre_base(g * FG + u, O, a.ostride);
    Mats<K, MODE> M;
    M.template load<true>(a.tab, L.cls);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    // the loads of row i+1 are issued before row i's barrier and stores
    CellVals<K, MODE, FG> prev, cur;
    if (active) {
        coop_load<K, MODE, FG>(a.src, a.pstride, L.base + uint32_t(ib) * a.inner, jb, a.ostride, mean,
                               prev);
        coop_load<K, MODE, FG>(a.src, a.pstride, L.base + uint32_t(ia) * a.inner, jb, a.ostride, mean,
                               cur);
    }
    int buf = 0;
    for (uint32_t i = L.i0; i < L.i1; ++i) {
        ++ia;
        if (ia == N) ia = 0;
        CellVals<K, MODE, FG> nxt, out;
        if (active) {
            if (i + 1 < L.i1)
                coop_load<K, MODE, FG>(a.src, a.pstride, L.base + uint32_t(ia) * a.inner, jb, a.ostride,
                                       mean, nxt);
            coop_combine<K, MODE, FG>(M, cur, prev, mean, out);
            smax[buf][g][lane] = local_max<K, MODE, FG>(out);
        }
        __syncthreads();
        if (active) {
            float mx = 0.0f;
#pragma unroll
            for (int q = 0; q < G; ++q) mx = fmaxf(mx, smax[buf][q][lane]);
            float s, inv;
            pow2_scale(mx, s, inv);
            coop_store<K, MODE, FG>(a.dst, a.pstride, L.base + i * a.inner, jb, a.ostride, mean, s, inv,
                                    out);
            prev = cur;
            cur = nxt;
        }
        buf ^= 1;
    }
}

// ---------------------------------------------------------------- scaled stores, cell records

// Record layout of the scaled stores for the shapes that fill a record well:
// the higher coefficients of a cell are one record of R = round_up(o^d, 8)
// 16-bit slots, slot J holding coefficient J (slot 0 and the padding slots
// stay zero).  A thread reads and writes a whole cell with 16-byte vectors;
// with the sweep dimension M a template parameter, the slots of every fibre
// are compile-time register positions.
constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }
template <int K, int D>
struct RecShape {
    static constexpr int O = K + 1;
    static constexpr int NC = ipow_c(O, D);
    static constexpr int R = (NC + 7) / 8 * 8;
    static constexpr int NV = R / 8;   // 16-byte vectors per record
    static constexpr int NF = NC / O;  // fibres
};

// Slot of coefficient l of fibre f for a sweep along dimension M.
template <int K, int M>
__host__ __device__ constexpr int rec_slot(int f, int l)
{
    return (f / ipow_c(K + 1, M)) * ipow_c(K + 1, M + 1) + (f % ipow_c(K + 1, M)) + l * ipow_c(K + 1, M);
}

template <int MODE>
__device__ __forceinline__ float dec16(uint32_t bits)
{
    if constexpr (MODE == M_BF16)
        return __uint_as_float(bits << 16);
    else
        return __half2float(__ushort_as_half((unsigned short)bits));
}
template <int MODE>
__device__ __forceinline__ uint32_t enc16(float v)
{
    if constexpr (MODE == M_BF16)
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    else
        return __half_as_ushort(__float2half_rn(v));
}

// Two values to a packed pair of 16-bit codes (lo in the low half), rounded
// to nearest even: one paired conversion instead of two conversions, a
// shift and an or (the same bits as enc16 on each).
template <int MODE>
__device__ __forceinline__ uint32_t enc16x2(float lo, float hi)
{
    if constexpr (MODE == M_BF16) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&p);
    } else {
        const __half2 p = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&p);
    }
}

template <int MODE, int NV>
__device__ __forceinline__ float rec_get(const uint4 (&r)[NV], int J)
{
    const uint4& q = r[J / 8];
    const int w = (J % 8) / 2;
    const uint32_t word = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
    return dec16<MODE>((J & 1) ? (word >> 16) : (word & 0xffffu));
}

// New record of one cell from the records of its source cells a and b.
template <int K, int MODE, int D, int M>
__device__ __forceinline__ void rec_combine(const Mats<K, MODE>& M_, const uint4 (&ra)[RecShape<K, D>::NV],
                                            float sa, double ma, const uint4 (&rb)[RecShape<K, D>::NV],
                                            float sb, double mb, float (&out)[RecShape<K, D>::R],
                                            double& om)
{
    using RS = RecShape<K, D>;
    constexpr int O = K + 1;
#pragma unroll
    for (int f = 0; f < RS::NF; ++f) {
        CellVals<K, MODE, 1> va, vb, vo;
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int J = rec_slot<K, M>(f, l);
            va.v[0][l] = J == 0 ? 0.0f : rec_get<MODE, RS::NV>(ra, J) * sa;
            vb.v[0][l] = J == 0 ? 0.0f : rec_get<MODE, RS::NV>(rb, J) * sb;
        }
        if (f == 0) {
            va.m = ma;
            vb.m = mb;
            combine<K, MODE, 1, true>(M_, va, vb, vo);
            om = vo.m;
        } else {
            combine<K, MODE, 1, false>(M_, va, vb, vo);
        }
#pragma unroll
        for (int l = 0; l < O; ++l) out[rec_slot<K, M>(f, l)] = vo.v[0][l];
    }
}

// Scale (cell-wide maximum) and pack a record; slot 0 and padding are zero.
template <int K, int MODE, int D>
__device__ __forceinline__ float rec_pack(float (&out)[RecShape<K, D>::R], uint4 (&ro)[RecShape<K, D>::NV])
{
    using RS = RecShape<K, D>;
    float mx = 0.0f;
#pragma unroll
    for (int J = 1; J < RS::NC; ++J) mx = fmaxf(mx, fabsf(out[J]));
    float s, inv;
    pow2_scale(mx, s, inv);
#pragma unroll
    for (int q = 0; q < RS::NV; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int J0 = 8 * q + 2 * h, J1 = J0 + 1;
            // slot 0 and padding slots encode +0, whose code is 0
            const float lo = (J0 >= 1 && J0 < RS::NC) ? out[J0] * inv : 0.0f;
            const float hi = (J1 >= 1 && J1 < RS::NC) ? out[J1] * inv : 0.0f;
            w[h] = enc16x2<MODE>(lo, hi);
        }
        ro[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return s;
}

template <int K, int D>
__device__ __forceinline__ void rec_load(const void* hi, uint32_t c, uint4 (&r)[RecShape<K, D>::NV])
{
    const uint4* p = static_cast<const uint4*>(hi) + size_t(c) * RecShape<K, D>::NV;
#pragma unroll
    for (int q = 0; q < RecShape<K, D>::NV; ++q) r[q] = __ldg(p + q);
}

template <int K, int D>
__device__ __forceinline__ void rec_store(void* hi, uint32_t c, const uint4 (&r)[RecShape<K, D>::NV])
{
    uint4* p = static_cast<uint4*>(hi) + size_t(c) * RecShape<K, D>::NV;
#pragma unroll
    for (int q = 0; q < RecShape<K, D>::NV; ++q) p[q] = r[q];
}

// Sweep along dimension 0 on cell records: one thread per target cell.
template <int K, int MODE, int D>
__global__ void __launch_bounds__(128) k_sweep_unit_rec(const SweepArgs a)
{
    using RS = RecShape<K, D>;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.cells) return;
    const uint32_t line = a.fdN.div(c);
    const uint32_t i = c - line * a.N;
    const uint32_t cls = shift_class(a, 0, line);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    int32_t ia = int32_t(i) - sig;
    ia += ia < 0 ? int32_t(a.N) : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? int32_t(a.N) : 0;
    const uint32_t ca = c - i + uint32_t(ia);
    const uint32_t cb = c - i + uint32_t(ib);
    Mats<K, MODE> M;
    M.template load<true>(a.tab, cls);
    uint4 ra[RS::NV], rb[RS::NV];
    rec_load<K, D>(a.src.hi, ca, ra);
    rec_load<K, D>(a.src.hi, cb, rb);
    double om;
    float out[RS::R];
    rec_combine<K, MODE, D, 0>(M, ra, __ldg(a.src.scale + ca), __ldg(a.src.mean + ca), rb,
                               __ldg(a.src.scale + cb), __ldg(a.src.mean + cb), out, om);
    uint4 ro[RS::NV];
    const float s = rec_pack<K, MODE, D>(out, ro);
    rec_store<K, D>(a.dst.hi, c, ro);
    a.dst.scale[c] = s;
    a.dst.mean[c] = om;
}

// Sweep along dimension M on cell records: one thread per line walking its
// chunk, the previous source record kept in registers (also used along
// dimension 0, where the lines are contiguous runs of records).  With PF the
// next source record is loaded before the current one is computed.
template <int K, int MODE, int D, int M, bool PF>
__global__ void __launch_bounds__(128) k_sweep_strided_rec(const SweepArgs a)
{
    using RS = RecShape<K, D>;
    const LineSetup L = line_setup_grid(a, 1);
    if (!L.active) return;
    Mats<K, MODE> Mt;
    Mt.template load<true>(a.tab, L.cls);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    uint4 prev[RS::NV];
    uint32_t cb = L.base + uint32_t(ib) * a.inner;
    rec_load<K, D>(a.src.hi, cb, prev);
    float sp = __ldg(a.src.scale + cb);
    double mp = __ldg(a.src.mean + cb);
    uint4 cur[RS::NV];
    float sc = 0.0f;
    double mc = 0.0;
    if constexpr (PF) {
        const uint32_t ca = L.base + uint32_t(ia) * a.inner;
        rec_load<K, D>(a.src.hi, ca, cur);
        sc = __ldg(a.src.scale + ca);
        mc = __ldg(a.src.mean + ca);
    }
    for (uint32_t i = L.i0; i < L.i1; ++i) {
        uint4 nxt[RS::NV];
        float sn = 0.0f;
        double mn = 0.0;
        if constexpr (PF) {
            if (i + 1 < L.i1) {
                int32_t in = ia + 1;
                in -= in == N ? N : 0;
                const uint32_t cn = L.base + uint32_t(in) * a.inner;
                rec_load<K, D>(a.src.hi, cn, nxt);
                sn = __ldg(a.src.scale + cn);
                mn = __ldg(a.src.mean + cn);
            }
        } else {
            const uint32_t ca = L.base + uint32_t(ia) * a.inner;
            rec_load<K, D>(a.src.hi, ca, cur);
            sc = __ldg(a.src.scale + ca);
            mc = __ldg(a.src.mean + ca);
        }
        float out[RS::R];
        double om;
        rec_combine<K, MODE, D, M>(Mt, cur, sc, mc, prev, sp, mp, out, om);
        uint4 ro[RS::NV];
        const float s = rec_pack<K, MODE, D>(out, ro);
        const uint32_t c = L.base + i * a.inner;
        rec_store<K, D>(a.dst.hi, c, ro);
        a.dst.scale[c] = s;
        a.dst.mean[c] = om;
#pragma unroll
        for (int q = 0; q < RS::NV; ++q) prev[q] = cur[q];
        sp = sc;
        mp = mc;
        if constexpr (PF) {
#pragma unroll
            for (int q = 0; q < RS::NV; ++q) cur[q] = nxt[q];
            sc = sn;
            mc = mn;
        }
        ++ia;
        if (ia == N) ia = 0;
    }
}

// ---------------------------------------------------------------- strided, cp.async ring

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    static_assert(BYTES == 4 || BYTES == 8, "cp.async element size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(smem)), "l"(gmem),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Dynamic shared memory of k_sweep_strided_async with B threads per block:
// P+1 row slots, each with one FP64 mean word and FT*(k+1) values per thread.
template <int K, int MODE, int FT, int P, int B>
constexpr size_t strided_async_smem()
{
    return size_t(P + 1) * size_t(B) * (8 + size_t(FT) * (K + 1) * sizeof(typename St<MODE>::T));
}

template <int K, int MODE, int FT, int P, int B, bool MEAN>
__device__ __forceinline__ void async_body(const SweepArgs& a, const LineSetup& L)
{
    using T = typename St<MODE>::T;
    constexpr int O = K + 1;
    constexpr int S = P + 1;
    constexpr int V = FT * O;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t tid = threadIdx.x;
    // [slot][B] means, then [slot][V][B] values: every offset below is a
    // compile-time constant from the thread's own column
    double* sm_mean = reinterpret_cast<double*>(smem_raw) + tid;
    T* sm_val = reinterpret_cast<T*>(smem_raw + size_t(S) * B * 8) + tid;

    int jb[FT];
    group_bases<FT>(L.fbase, a.nfib, O, a.ostride, jb);
    Mats<K, MODE> M;
    M.template load<MEAN>(a.tab, L.cls);
    GroupPtrs<K, MODE, FT, MEAN> G;
    G.init(a.src, a.dst, a.pstride, jb, a.ostride, L.base);

    const int32_t N = int32_t(a.N);
    // rows in consumption order: row 0 is source cell i0-sigma-1, row q >= 1
    // the source cell i0+q-1-sigma of target i0+q-1; all periodic in N
    const int nrows = int(L.i1 - L.i0) + 1;
    int32_t frow = int32_t(L.i0) - L.sig - 1;
    frow += frow < 0 ? N : 0;
    frow += frow < 0 ? N : 0;

    auto fetch = [&](int slot, uint32_t off) {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0)
                    cp_async<8>(sm_mean + slot * B, G.sm + off);
                else
                    cp_async<sizeof(T)>(sm_val + (slot * V + u * O + l) * B, G.s[u][l] + off);
            }
    };
    auto read = [&](int slot, CellVals<K, MODE, FT>& cv) {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0) {
                    cv.m = sm_mean[slot * B];
                    cv.v[0][0] = 0;
                } else {
                    cv.v[u][l] = sm_val[(slot * V + u * O + l) * B];
                }
            }
    };

#pragma unroll
    for (int q = 0; q < P; ++q) {
        if (q < nrows) {
            fetch(q, uint32_t(frow) * a.inner);
            ++frow;
            frow -= frow >= N ? N : 0;
        }
        cp_async_commit();
    }
    CellVals<K, MODE, FT> prev, cur;
    int slot = 0;    // slot of row q
    int rslot = P;   // slot that row q + P goes to (= slot of row q - 1)
    for (int q = 0; q < nrows; ++q) {
        cp_async_wait<P - 1>();
        read(slot, cur);
        if (q + P < nrows) {
            fetch(rslot, uint32_t(frow) * a.inner);
            ++frow;
            frow -= frow >= N ? N : 0;
        }
        cp_async_commit();
        if (q > 0) {
            CellVals<K, MODE, FT> out;
            combine<K, MODE, FT, MEAN>(M, cur, prev, out);
            G.store((L.i0 + uint32_t(q) - 1) * a.inner, out);
        }
        prev = cur;
        rslot = slot;
        slot = slot + 1 == S ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

// Same walk as k_sweep_strided, but the source rows are fetched P rows ahead
// with cp.async into a per-thread ring of P+1 row slots in shared memory, so
// every thread keeps P rows of loads in flight while it computes.  A thread
// only reads slots it filled itself (cp.async.wait_group makes them visible
// to the issuing thread), so no block barrier is needed; a slot is refilled
// one iteration after it was read and its values were used.  B threads per
// block.
template <int K, int MODE, int FT, int P, int B>
__global__ void __launch_bounds__(B) k_sweep_strided_async(const SweepArgs a)
{
    static_assert(!St<MODE>::scaled, "cp.async ring needs 4- or 8-byte elements");
    const LineSetup L = line_setup_grid(a, FT);
    if (!L.active) return;
    if (St<MODE>::mean64 && L.fbase == 0)
        async_body<K, MODE, FT, P, B, true>(a, L);
    else
        async_body<K, MODE, FT, P, B, false>(a, L);
}

}  // namespace sl
