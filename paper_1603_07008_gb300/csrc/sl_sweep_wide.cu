// sl_sweep_wide.cu -- sweeps of the stores with FP32 planes ("# double" =
// 0 .. 3 of Sec. III-A) with every row computed in FP64 arithmetic: each
// FP32 coefficient is widened to FP64 on load, the update rule of Sec. II-A
// is evaluated with the FP64 matrices, and the new FP32 coefficients are
// rounded once (to nearest, ties to even) on store.  The stores keep their
// layout and bytes; only the arithmetic differs from their own sweeps (which
// compute the rows of FP32 coefficients in FP32).
//
// Sec. III-A states which coefficients are stored in double precision, not
// the precision of the arithmetic; this is the reading in which a store
// differs from the FP64 scheme only by the rounding of what it stores.
//
// One thread updates one fibre of one target cell (sweep along dimension 0,
// the fibre is blockIdx.y's) or walks one fibre along a chunk of a line
// (other dimensions), like the sweeps of the general split stores.  The
// entries of a fibre are FP64 or FP32 according to the store's layout:
//   WL_MIXED   -- the mixed store: coefficient 0 (the mean) in its FP64 plane,
//                 coefficient J >= 1 at hi + (J-1) * pstride;
//   WL_ALL32   -- the all-FP32 store: coefficient J at hi + (J-1) * pstride
//                 for every J (hi points one plane into the FP32 block);
//   WL_MAPPED  -- "# double" = 2, 3: the coefficient map gives each J its
//                 FP64 (map < 0) or FP32 (map >= 0) plane.
// Whether an entry is FP64 depends on the fibre only, so it is uniform per
// block.  The fibre of the mean, when the mean is FP64, takes the
// conservation form of the FP64 store (row 0: a_0 + alpha (b_0 - a_0) +
// sum_{l>=1} A_0l (a_l - b_l); rows j >= 1 use B_j0 = -A_j0); every other
// fibre, and the mean's fibre of the all-FP32 store, the plain sums.
//
// The FP64 pipe of GB300 runs at a small fraction of the FP32 rate, so these
// sweeps cost about as much per coefficient as the FP64 store's (2o FP64 FMAs
// per coefficient); they exist for accuracy, not speed.  The conversions take
// an integer-pipe path for normal values and the conversion instructions
// otherwise, so their results are the IEEE conversions for every input.
#include "sl_sweep.cuh"

namespace sl {

namespace {

enum : int { WL_MIXED = 0, WL_ALL32 = 1, WL_MAPPED = 2 };

// binary32 -> binary64, exact for every input.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t e = (__float_as_uint(x) >> 23) & 0xffu;
    if (e - 1u < 254u) return f2d_fast(x);   // normal
    return double(x);
}

// binary64 -> binary32, rounded to nearest even, for every input.
__device__ __forceinline__ float narrow(double x)
{
    const uint32_t e = (uint32_t(__double2hiint(x)) >> 20) & 0x7ffu;
    if (e - 897u < 254u) return d2f_fast(x, false);   // result normal or overflowing
    return __double2float_rn(x);
}

template <int K>
struct WMats {
    static constexpr int O = K + 1;
    double a[O][O], b[O][O];
    double alpha;

    __device__ __forceinline__ void load(const ShiftTable& t, uint32_t cls)
    {
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
        alpha = __ldg(t.alpha + cls);
    }
};

// Source and target addresses of the o entries of one fibre (coefficients
// jb + l * ostride), offset by a base cell; bit l of `wide` set when entry l
// is an FP64 coefficient.
template <int K, int LAYOUT>
struct WPtrs {
    static constexpr int O = K + 1;
    const void* s[O];
    void* d[O];
    uint32_t wide;

    __device__ __forceinline__ void init(const SweepArgs& a, int jb, uint32_t base)
    {
        wide = 0;
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int J = jb + l * a.ostride;
            if (LAYOUT == WL_MAPPED) {
                const int e = __ldg(a.cmap + J);
                if (e < 0) {
                    s[l] = a.src.mean + int64_t(-1 - e) * a.pstride + base;
                    d[l] = a.dst.mean + int64_t(-1 - e) * a.pstride + base;
                    wide |= 1u << l;
                } else {
                    s[l] = static_cast<const float*>(a.src.hi) + int64_t(e) * a.pstride + base;
                    d[l] = static_cast<float*>(a.dst.hi) + int64_t(e) * a.pstride + base;
                }
            } else if (LAYOUT == WL_MIXED && J == 0) {
                s[l] = a.src.mean + base;
                d[l] = a.dst.mean + base;
                wide |= 1u << l;
            } else {
                s[l] = plane_ptr<float>(a.src.hi, a.pstride, J) + base;
                d[l] = plane_ptr_w<float>(a.dst.hi, a.pstride, J) + base;
            }
        }
    }
    __device__ __forceinline__ void load(uint32_t off, double (&v)[O]) const
    {
#pragma unroll
        for (int l = 0; l < O; ++l)
            v[l] = (wide >> l) & 1u ? __ldg(static_cast<const double*>(s[l]) + off)
                                    : widen(__ldg(static_cast<const float*>(s[l]) + off));
    }
    __device__ __forceinline__ void store(uint32_t off, const double (&v)[O]) const
    {
#pragma unroll
        for (int l = 0; l < O; ++l) {
            if ((wide >> l) & 1u)
                static_cast<double*>(d[l])[off] = v[l];
            else
                static_cast<float*>(d[l])[off] = narrow(v[l]);
        }
    }
    // the fibre of an FP64 mean takes the conservation form
    __device__ __forceinline__ bool conserving(int jb) const { return jb == 0 && (wide & 1u); }
};

// New entries o of one fibre from the source cells a = c_{i-sigma} and
// b = c_{i-sigma-1} (update rule of Sec. II-A), in FP64.
template <int K>
__device__ __forceinline__ void wcombine(const WMats<K>& M, const double (&a)[K + 1], const double (&b)[K + 1],
                                         double (&o)[K + 1], bool cons)
{
    constexpr int O = K + 1;
    if (cons) {
        const double t = b[0] - a[0];
        double r = fma(M.alpha, t, a[0]);
#pragma unroll
        for (int l = 1; l < O; ++l) r = fma(M.a[0][l], a[l] - b[l], r);
        o[0] = r;
#pragma unroll
        for (int j = 1; j < O; ++j) {
            double s = -M.a[j][0] * t;
#pragma unroll
            for (int l = 1; l < O; ++l) {
                s = fma(M.a[j][l], a[l], s);
                s = fma(M.b[j][l], b[l], s);
            }
            o[j] = s;
        }
    } else {
#pragma unroll
        for (int j = 0; j < O; ++j) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < O; ++l) {
                s = fma(M.a[j][l], a[l], s);
                s = fma(M.b[j][l], b[l], s);
            }
            o[j] = s;
        }
    }
}

// Sweep along dimension 0: one thread per target cell of fibre blockIdx.y
// (fibre stride 1, so its coefficients are jb .. jb + k with jb = o * fibre).
template <int K, int LAYOUT>
__global__ void __launch_bounds__(256) k_wide_unit(const SweepArgs a)
{
    constexpr int O = K + 1;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.cells) return;
    const int jb = int(blockIdx.y) * O;
    const uint32_t line = a.fdN.div(c);
    const uint32_t i = c - line * a.N;
    const uint32_t cls = shift_class(a, 0, line);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(i) - sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    WMats<K> M;
    M.load(a.tab, cls);
    WPtrs<K, LAYOUT> P;
    P.init(a, jb, c - i);
    double va[O], vb[O], vo[O];
    P.load(uint32_t(ia), va);
    P.load(uint32_t(ib), vb);
    wcombine<K>(M, va, vb, vo, P.conserving(jb));
    P.store(i, vo);
}

// Sweep along dimension m > 0: one thread per line, fibre and chunk of the
// line (blockIdx.y = chunk * nfg + fibre), walking its target cells U per
// step with the step's loads issued first; the source cell i - sigma of one
// target is the source cell i - sigma - 1 of the next, so it stays in
// registers.
template <int K, int LAYOUT, int U>
__global__ void __launch_bounds__(128) k_wide_strided(const SweepArgs a)
{
    constexpr int O = K + 1;
    const LineSetup L = line_setup_grid(a, 1);
    if (!L.active) return;
    const int jb = fibre_base(L.fbase, O, a.ostride);
    WMats<K> M;
    M.load(a.tab, L.cls);
    WPtrs<K, LAYOUT> P;
    P.init(a, jb, L.base);
    const bool cons = P.conserving(jb);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    double prev[O];
    P.load(uint32_t(ib) * a.inner, prev);
    uint32_t i = L.i0;
    for (; i + U <= L.i1; i += U) {
        double cur[U][O];
#pragma unroll
        for (int s = 0; s < U; ++s) {
            int32_t x = ia + s;
            x -= x >= N ? N : 0;
            P.load(uint32_t(x) * a.inner, cur[s]);
        }
#pragma unroll
        for (int s = 0; s < U; ++s) {
            double o[O];
            wcombine<K>(M, cur[s], s == 0 ? prev : cur[s - 1], o, cons);
            P.store((i + s) * a.inner, o);
        }
#pragma unroll
        for (int l = 0; l < O; ++l) prev[l] = cur[U - 1][l];
        ia += U;
        ia -= ia >= N ? N : 0;
    }
    for (; i < L.i1; ++i) {
        double cur[O], o[O];
        P.load(uint32_t(ia) * a.inner, cur);
        wcombine<K>(M, cur, prev, o, cons);
        P.store(i * a.inner, o);
#pragma unroll
        for (int l = 0; l < O; ++l) prev[l] = cur[l];
        ++ia;
        if (ia == N) ia = 0;
    }
}

template <int K, int LAYOUT>
cudaError_t wide_shape(const SweepLaunch& L)
{
    const SweepArgs& a = L.args;
    if (a.nfg != a.nfib) return cudaErrorInvalidValue;   // one fibre per thread
    if (LAYOUT == WL_MAPPED && !a.cmap) return cudaErrorInvalidValue;
    if (L.unit) {
        const dim3 grid((a.cells + 255) / 256, uint32_t(a.nfib));
        k_wide_unit<K, LAYOUT><<<grid, 256, 0, L.stream>>>(a);
        return cudaGetLastError();
    }
    if (a.chunk == 0) return cudaErrorInvalidValue;
    const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
    const dim3 grid((a.lines + 127) / 128, nchunk * uint32_t(a.nfg));
    // one cell per step: 72 registers at k = 2, 7 blocks per SM; the FP64
    // pipe then keeps more warps to draw on (4D 64^4: 635 GB/s against 603
    // with two cells per step and 588 with four)
    k_wide_strided<K, LAYOUT, 1><<<grid, 128, 0, L.stream>>>(a);
    return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t wide_degree(const SweepLaunch& L)
{
    switch (L.K) {
    case 0: return wide_shape<0, LAYOUT>(L);
    case 1: return wide_shape<1, LAYOUT>(L);
    case 2: return wide_shape<2, LAYOUT>(L);
    case 3: return wide_shape<3, LAYOUT>(L);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_sweep_wide(const SweepLaunch& L)
{
    switch (L.mode) {
    case M_F32: return wide_degree<WL_MIXED>(L);
    case M_F32ALL: return wide_degree<WL_ALL32>(L);
    case M_SPLIT2:
    case M_SPLIT3: return wide_degree<WL_MAPPED>(L);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sl
