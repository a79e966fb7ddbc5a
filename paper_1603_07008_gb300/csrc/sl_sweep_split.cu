// sl_sweep_split.cu -- sweeps of the general split stores, "# double" = q of
// Sec. III-A (Table II) for q = 2 and 3: the coefficients c_{j_0..j_{d-1}}
// whose every per-dimension index j_m is below q in FP64 planes, all others
// in FP32 planes.  In one dimension these are c_0 .. c_{q-1}, the stores of
// the paper's tables.
//
// A fibre along the sweep dimension (its other indices fixed) either has
// every other index below q -- then its entries l < q are FP64 and l >= q
// FP32 (an "S" fibre) -- or not, and then all its entries are FP32 (an "F"
// fibre).  One thread updates one fibre of one target cell (dimension 0) or
// walks one fibre along a chunk of a line (dimensions > 0); the fibre is
// blockIdx.y's, so the S/F choice is uniform per block.
//
// Arithmetic of an S fibre with the source cells a = c_{i-sigma} and
// b = c_{i-sigma-1} (update rule of Sec. II-A):
//   row 0, in the conservation form of the mixed store:
//     c'_0 = a_0 + alpha (b_0 - a_0) + sum_{1<=l<q} A_0l (a_l - b_l) + (G(a) - G(b)),
//     G(c) = sum_{l>=q} A_0l c_l formed in FP32, a function of one cell, so
//     the FP64 differences telescope along a line and mass is conserved to
//     FP64 rounding;
//   rows 1 <= j < q, in FP64:
//     A_j0 (a_0 - b_0) + sum_{1<=l<q} (A_jl a_l + B_jl b_l) + P_j,
//     P_j = sum_{l>=q} (A_jl a_l + B_jl b_l) formed in FP32 (its inputs are
//     FP32 values);
//   rows j >= q, in FP32:
//     A_j0 fl32(a_0 - b_0) + sum_{1<=l<q} (A_jl fl32(a_l) + B_jl fl32(b_l))
//     + sum_{l>=q} (A_jl a_l + B_jl b_l).
// The identities used are the projection's: A_00 + B_00 = 1, B_0l = -A_0l
// (l >= 1) and B_j0 = -A_j0 (j >= 1).  F fibres are computed in FP32.
//
// An S fibre costs 9 (q = 2) or 19 (q = 3) FP64-pipe instructions per target
// cell (the difference G(a) - G(b) is formed on the integer pipe, sub_widened).
// GB300 issues FP64 at a small fraction of its FP32 rate, so in one
// dimension these stores are bound by the FP64 pipe, not by HBM; the
// conversions run on the integer pipe (f2d_fast, d2f_fast) and the per-cell
// values G(c) and fl32(c_l) are formed once per source cell in the walks.
#include "sl_sweep.cuh"

namespace sl {

namespace {

template <int K, int Q>
struct SMats {
    static constexpr int O = K + 1;
    float a[O][O], b[O][O];
    double a64[Q][Q], b64[Q][Q];   // the FP64 block j, l < q
    double alpha;

    __device__ __forceinline__ void load(const ShiftTable& t, uint32_t cls)
    {
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
        const double* p64 = t.ab64 + size_t(cls) * ab_stride64(O);
#pragma unroll
        for (int j = 0; j < Q; ++j)
#pragma unroll
            for (int l = 0; l < Q; ++l) {
                a64[j][l] = __ldg(p64 + j * O + l);
                b64[j][l] = __ldg(p64 + O * O + j * O + l);
            }
        alpha = __ldg(t.alpha + cls);
    }
};

// One source cell of an S fibre with its per-cell derived values.
template <int K, int Q>
struct SCell {
    static constexpr int O = K + 1;
    double d[Q];       // entries 0 .. q-1
    float f[O - Q];    // entries q .. o-1
    float g;           // G(c)
    float r[Q];        // fl32(d[l]) for l >= 1
};

template <int K, int Q>
__device__ __forceinline__ void s_prepare(const SMats<K, Q>& M, SCell<K, Q>& v)
{
    constexpr int O = K + 1;
    float g = 0.0f;
#pragma unroll
    for (int l = Q; l < O; ++l) g = fmaf(M.a[0][l], v.f[l - Q], g);
    v.g = g;
    v.r[0] = 0.0f;
#pragma unroll
    for (int l = 1; l < Q; ++l) v.r[l] = d2f_fast(v.d[l], false);
}

template <int K, int Q>
__device__ __forceinline__ void s_combine(const SMats<K, Q>& M, const SCell<K, Q>& a, const SCell<K, Q>& b,
                                          double (&od)[Q], float (&of)[K + 1 - Q])
{
    constexpr int O = K + 1;
    const double t0 = b.d[0] - a.d[0];
    double r = fma(M.alpha, t0, a.d[0]);
#pragma unroll
    for (int l = 1; l < Q; ++l) r = fma(M.a64[0][l], a.d[l] - b.d[l], r);
    od[0] = r + sub_widened(a.g, b.g);
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        float p = 0.0f;
#pragma unroll
        for (int l = Q; l < O; ++l) {
            p = fmaf(M.a[j][l], a.f[l - Q], p);
            p = fmaf(M.b[j][l], b.f[l - Q], p);
        }
        double s = -M.a64[j][0] * t0;
#pragma unroll
        for (int l = 1; l < Q; ++l) {
            s = fma(M.a64[j][l], a.d[l], s);
            s = fma(M.b64[j][l], b.d[l], s);
        }
        od[j] = s + f2d_fast(p);
    }
    const float dm = d2f_fast(t0, true);   // fl32(a_0 - b_0)
#pragma unroll
    for (int j = Q; j < O; ++j) {
        float acc = M.a[j][0] * dm;
#pragma unroll
        for (int l = 1; l < Q; ++l) {
            acc = fmaf(M.a[j][l], a.r[l], acc);
            acc = fmaf(M.b[j][l], b.r[l], acc);
        }
#pragma unroll
        for (int l = Q; l < O; ++l) {
            acc = fmaf(M.a[j][l], a.f[l - Q], acc);
            acc = fmaf(M.b[j][l], b.f[l - Q], acc);
        }
        of[j - Q] = acc;
    }
}

template <int K>
__device__ __forceinline__ void f_combine(const float (&A)[K + 1][K + 1], const float (&B)[K + 1][K + 1],
                                          const float (&a)[K + 1], const float (&b)[K + 1], float (&o)[K + 1])
{
#pragma unroll
    for (int j = 0; j <= K; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int l = 0; l <= K; ++l) {
            acc = fmaf(A[j][l], a[l], acc);
            acc = fmaf(B[j][l], b[l], acc);
        }
        o[j] = acc;
    }
}

// Planes of coefficient map entry e (see Planes).
__device__ __forceinline__ double* lo_plane(const Planes& p, int64_t ps, int e)
{
    return p.mean + int64_t(-1 - e) * ps;
}
__device__ __forceinline__ float* hi_plane(const Planes& p, int64_t ps, int e)
{
    return static_cast<float*>(p.hi) + int64_t(e) * ps;
}

// Source and target pointers of one fibre (coefficients jb + l * ostride),
// offset by a base cell.
template <int K, int Q>
struct SPtrs {
    static constexpr int O = K + 1;
    const double* sd[Q];
    double* dd[Q];
    const float* sf[O - Q];
    float* df[O - Q];

    __device__ __forceinline__ void init(const SweepArgs& a, int jb, uint32_t base)
    {
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int e = __ldg(a.cmap + jb + l * a.ostride);
            if (l < Q) {
                sd[l] = lo_plane(a.src, a.pstride, e) + base;
                dd[l] = lo_plane(a.dst, a.pstride, e) + base;
            } else {
                sf[l - Q] = hi_plane(a.src, a.pstride, e) + base;
                df[l - Q] = hi_plane(a.dst, a.pstride, e) + base;
            }
        }
    }
    __device__ __forceinline__ void load(uint32_t off, SCell<K, Q>& v) const
    {
#pragma unroll
        for (int l = 0; l < Q; ++l) v.d[l] = __ldg(sd[l] + off);
#pragma unroll
        for (int l = 0; l < O - Q; ++l) v.f[l] = __ldg(sf[l] + off);
    }
    __device__ __forceinline__ void store(uint32_t off, const double (&od)[Q], const float (&of)[O - Q]) const
    {
#pragma unroll
        for (int l = 0; l < Q; ++l) dd[l][off] = od[l];
#pragma unroll
        for (int l = 0; l < O - Q; ++l) df[l][off] = of[l];
    }
};

template <int K>
struct FPtrs {
    static constexpr int O = K + 1;
    const float* s[O];
    float* d[O];

    __device__ __forceinline__ void init(const SweepArgs& a, int jb, uint32_t base)
    {
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int e = __ldg(a.cmap + jb + l * a.ostride);
            s[l] = hi_plane(a.src, a.pstride, e) + base;
            d[l] = hi_plane(a.dst, a.pstride, e) + base;
        }
    }
    __device__ __forceinline__ void load(uint32_t off, float (&v)[O]) const
    {
#pragma unroll
        for (int l = 0; l < O; ++l) v[l] = __ldg(s[l] + off);
    }
    __device__ __forceinline__ void store(uint32_t off, const float (&v)[O]) const
    {
#pragma unroll
        for (int l = 0; l < O; ++l) d[l][off] = v[l];
    }
};

// ---------------------------------------------------------------- dimension 0

// One thread per target cell of fibre blockIdx.y (fibre stride 1, so the
// fibre's coefficients are jb .. jb + k with jb = blockIdx.y * o).
template <int K, int Q>
__global__ void __launch_bounds__(256) k_split_unit(const SweepArgs a)
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
    const uint32_t ls = c - i;   // first cell of the line
    SMats<K, Q> M;
    M.load(a.tab, cls);
    if (__ldg(a.cmap + jb) < 0) {
        SPtrs<K, Q> P;
        P.init(a, jb, ls);
        SCell<K, Q> va, vb;
        P.load(uint32_t(ia), va);
        P.load(uint32_t(ib), vb);
        s_prepare<K, Q>(M, va);
        s_prepare<K, Q>(M, vb);
        double od[Q];
        float of[O - Q];
        s_combine<K, Q>(M, va, vb, od, of);
        P.store(i, od, of);
    } else {
        FPtrs<K> P;
        P.init(a, jb, ls);
        float va[O], vb[O], vo[O];
        P.load(uint32_t(ia), va);
        P.load(uint32_t(ib), vb);
        f_combine<K>(M.a, M.b, va, vb, vo);
        P.store(i, vo);
    }
}

// ---------------------------------------------------------------- dimensions > 0

// The walk of strided_body (sl_sweep.cuh): one thread per line, fibre and
// chunk; U cells per step, their loads issued before any arithmetic.
template <int K, int Q, int U>
__device__ __forceinline__ void s_walk(const SweepArgs& a, const LineSetup& L, int jb)
{
    constexpr int O = K + 1;
    SMats<K, Q> M;
    M.load(a.tab, L.cls);
    SPtrs<K, Q> P;
    P.init(a, jb, L.base);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    SCell<K, Q> prev;
    P.load(uint32_t(ib) * a.inner, prev);
    s_prepare<K, Q>(M, prev);
    uint32_t i = L.i0;
    if constexpr (U > 1) {
        for (; i + U <= L.i1; i += U) {
            SCell<K, Q> cur[U];
#pragma unroll
            for (int s = 0; s < U; ++s) {
                int32_t x = ia + s;
                x -= x >= N ? N : 0;
                P.load(uint32_t(x) * a.inner, cur[s]);
            }
#pragma unroll
            for (int s = 0; s < U; ++s) s_prepare<K, Q>(M, cur[s]);
#pragma unroll
            for (int s = 0; s < U; ++s) {
                double od[Q];
                float of[O - Q];
                s_combine<K, Q>(M, cur[s], s == 0 ? prev : cur[s - 1], od, of);
                P.store((i + s) * a.inner, od, of);
            }
            prev = cur[U - 1];
            ia += U;
            ia -= ia >= N ? N : 0;
        }
    }
    for (; i < L.i1; ++i) {
        SCell<K, Q> cur;
        P.load(uint32_t(ia) * a.inner, cur);
        s_prepare<K, Q>(M, cur);
        double od[Q];
        float of[O - Q];
        s_combine<K, Q>(M, cur, prev, od, of);
        P.store(i * a.inner, od, of);
        prev = cur;
        ++ia;
        if (ia == N) ia = 0;
    }
}

template <int K, int U>
__device__ __forceinline__ void f_walk(const SweepArgs& a, const LineSetup& L, int jb, const float (&A)[K + 1][K + 1],
                                       const float (&B)[K + 1][K + 1])
{
    constexpr int O = K + 1;
    FPtrs<K> P;
    P.init(a, jb, L.base);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    float prev[O];
    P.load(uint32_t(ib) * a.inner, prev);
    uint32_t i = L.i0;
    if constexpr (U > 1) {
        for (; i + U <= L.i1; i += U) {
            float cur[U][O];
#pragma unroll
            for (int s = 0; s < U; ++s) {
                int32_t x = ia + s;
                x -= x >= N ? N : 0;
                P.load(uint32_t(x) * a.inner, cur[s]);
            }
#pragma unroll
            for (int s = 0; s < U; ++s) {
                float o[O];
                f_combine<K>(A, B, cur[s], s == 0 ? prev : cur[s - 1], o);
                P.store((i + s) * a.inner, o);
            }
#pragma unroll
            for (int l = 0; l < O; ++l) prev[l] = cur[U - 1][l];
            ia += U;
            ia -= ia >= N ? N : 0;
        }
    }
    for (; i < L.i1; ++i) {
        float cur[O], o[O];
        P.load(uint32_t(ia) * a.inner, cur);
        f_combine<K>(A, B, cur, prev, o);
        P.store(i * a.inner, o);
#pragma unroll
        for (int l = 0; l < O; ++l) prev[l] = cur[l];
        ++ia;
        if (ia == N) ia = 0;
    }
}

template <int K, int Q, int U>
__global__ void __launch_bounds__(128) k_split_strided(const SweepArgs a)
{
    const LineSetup L = line_setup_grid(a, 1);
    if (!L.active) return;
    const int jb = fibre_base(L.fbase, K + 1, a.ostride);
    if (__ldg(a.cmap + jb) < 0) {
        s_walk<K, Q, U>(a, L, jb);
    } else {
        SMats<K, Q> M;
        M.load(a.tab, L.cls);
        f_walk<K, U>(a, L, jb, M.a, M.b);
    }
}

template <int K, int Q>
cudaError_t split_shape(const SweepLaunch& L)
{
    const SweepArgs& a = L.args;
    if (L.ft != 1 || !a.cmap) return cudaErrorInvalidValue;
    if (L.unit) {
        if (L.unroll != 1 || L.block < 32 || L.block > 256) return cudaErrorInvalidValue;
        const dim3 grid((a.cells + L.block - 1) / L.block, uint32_t(a.nfib));
        k_split_unit<K, Q><<<grid, L.block, 0, L.stream>>>(a);
        return cudaGetLastError();
    }
    if (L.block < 32 || L.block > 128 || a.chunk == 0) return cudaErrorInvalidValue;
    const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
    const dim3 grid((a.lines + L.block - 1) / L.block, nchunk * uint32_t(a.nfg));
    switch (L.unroll) {
    case 1: k_split_strided<K, Q, 1><<<grid, L.block, 0, L.stream>>>(a); break;
    case 2: k_split_strided<K, Q, 2><<<grid, L.block, 0, L.stream>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_split(const SweepLaunch& L)
{
    const int q = split_q(L.mode);
    if (q == 2 && L.K == 2) return split_shape<2, 2>(L);
    if (q == 2 && L.K == 3) return split_shape<3, 2>(L);
    if (q == 3 && L.K == 3) return split_shape<3, 3>(L);
    return cudaErrorInvalidValue;
}

}  // namespace sl
