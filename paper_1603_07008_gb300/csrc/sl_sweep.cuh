// sl_sweep.cuh -- the sLdG projection-sweep kernels for sm_103a.
//
// Every target cell i of a line gets, for every fibre of coefficients that
// varies only in the sweep dimension's index j,
//     c'_j = sum_l A_jl(alpha) c_{i-sigma, l} + B_jl(alpha) c_{i-sigma-1, l}
// (Sec. II-A, update rule).  The work is one load and one store per degree of
// freedom against 4o-1 flops (Sec. II-A), so the kernels are HBM-bound on
// CUDA cores; no tensor cores are involved.
//
// Two launch shapes:
//   * unit stride (sweep along dimension 0): one thread per target cell,
//     consecutive threads on consecutive cells of a line, so every plane
//     access of a warp is one coalesced segment.  The second source cell
//     (i-sigma-1) is the first source cell of the neighbouring lane, so its
//     load is served by L1.
//   * strided (sweep along dimension m > 0): one thread per line (consecutive
//     threads on consecutive inner indices, again coalesced), walking along
//     the sweep dimension and keeping the previous source cell in registers,
//     so every source value is read from HBM once.
//
// Precision (split store): the cell mean c_{0..0} lives in an FP64 plane.
// Its row is computed in FP64 in the form
//     c'_0 = a_0 + alpha (b_0 - a_0) + sum_{l>=1} A_0l (a_l - b_l),
// which uses the exact identities A_00 + B_00 = 1 and B_0l = -A_0l (l >= 1)
// of the projection, so the sum over a line telescopes and mass is conserved
// to FP64 rounding (Sec. II-A, III-A).  The other rows of the mean's fibre
// take the l = 0 term as the FP64 difference A_j0 (a_0 - b_0) (B_j0 = -A_j0),
// rounded once to the arithmetic type; everything else is computed in the
// arithmetic type of the mode (FP64, or FP32 for the mixed modes).
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
};
template <>
struct St<M_F32> {
    using T = float;
    using R = float;
    static constexpr bool scaled = false;
};
template <>
struct St<M_BF16> {
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool scaled = true;
};
template <>
struct St<M_FP16> {
    using T = __half;
    using R = float;
    static constexpr bool scaled = true;
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

template <int K, int MODE, int FT>
struct CellVals {
    typename St<MODE>::R v[FT][K + 1];   // v[u][0] of fibre 0 is unused: the mean is in m
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

    __device__ __forceinline__ void load(const ShiftTable& t, uint32_t cls, bool need_f0)
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
        if (need_f0) {
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

// Load the FT fibres (base coefficient indices jb[u], stride ostride along the
// fibre) of cell c.  Fibre index f = fbase + u; fibres >= nfib are skipped.
template <int K, int MODE, int FT>
__device__ __forceinline__ void load_cell(const Planes& p, int64_t pstride, uint32_t c,
                                          const int (&jb)[FT], int ostride, int fbase, int nfib,
                                          CellVals<K, MODE, FT>& cv)
{
    using T = typename St<MODE>::T;
    constexpr int O = K + 1;
    float s = 1.0f;
    if constexpr (St<MODE>::scaled) s = __ldg(p.scale + c);
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        if (fbase + u >= nfib) break;
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int J = jb[u] + l * ostride;
            if (J == 0) {
                cv.m = __ldg(p.mean + c);
                cv.v[u][0] = 0;
            } else {
                auto raw = ld_raw(plane_ptr<T>(p.hi, pstride, J) + c);
                if constexpr (St<MODE>::scaled) raw *= s;
                cv.v[u][l] = raw;
            }
        }
    }
}

// New values of one target cell from its source cells a (= i - sigma) and
// b (= i - sigma - 1).
template <int K, int MODE, int FT>
__device__ __forceinline__ void combine(const Mats<K, MODE>& M, const CellVals<K, MODE, FT>& a,
                                        const CellVals<K, MODE, FT>& b, int fbase, int nfib,
                                        CellVals<K, MODE, FT>& out)
{
    using R = typename St<MODE>::R;
    constexpr int O = K + 1;
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        if (fbase + u >= nfib) break;
        if (fbase + u == 0) {
            double d = a.m + M.alpha * (b.m - a.m);
#pragma unroll
            for (int l = 1; l < O; ++l) d += M.a0[l] * (double(a.v[u][l]) - double(b.v[u][l]));
            out.m = d;
            out.v[u][0] = 0;
            const double dm = a.m - b.m;
#pragma unroll
            for (int j = 1; j < O; ++j) {
                R acc = R(M.aj0[j] * dm);
#pragma unroll
                for (int l = 1; l < O; ++l) {
                    acc = fma(M.a[j][l], a.v[u][l], acc);
                    acc = fma(M.b[j][l], b.v[u][l], acc);
                }
                out.v[u][j] = acc;
            }
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

template <int K, int MODE, int FT>
__device__ __forceinline__ void store_cell(const Planes& p, int64_t pstride, uint32_t c,
                                           const int (&jb)[FT], int ostride, int fbase, int nfib,
                                           const CellVals<K, MODE, FT>& cv)
{
    using T = typename St<MODE>::T;
    using R = typename St<MODE>::R;
    constexpr int O = K + 1;
    R inv = R(1);
    if constexpr (St<MODE>::scaled) {
        // one scale for the whole cell: the group holds every fibre
        float mx = 0.0f;
#pragma unroll
        for (int u = 0; u < FT; ++u) {
            if (fbase + u >= nfib) break;
#pragma unroll
            for (int l = 0; l < O; ++l) mx = fmaxf(mx, fabsf(cv.v[u][l]));
        }
        float s;
        pow2_scale(mx, s, inv);
        p.scale[c] = s;
    }
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        if (fbase + u >= nfib) break;
#pragma unroll
        for (int l = 0; l < O; ++l) {
            const int J = jb[u] + l * ostride;
            if (J == 0) {
                p.mean[c] = cv.m;
            } else {
                R v = cv.v[u][l];
                if constexpr (St<MODE>::scaled) v *= inv;
                st_raw(plane_ptr_w<T>(p.hi, pstride, J) + c, v);
            }
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

// Sweep along dimension 0: one thread per target cell (and fibre group
// blockIdx.y).  For dimension 0 the fibre stride is 1, so the fibre with
// index f holds coefficients f*o .. f*o + k.
template <int K, int MODE, int FT>
__global__ void __launch_bounds__(256) k_sweep_unit(const SweepArgs a)
{
    constexpr int O = K + 1;
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.cells) return;
    const int fbase = blockIdx.y * FT;
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

    int jb[FT];
#pragma unroll
    for (int u = 0; u < FT; ++u) jb[u] = (fbase + u) * O;

    Mats<K, MODE> M;
    M.load(a.tab, cls, fbase == 0);
    CellVals<K, MODE, FT> va, vb, out;
    load_cell<K, MODE, FT>(a.src, a.pstride, ca, jb, 1, fbase, a.nfib, va);
    load_cell<K, MODE, FT>(a.src, a.pstride, cb, jb, 1, fbase, a.nfib, vb);
    combine<K, MODE, FT>(M, va, vb, fbase, a.nfib, out);
    store_cell<K, MODE, FT>(a.dst, a.pstride, c, jb, 1, fbase, a.nfib, out);
}

// ---------------------------------------------------------------- strided

// Sweep along dimension m > 0: one thread per line (and fibre group and
// chunk of the line, blockIdx.y = chunk * nfg + group).  The thread walks the
// target cells i0 .. i1-1 of its chunk, U cells per step: it issues the loads
// of the U new source cells first, then computes and stores the U targets.
// The source cell i - sigma of one target is the source cell i - sigma - 1
// of the next, so every source value is loaded once.
template <int K, int MODE, int FT, int U>
__global__ void __launch_bounds__(128) k_sweep_strided(const SweepArgs a)
{
    constexpr int O = K + 1;
    const uint32_t line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= a.lines) return;
    const uint32_t grp = blockIdx.y % uint32_t(a.nfg);
    const uint32_t chunk = blockIdx.y / uint32_t(a.nfg);
    const int fbase = int(grp) * FT;
    const uint32_t outer = a.fdInner.div(line);
    const uint32_t inn = line - outer * a.inner;
    const uint32_t base = outer * a.N * a.inner + inn;
    const uint32_t cls = shift_class(a, inn, outer);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    const uint32_t i0 = chunk * a.chunk;
    uint32_t i1 = i0 + a.chunk;
    if (i1 > a.N) i1 = a.N;
    if (i0 >= i1) return;

    int jb[FT];
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        const int f = fbase + u;
        jb[u] = (f / a.ostride) * (O * a.ostride) + (f % a.ostride);
    }

    Mats<K, MODE> M;
    M.load(a.tab, cls, fbase == 0);
    int32_t ia = int32_t(i0) - sig;
    ia += ia < 0 ? int32_t(a.N) : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? int32_t(a.N) : 0;
    const int32_t N = int32_t(a.N);

    CellVals<K, MODE, FT> prev;
    load_cell<K, MODE, FT>(a.src, a.pstride, base + uint32_t(ib) * a.inner, jb, a.ostride, fbase,
                           a.nfib, prev);
    uint32_t i = i0;
    if constexpr (U > 1) {
        for (; i + U <= i1; i += U) {
            CellVals<K, MODE, FT> cur[U];
#pragma unroll
            for (int s = 0; s < U; ++s) {
                int32_t x = ia + s;
                x -= x >= N ? N : 0;
                load_cell<K, MODE, FT>(a.src, a.pstride, base + uint32_t(x) * a.inner, jb,
                                       a.ostride, fbase, a.nfib, cur[s]);
            }
#pragma unroll
            for (int s = 0; s < U; ++s) {
                CellVals<K, MODE, FT> out;
                combine<K, MODE, FT>(M, cur[s], s == 0 ? prev : cur[s - 1], fbase, a.nfib, out);
                store_cell<K, MODE, FT>(a.dst, a.pstride, base + (i + s) * a.inner, jb, a.ostride,
                                        fbase, a.nfib, out);
            }
            prev = cur[U - 1];
            ia += U;
            ia -= ia >= N ? N : 0;
        }
    }
    for (; i < i1; ++i) {
        CellVals<K, MODE, FT> cur, out;
        load_cell<K, MODE, FT>(a.src, a.pstride, base + uint32_t(ia) * a.inner, jb, a.ostride,
                               fbase, a.nfib, cur);
        combine<K, MODE, FT>(M, cur, prev, fbase, a.nfib, out);
        store_cell<K, MODE, FT>(a.dst, a.pstride, base + i * a.inner, jb, a.ostride, fbase, a.nfib,
                                out);
        prev = cur;
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

// Dynamic shared memory of k_sweep_strided_async for `block` threads.
template <int K, int MODE, int FT, int P>
constexpr size_t strided_async_smem(int block)
{
    return size_t(P + 1) * size_t(block) * (8 + size_t(FT) * (K + 1) * sizeof(typename St<MODE>::T));
}

// Same walk as k_sweep_strided, but the source rows are fetched P rows ahead
// with cp.async into a per-thread ring of P+1 row slots in shared memory, so
// every thread keeps P rows of loads in flight while it computes.  A thread
// only reads slots it filled itself (cp.async.wait_group makes them visible
// to the issuing thread), so no block barrier is needed; a slot is refilled
// one iteration after it was read and its values were used.
template <int K, int MODE, int FT, int P>
__global__ void __launch_bounds__(128) k_sweep_strided_async(const SweepArgs a)
{
    static_assert(!St<MODE>::scaled, "cp.async ring needs 4- or 8-byte elements");
    using T = typename St<MODE>::T;
    constexpr int O = K + 1;
    constexpr int S = P + 1;
    constexpr int V = FT * O;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t nthr = blockDim.x;
    const uint32_t tid = threadIdx.x;
    double* sm_mean = reinterpret_cast<double*>(smem_raw);
    T* sm_val = reinterpret_cast<T*>(smem_raw + size_t(S) * nthr * 8);

    const uint32_t line = blockIdx.x * blockDim.x + tid;
    if (line >= a.lines) return;
    const uint32_t grp = blockIdx.y % uint32_t(a.nfg);
    const uint32_t chunk = blockIdx.y / uint32_t(a.nfg);
    const int fbase = int(grp) * FT;
    const uint32_t outer = a.fdInner.div(line);
    const uint32_t inn = line - outer * a.inner;
    const uint32_t base = outer * a.N * a.inner + inn;
    const uint32_t cls = shift_class(a, inn, outer);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    const uint32_t i0 = chunk * a.chunk;
    uint32_t i1 = i0 + a.chunk;
    if (i1 > a.N) i1 = a.N;
    if (i0 >= i1) return;
    const int32_t N = int32_t(a.N);

    int jb[FT];
#pragma unroll
    for (int u = 0; u < FT; ++u) {
        const int f = fbase + u;
        jb[u] = (f / a.ostride) * (O * a.ostride) + (f % a.ostride);
    }
    Mats<K, MODE> M;
    M.load(a.tab, cls, fbase == 0);

    // rows in consumption order: row 0 is source cell i0-sigma-1, row q >= 1
    // the source cell i0+q-1-sigma of target i0+q-1; all periodic in N
    const int nrows = int(i1 - i0) + 1;
    int32_t frow = int32_t(i0) - sig - 1;
    frow += frow < 0 ? N : 0;
    frow += frow < 0 ? N : 0;

    auto fetch = [&](int slot, uint32_t cell) {
#pragma unroll
        for (int u = 0; u < FT; ++u) {
            if (fbase + u >= a.nfib) break;
#pragma unroll
            for (int l = 0; l < O; ++l) {
                const int J = jb[u] + l * a.ostride;
                if (J == 0)
                    cp_async<8>(sm_mean + size_t(slot) * nthr + tid, a.src.mean + cell);
                else
                    cp_async<sizeof(T)>(sm_val + (size_t(slot) * V + u * O + l) * nthr + tid,
                                        plane_ptr<T>(a.src.hi, a.pstride, J) + cell);
            }
        }
    };
    auto read = [&](int slot, CellVals<K, MODE, FT>& cv) {
#pragma unroll
        for (int u = 0; u < FT; ++u) {
            if (fbase + u >= a.nfib) break;
#pragma unroll
            for (int l = 0; l < O; ++l) {
                const int J = jb[u] + l * a.ostride;
                if (J == 0) {
                    cv.m = sm_mean[size_t(slot) * nthr + tid];
                    cv.v[u][0] = 0;
                } else {
                    cv.v[u][l] = sm_val[(size_t(slot) * V + u * O + l) * nthr + tid];
                }
            }
        }
    };

#pragma unroll
    for (int q = 0; q < P; ++q) {
        if (q < nrows) {
            fetch(q, base + uint32_t(frow) * a.inner);
            ++frow;
            frow -= frow >= N ? N : 0;
        }
        cp_async_commit();
    }
    CellVals<K, MODE, FT> prev, cur;
    int slot = 0;           // slot of row q
    int rslot = P;          // slot that row q + P goes to (= slot of row q - 1)
    for (int q = 0; q < nrows; ++q) {
        cp_async_wait<P - 1>();
        read(slot, cur);
        if (q + P < nrows) {
            fetch(rslot, base + uint32_t(frow) * a.inner);
            ++frow;
            frow -= frow >= N ? N : 0;
        }
        cp_async_commit();
        if (q > 0) {
            CellVals<K, MODE, FT> out;
            combine<K, MODE, FT>(M, cur, prev, fbase, a.nfib, out);
            store_cell<K, MODE, FT>(a.dst, a.pstride, base + (i0 + uint32_t(q) - 1) * a.inner, jb,
                                    a.ostride, fbase, a.nfib, out);
        }
        prev = cur;
        rslot = slot;
        slot = slot + 1 == S ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

}  // namespace sl
