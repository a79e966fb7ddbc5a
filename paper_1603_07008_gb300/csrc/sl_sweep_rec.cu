// sl_sweep_rec.cu -- sweeps of the per-cell-scaled BF16/FP16 cell records of
// degree 1 in five and six dimensions, a cell shared by a group of G = R/16
// lanes.  Each lane holds two 16-byte chunks (16 slots) of the record,
// chosen for the sweep dimension M so that both coefficients of every fibre
// it holds are its own: the projection (Sec. II-A update rule) pairs slots J
// and J + 2^M, which lie in one chunk for M <= 2 and in chunks c and c + 2^(M-3)
// otherwise.  A warp's access of one chunk per lane then covers 32/G records
// (a quarter or half of each), instead of one 16-byte piece of 32 different
// records as when a thread holds a whole cell, so the L1 data pipe stops
// limiting the sweep, while the only exchange between lanes is the cell-wide
// maximum of the new scale.  Every result is computed with the same
// operations in the same order as when one thread holds the whole cell, so
// both forms give bit-identical states.
#include "sl_sweep.cuh"

namespace sl {

namespace {

// Chunks of lane h of a group of G lanes for a sweep along dimension M: c0
// (lane-local slots 0..7) and c0 + d (slots 8..15).  For M >= 3 the two
// coefficients of a fibre lie 2^(M-3) chunks apart: d = 2^(M-3) and c0 = h
// with a zero bit inserted at position log2(d).  For M < 3 they lie in one
// chunk, so any chunks will do: c0 = h and d = G, so that each of the two
// loads and stores of a group covers G neighbouring chunks (half a record).
template <int M, int G>
struct LgChunks {
    static constexpr int b = M > 3 ? M - 3 : 0;
    static constexpr int d = M < 3 ? G : 1 << b;
    __device__ __forceinline__ static int c0(int h)
    {
        return M < 3 ? h : ((h >> b) << (b + 1)) | (h & ((1 << b) - 1));
    }
};

// Lane-local slot stride between the two coefficients of a fibre along M.
template <int M>
__host__ __device__ constexpr int lg_stride()
{
    return M < 3 ? (1 << M) : 8;
}

// This lane's two source chunks of one cell with the cell's scale and mean.
struct LgRow {
    uint4 q0, q1;
    float s;
    double m;
};

template <int R>
__device__ __forceinline__ LgRow lg_load(const SweepArgs& a, uint32_t cell, int c0, int d)
{
    const uint4* p = static_cast<const uint4*>(a.src.hi) + size_t(cell) * (R / 8);
    LgRow r;
    r.q0 = __ldg(p + c0);
    r.q1 = __ldg(p + c0 + d);
    r.s = __ldg(a.src.scale + cell);
    r.m = __ldg(a.src.mean + cell);
    return r;
}

__device__ __forceinline__ uint32_t lg_word(const uint4& q, int w)
{
    return w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
}

// Lane-local slot q (0..15) times the cell's scale.
template <int MODE>
__device__ __forceinline__ float lg_val(const LgRow& r, int q)
{
    const uint32_t w = lg_word(q < 8 ? r.q0 : r.q1, (q & 7) / 2);
    return dec16<MODE>((q & 1) ? (w >> 16) : (w & 0xffffu)) * r.s;
}

// Row j of one fibre (a0, a1 from source cell a = i - sigma, b0, b1 from
// b = i - sigma - 1), in the order of the one-thread-per-cell form.
__device__ __forceinline__ float lg_row(float A0, float B0, float A1, float B1, float a0, float b0,
                                       float a1, float b1)
{
    float acc = 0.0f;
    acc = fmaf(A0, a0, acc);
    acc = fmaf(B0, b0, acc);
    acc = fmaf(A1, a1, acc);
    acc = fmaf(B1, b1, acc);
    return acc;
}

// New values of this lane's 16 slots of a target cell; om (the new mean) is
// valid on lane 0 of the group, which holds the mean's fibre (slots 0 and
// 2^M of the record, lane-local 0 and st).
template <int MODE, int M>
__device__ __forceinline__ void lg_combine(const Mats<1, MODE>& T, const LgRow& ra, const LgRow& rb, int h,
                                           float (&out)[16], double& om)
{
    constexpr int st = lg_stride<M>();
    om = 0.0;
#pragma unroll
    for (int q0 = 0; q0 < 16; ++q0) {
        if (q0 & st) continue;
        const int q1 = q0 | st;
        const float a0 = lg_val<MODE>(ra, q0), a1 = lg_val<MODE>(ra, q1);
        const float b0 = lg_val<MODE>(rb, q0), b1 = lg_val<MODE>(rb, q1);
        if (q0 == 0 && h == 0) {
            // the mean's fibre: FP64 conservation form with the per-cell FP32
            // sums G(c) = fl32(A_01 c_1), and its row 1
            float ga = 0.0f, gb = 0.0f;
            ga = fmaf(T.a[0][1], a1, ga);
            gb = fmaf(T.a[0][1], b1, gb);
            float dm;
            // FP64 subtraction: these kernels keep the integer pipe busier than
            // the FP64 pipe (the integer-pipe difference measured 5% slower)
            om = mean_row_lp<CV_FP64SUB>(T.alpha, ra.m, rb.m, ga, gb, dm);
            float acc = T.a[1][0] * dm;
            acc = fmaf(T.a[1][1], a1, acc);
            acc = fmaf(T.b[1][1], b1, acc);
            out[q0] = 0.0f;
            out[q1] = acc;
        } else {
            out[q0] = lg_row(T.a[0][0], T.b[0][0], T.a[0][1], T.b[0][1], a0, b0, a1, b1);
            out[q1] = lg_row(T.a[1][0], T.b[1][0], T.a[1][1], T.b[1][1], a0, b0, a1, b1);
        }
    }
}

// Scale by the cell-wide maximum, encode and store this lane's chunks; lane 0
// of the group also stores the mean and the scale.
template <int MODE, int G, int R>
__device__ __forceinline__ void lg_store(const SweepArgs& a, uint32_t c, int h, int c0, int d, unsigned gmask,
                                         const float (&out)[16], double om)
{
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fabsf(out[q]));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(gmask, mx, o));
    float sc, inv;
    pow2_scale(mx, sc, inv);
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = enc16x2<MODE>(out[2 * k] * inv, out[2 * k + 1] * inv);
    if (h == 0) w[0] &= 0xffff0000u;   // slot 0 (the mean's) stays zero
    uint4* p = static_cast<uint4*>(a.dst.hi) + size_t(c) * (R / 8);
    p[c0] = make_uint4(w[0], w[1], w[2], w[3]);
    p[c0 + d] = make_uint4(w[4], w[5], w[6], w[7]);
    if (h == 0) {
        a.dst.scale[c] = sc;
        a.dst.mean[c] = om;
    }
}

// One group of G lanes per line (and chunk of the line, blockIdx.y), walking
// its target cells U per step with the loads of a step issued first.  All
// lanes of a group share the line, so they stay converged for the shuffles
// of the cell maximum.
template <int MODE, int D, int M, int U>
__global__ void __launch_bounds__(256) k_sweep_rec_lg(const SweepArgs a)
{
    constexpr int R = RecShape<1, D>::R;
    constexpr int G = R / 16;
    using C = LgChunks<M, G>;
    const uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int h = int(threadIdx.x) & (G - 1);
    const int lane = int(threadIdx.x) & 31;
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    const int c0 = C::c0(h);
    const uint64_t line = t / G;
    if (line >= a.lines) return;
    const LineSetup L = line_setup(a, uint32_t(line), 0, blockIdx.y, 1);
    if (!L.active) return;
    Mats<1, MODE> T;
    T.template load<true>(a.tab, L.cls);
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(L.i0) - L.sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    LgRow prev = lg_load<R>(a, L.base + uint32_t(ib) * a.inner, c0, C::d);
    auto emit = [&](uint32_t i, const LgRow& cur, const LgRow& pr) {
        float out[16];
        double om;
        lg_combine<MODE, M>(T, cur, pr, h, out, om);
        lg_store<MODE, G, R>(a, L.base + i * a.inner, h, c0, C::d, gmask, out, om);
    };
    uint32_t i = L.i0;
    if constexpr (U > 1) {
        for (; i + U <= L.i1; i += U) {
            LgRow cur[U];
#pragma unroll
            for (int s = 0; s < U; ++s) {
                int32_t x = ia + s;
                x -= x >= N ? N : 0;
                cur[s] = lg_load<R>(a, L.base + uint32_t(x) * a.inner, c0, C::d);
            }
#pragma unroll
            for (int s = 0; s < U; ++s) emit(i + s, cur[s], s == 0 ? prev : cur[s - 1]);
            prev = cur[U - 1];
            ia += U;
            ia -= ia >= N ? N : 0;
        }
    }
    for (; i < L.i1; ++i) {
        const LgRow cur = lg_load<R>(a, L.base + uint32_t(ia) * a.inner, c0, C::d);
        emit(i, cur, prev);
        prev = cur;
        ++ia;
        if (ia == N) ia = 0;
    }
}

template <int MODE, int D, int M>
cudaError_t lg_walk(const SweepLaunch& L, dim3 grid)
{
    switch (L.unroll) {
    case 1: k_sweep_rec_lg<MODE, D, M, 1><<<grid, L.block, 0, L.stream>>>(L.args); break;
    case 2: k_sweep_rec_lg<MODE, D, M, 2><<<grid, L.block, 0, L.stream>>>(L.args); break;
    case 4: k_sweep_rec_lg<MODE, D, M, 4><<<grid, L.block, 0, L.stream>>>(L.args); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int MODE, int D>
cudaError_t lg_dims(const SweepLaunch& L)
{
    constexpr int G = RecShape<1, D>::R / 16;
    const SweepArgs& a = L.args;
    if (L.ndim != D || L.rec != RecShape<1, D>::R || L.dim < 0 || L.dim >= D || a.chunk == 0 ||
        L.block % 32 != 0 || L.block < 32 || L.block > 256)
        return cudaErrorInvalidValue;
    const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
    const uint64_t threads = uint64_t(a.lines) * G;
    const dim3 grid(uint32_t((threads + L.block - 1) / L.block), nchunk);
    switch (L.dim) {
    case 0: return lg_walk<MODE, D, 0>(L, grid);
    case 1: return lg_walk<MODE, D, 1>(L, grid);
    case 2: return lg_walk<MODE, D, 2>(L, grid);
    case 3: return lg_walk<MODE, D, 3>(L, grid);
    case 4: return lg_walk<MODE, D, 4>(L, grid);
    case 5:
        if constexpr (D > 5) return lg_walk<MODE, D, 5>(L, grid);
        break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sweep_rec_lanes(const SweepLaunch& L)
{
    if (L.K != 1) return cudaErrorInvalidValue;
    if (L.mode == M_BF16) {
        if (L.ndim == 6) return lg_dims<M_BF16, 6>(L);
        if (L.ndim == 5) return lg_dims<M_BF16, 5>(L);
    }
    if (L.mode == M_FP16) {
        if (L.ndim == 6) return lg_dims<M_FP16, 6>(L);
        if (L.ndim == 5) return lg_dims<M_FP16, 5>(L);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sl
