// sl_nodal.cu -- the x-sweep with the velocity taken at the Gauss-Legendre
// nodes of every v-cell ("nodal in v").
//
// In several dimensions the x-advection v d_x f (Sec. II, splitting) has a
// velocity that varies inside a v-cell.  The plain sweep takes one velocity
// per v-cell (its centre).  Here, for the x-dimension m paired with the
// v-dimension p, the coefficients of a cell are evaluated at the o nodes
// eta_q of the v-cell, U_q(l) = sum_jv c_{l,jv} P_jv(eta_q); each node is
// swept along x with its own shift s_{j,q} = v(eta_q) tau / h_m (the update
// rule of Sec. II-A), v(eta) = lo_p + (j + 1/2 + eta / 2) h_p; and the new
// coefficients are the o-point Gauss rule of the new nodal values,
// c'_{jx,jv} = (2 jv + 1) / 2 sum_q w_q P_jv(eta_q) U'_q(jx) (eq. (cj) along v).
//
// One thread per target cell and group of fibres of coefficients varying in
// (j_m, j_p), for any x-dimension: consecutive threads take consecutive
// cells, so every plane access is coalesced; the source cells of a node are
// the target's line shifted by sigma_q, and the nodes' source cells, equal
// for most cells (the node shifts of one v-cell differ by h_p tau / h_m),
// are loaded once per distinct sigma.  Along x-dimensions > 0 the FP32
// fibres of the mixed store take a run of consecutive targets per thread
// instead, and each source cell's node values are formed once per run.
//
// Stores: FP64, and the mixed FP32 store.  In the mixed store the fibre of
// the cell mean keeps everything that reaches the mean in FP64: the node
// value of row 0, U_q(0) = c_{0,0} + sum_{jv>=1} c_{0,jv} P_jv(eta_q), row 0
// of each node in the conservation form of the plain sweep (with the per-cell
// FP32 sums G_q(c) = sum_{l>=1} fl32(A_0l U_q(l))), and c'_{0,0} =
// sum_q w'_q U'_q(0), where the weights w'_q = w_q / 2 are rounded so that
// they sum to exactly one.  The node values enter c'_{0,jv} (jv >= 1) as FP32
// differences U'_q(0) - c'_{0,0} (the Gauss rule maps a constant to zero for
// jv >= 1).  Everything else is FP32.
#include "sl_sweep.cuh"
#include "sl_nodal.h"

#include <cmath>

namespace sl {

namespace {

// FP32 fibres per thread of the mixed store's nodal sweep (its walk form holds
// the raw values and node values of two source cells per fibre; with one
// target per thread two fibres per thread measured 17% faster than one at
// k = 2).
__host__ __device__ constexpr int nodal_ftw(int K) { return K == 0 ? 4 : K == 3 ? 1 : 2; }

// Base coefficient index of 2D fibre g: its digits along the dimensions other
// than x and v, in increasing dimension order.
template <int O>
__device__ __forceinline__ int nodal_fibre_base(const NodalArgs& a, int g)
{
    int base = 0, stride = 1;
    for (int m = 0; m < a.ndim; ++m) {
        if (m != a.xdim && m != a.vdim) {
            base += (g % O) * stride;
            g /= O;
        }
        stride *= O;
    }
    return base;
}

// One class record of the node table (A then B, padded to 16 bytes), read
// with 16-byte vector loads.
template <int O>
__device__ __forceinline__ void load_ab(const ShiftTable& t, uint32_t cls, float (&A)[O][O], float (&B)[O][O])
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
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            A[x][l] = v[x * O + l];
            B[x][l] = v[O * O + x * O + l];
        }
}
template <int O>
__device__ __forceinline__ void load_ab(const ShiftTable& t, uint32_t cls, double (&A)[O][O], double (&B)[O][O])
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
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int l = 0; l < O; ++l) {
            A[x][l] = v[x * O + l];
            B[x][l] = v[O * O + x * O + l];
        }
}

template <typename T>
__device__ __forceinline__ const T* coef_plane(const Planes& p, int64_t ps, int J)
{
    return static_cast<const T*>(p.hi) + int64_t(J - 1) * ps;
}

// Coefficient J >= 1 of cell `cell` in the FP32 block of the source and the
// destination (OFF32: the block's base plus a 32-bit element offset).
template <bool OFF32>
__device__ __forceinline__ float ld_hi(const NodalArgs& a, int J, uint32_t cell)
{
    if constexpr (OFF32)
        return __ldg(static_cast<const float*>(a.src.hi) + (uint32_t(J - 1) * uint32_t(a.pstride) + cell));
    else
        return __ldg(coef_plane<float>(a.src, a.pstride, J) + cell);
}
template <bool OFF32>
__device__ __forceinline__ void st_hi(const NodalArgs& a, int J, uint32_t cell, float v)
{
    if constexpr (OFF32)
        static_cast<float*>(a.dst.hi)[uint32_t(J - 1) * uint32_t(a.pstride) + cell] = v;
    else
        static_cast<float*>(a.dst.hi)[int64_t(J - 1) * a.pstride + cell] = v;
}

// Every fibre of the FP64 store (R = double), the whole computation in FP64;
// for R = float the same steps in FP32 (the mixed store's FP32 fibres take
// the grouped form, nodal_fp32_group).
template <int K, typename R>
__device__ __forceinline__ void nodal_plain(const NodalArgs& a, uint32_t c, uint32_t i, uint32_t line0, uint32_t j,
                                            int base)
{
    constexpr int O = K + 1;
    const bool has_mean = sizeof(R) == 8 && base == 0;   // the FP64 store's J = 0 is the mean plane
    R acc[O][O];
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) acc[x][v] = R(0);
    R va[O][O], vb[O][O];
    const int32_t N = int32_t(a.N);
    auto load = [&](int32_t sig) {
        int32_t ia = int32_t(i) - sig;
        ia += ia < 0 ? N : 0;
        int32_t ib = ia - 1;
        ib += ib < 0 ? N : 0;
        const uint32_t ca = line0 + uint32_t(ia) * a.inner_x, cb = line0 + uint32_t(ib) * a.inner_x;
#pragma unroll
        for (int l = 0; l < O; ++l)
#pragma unroll
            for (int v = 0; v < O; ++v) {
                const int J = base + l * a.ostride + v * a.vstride;
                if (has_mean && J == 0) {
                    va[l][v] = R(__ldg(a.src.mean + ca));
                    vb[l][v] = R(__ldg(a.src.mean + cb));
                } else {
                    const R* p = coef_plane<R>(a.src, a.pstride, J);
                    va[l][v] = __ldg(p + ca);
                    vb[l][v] = __ldg(p + cb);
                }
            }
    };
    // the nodes of a v-cell nearly always share sigma: then the sources are
    // loaded once, else once per node
    int32_t sg[O];
    bool same = true;
#pragma unroll
    for (int q = 0; q < O; ++q) {
        sg[q] = __ldg(a.tab.sigma + j * O + q);
        same = same && sg[q] == sg[0];
    }
    if (same) load(sg[0]);
#pragma unroll
    for (int q = 0; q < O; ++q) {
        const uint32_t cls = j * O + q;
        if (!same) load(sg[q]);
        R A[O][O], B[O][O];
        load_ab<O>(a.tab, cls, A, B);
        R ua[O], ub[O];
#pragma unroll
        for (int l = 0; l < O; ++l) {
            R sa = R(0), sb = R(0);
#pragma unroll
            for (int v = 0; v < O; ++v) {
                const R e = sizeof(R) == 8 ? R(a.eval64[q][v]) : R(a.eval32[q][v]);
                sa = fma(va[l][v], e, sa);
                sb = fma(vb[l][v], e, sb);
            }
            ua[l] = sa;
            ub[l] = sb;
        }
        R up[O];
        if constexpr (sizeof(R) == 8) {
            // row 0 in the conservation form; the l = 0 term of the other
            // rows from the difference of the sources
            const double t = ub[0] - ua[0];
            double r = fma(__ldg(a.tab.alpha + cls), t, ua[0]);
#pragma unroll
            for (int l = 1; l < O; ++l) r = fma(A[0][l], ua[l] - ub[l], r);
            up[0] = r;
#pragma unroll
            for (int x = 1; x < O; ++x) {
                double s = -A[x][0] * t;
#pragma unroll
                for (int l = 1; l < O; ++l) {
                    s = fma(A[x][l], ua[l], s);
                    s = fma(B[x][l], ub[l], s);
                }
                up[x] = s;
            }
        } else {
#pragma unroll
            for (int x = 0; x < O; ++x) {
                R s = R(0);
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    s = fma(A[x][l], ua[l], s);
                    s = fma(B[x][l], ub[l], s);
                }
                up[x] = s;
            }
        }
#pragma unroll
        for (int x = 0; x < O; ++x)
#pragma unroll
            for (int v = 0; v < O; ++v) {
                const R bw = sizeof(R) == 8 ? R(a.back64[v][q]) : R(a.back32[v][q]);
                acc[x][v] = fma(bw, up[x], acc[x][v]);
            }
    }
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) {
            const int J = base + x * a.ostride + v * a.vstride;
            if (has_mean && J == 0)
                a.dst.mean[c] = double(acc[x][v]);
            else
                static_cast<R*>(a.dst.hi)[int64_t(J - 1) * a.pstride + c] = acc[x][v];
        }
}

// FT FP32 fibres of the mixed store in one thread (bases jb[u]): the thread's
// index arithmetic, sigma and the node tables serve all of them.  OFF32: the
// FP32 block has fewer than 2^31 elements, so every address is the block's
// base plus a 32-bit element offset.
template <int K, int FT, bool OFF32>
__device__ __forceinline__ void nodal_fp32_group(const NodalArgs& a, uint32_t c, uint32_t i, uint32_t line0,
                                                 uint32_t j, const int (&jb)[FT])
{
    constexpr int O = K + 1;
    const int32_t N = int32_t(a.N);
    float va[FT][O][O], vb[FT][O][O];
    auto load = [&](int32_t sig) {
        int32_t ia = int32_t(i) - sig;
        ia += ia < 0 ? N : 0;
        int32_t ib = ia - 1;
        ib += ib < 0 ? N : 0;
        const uint32_t ca = line0 + uint32_t(ia) * a.inner_x, cb = line0 + uint32_t(ib) * a.inner_x;
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l)
#pragma unroll
                for (int v = 0; v < O; ++v) {
                    const int J = jb[u] + l * a.ostride + v * a.vstride;
                    if constexpr (OFF32) {
                        const float* h = static_cast<const float*>(a.src.hi);
                        const uint32_t po = uint32_t(J - 1) * uint32_t(a.pstride);
                        va[u][l][v] = __ldg(h + (po + ca));
                        vb[u][l][v] = __ldg(h + (po + cb));
                    } else {
                        const float* p = coef_plane<float>(a.src, a.pstride, J);
                        va[u][l][v] = __ldg(p + ca);
                        vb[u][l][v] = __ldg(p + cb);
                    }
                }
    };
    int32_t sg[O];
    bool same = true;
#pragma unroll
    for (int q = 0; q < O; ++q) {
        sg[q] = __ldg(a.tab.sigma + j * O + q);
        same = same && sg[q] == sg[0];
    }
    if (same) load(sg[0]);
    float acc[FT][O][O];
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int x = 0; x < O; ++x)
#pragma unroll
            for (int v = 0; v < O; ++v) acc[u][x][v] = 0.0f;
#pragma unroll
    for (int q = 0; q < O; ++q) {
        if (!same) load(sg[q]);
        float A[O][O], B[O][O];
        load_ab<O>(a.tab, j * O + q, A, B);
#pragma unroll
        for (int u = 0; u < FT; ++u) {
            float ua[O], ub[O];
#pragma unroll
            for (int l = 0; l < O; ++l) {
                float sa = 0.0f, sb = 0.0f;
#pragma unroll
                for (int v = 0; v < O; ++v) {
                    sa = fmaf(va[u][l][v], a.eval32[q][v], sa);
                    sb = fmaf(vb[u][l][v], a.eval32[q][v], sb);
                }
                ua[l] = sa;
                ub[l] = sb;
            }
#pragma unroll
            for (int x = 0; x < O; ++x) {
                float s = 0.0f;
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    s = fmaf(A[x][l], ua[l], s);
                    s = fmaf(B[x][l], ub[l], s);
                }
#pragma unroll
                for (int v = 0; v < O; ++v) acc[u][x][v] = fmaf(a.back32[v][q], s, acc[u][x][v]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < FT; ++u)
#pragma unroll
        for (int x = 0; x < O; ++x)
#pragma unroll
            for (int v = 0; v < O; ++v) {
                const int J = jb[u] + x * a.ostride + v * a.vstride;
                if constexpr (OFF32)
                    static_cast<float*>(a.dst.hi)[uint32_t(J - 1) * uint32_t(a.pstride) + c] = acc[u][x][v];
                else
                    static_cast<float*>(a.dst.hi)[int64_t(J - 1) * a.pstride + c] = acc[u][x][v];
            }
}

// Targets per run of the walk form: kernel part 4 (x-dimensions > 0, the
// lanes of a warp on neighbouring x-lines) and part 5 (x-dimension 0, the
// lanes on neighbouring runs of one line, so two cells apart).
constexpr int kNodalRun = 4;
constexpr int kNodalRun0 = 2;

// The FT FP32 fibres of nodal_fp32_group for the run of cnt <= RUN
// consecutive targets i0 .. i0 + cnt - 1 of one x-line whose v-cell j has one
// sigma for all its nodes.  Target i reads the source cells a = i - sigma and
// b = i - sigma - 1, and the a of target i is the b of target i + 1, so the
// node values U_q(l) = sum_v c_{l,v} P_v(eta_q) of each source cell are
// formed once along the run (cnt + 1 cells) instead of twice per target.
// The loads of the next step's source cell are issued before the current
// step's arithmetic (measured 11% faster along dimension 1 of the 4D store
// at k = 2).  Every sum is taken in the order of nodal_fp32_group, so the
// results are the same bits.
template <int K, int FT, bool OFF32, int RUN>
__device__ __forceinline__ void nodal_fp32_walk(const NodalArgs& a, uint32_t line0, uint32_t i0, int cnt,
                                                uint32_t j, int32_t sig, const int (&jb)[FT])
{
    constexpr int O = K + 1;
    const int32_t N = int32_t(a.N);
    // raw values of the source cell at x along the line, and their node values
    auto load_cell = [&](int32_t x, float (&v)[FT][O][O]) {
        const uint32_t cx = line0 + uint32_t(x) * a.inner_x;
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l)
#pragma unroll
                for (int w = 0; w < O; ++w) {
                    const int J = jb[u] + l * a.ostride + w * a.vstride;
                    if constexpr (OFF32) {
                        const float* h = static_cast<const float*>(a.src.hi);
                        v[u][l][w] = __ldg(h + (uint32_t(J - 1) * uint32_t(a.pstride) + cx));
                    } else {
                        v[u][l][w] = __ldg(coef_plane<float>(a.src, a.pstride, J) + cx);
                    }
                }
    };
    auto node_values = [&](const float (&v)[FT][O][O], float (&U)[FT][O][O]) {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int q = 0; q < O; ++q)
#pragma unroll
                for (int l = 0; l < O; ++l) {
                    float s = 0.0f;
#pragma unroll
                    for (int w = 0; w < O; ++w) s = fmaf(v[u][l][w], a.eval32[q][w], s);
                    U[u][q][l] = s;
                }
    };
    int32_t xb = int32_t(i0) - sig - 1;   // sigma is in [0, N)
    xb += xb < 0 ? N : 0;
    float Ub[FT][O][O], Ua[FT][O][O], vn[FT][O][O];
    {
        float vb[FT][O][O];
        load_cell(xb, vb);
        node_values(vb, Ub);
    }
    int32_t xa = xb + 1;
    xa -= xa >= N ? N : 0;
    load_cell(xa, vn);
    for (int r = 0; r < RUN; ++r) {
        if (r >= cnt) break;
        float vc[FT][O][O];
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l)
#pragma unroll
                for (int w = 0; w < O; ++w) vc[u][l][w] = vn[u][l][w];
        int32_t xn = xa + 1;
        xn -= xn >= N ? N : 0;
        if (r + 1 < cnt) load_cell(xn, vn);   // the next step's source, in flight during this one
        node_values(vc, Ua);
        float acc[FT][O][O];
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int x = 0; x < O; ++x)
#pragma unroll
                for (int w = 0; w < O; ++w) acc[u][x][w] = 0.0f;
#pragma unroll
        for (int q = 0; q < O; ++q) {
            float A[O][O], B[O][O];
            load_ab<O>(a.tab, j * O + q, A, B);
#pragma unroll
            for (int u = 0; u < FT; ++u)
#pragma unroll
                for (int x = 0; x < O; ++x) {
                    float s = 0.0f;
#pragma unroll
                    for (int l = 0; l < O; ++l) {
                        s = fmaf(A[x][l], Ua[u][q][l], s);
                        s = fmaf(B[x][l], Ub[u][q][l], s);
                    }
#pragma unroll
                    for (int w = 0; w < O; ++w) acc[u][x][w] = fmaf(a.back32[w][q], s, acc[u][x][w]);
                }
        }
        const uint32_t c = line0 + (i0 + uint32_t(r)) * a.inner_x;
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int x = 0; x < O; ++x)
#pragma unroll
                for (int w = 0; w < O; ++w) {
                    const int J = jb[u] + x * a.ostride + w * a.vstride;
                    if constexpr (OFF32)
                        static_cast<float*>(a.dst.hi)[uint32_t(J - 1) * uint32_t(a.pstride) + c] = acc[u][x][w];
                    else
                        static_cast<float*>(a.dst.hi)[int64_t(J - 1) * a.pstride + c] = acc[u][x][w];
                }
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int q = 0; q < O; ++q)
#pragma unroll
                for (int l = 0; l < O; ++l) Ub[u][q][l] = Ua[u][q][l];
        xa = xn;
    }
}

// The fibre of the cell mean in the mixed store when the o nodes of the
// v-cell share sigma (so all nodes read the same two source cells a, b).
// In exact arithmetic, with t = m_b - m_a, delta_q(c) = sum_{jv>=1} c_{0,jv}
// P_jv(eta_q) and G_q(c) = sum_{l>=1} A_0l(alpha_q) U_q(c, l), the weighted
// row 0 of the nodes is
//     c'_{0,0} = m_a + alpha_bar t + E(a) - E(b),
//     alpha_bar = sum_q w'_q alpha_q,  E(c) = sum_q w'_q (G_q(c) - alpha_q delta_q(c)),
// because sum_q w'_q delta_q(c) = 0 (the Gauss rule of P_jv, jv >= 1).  E is a
// function of one cell (alpha_q and the matrices are fixed along a line), so
// it is formed in FP32 and the FP64 differences E(a) - E(b) telescope along
// the line: mass is conserved to FP64 rounding with four FP64 instructions
// per cell, alpha_bar being formed once per v-cell (launch_nodal_abar; the
// integer-pipe difference of sub_widened measured 11% slower in 2D).  The
// other coefficients of row 0 take the nodes' deviations from
// m_a + alpha_bar t, d_q = delta_q(a) + alpha_q (delta_q(b) - delta_q(a))
// + G_q(a) - G_q(b) + (alpha_q - alpha_bar) t, in FP32.
template <int K, bool OFF32>
__device__ __forceinline__ void nodal_mean_fibre_shared(const NodalArgs& a, uint32_t c, uint32_t i, uint32_t line0,
                                                        uint32_t j, int32_t sig)
{
    constexpr int O = K + 1;
    const int32_t N = int32_t(a.N);
    int32_t ia = int32_t(i) - sig;
    ia += ia < 0 ? N : 0;
    int32_t ib = ia - 1;
    ib += ib < 0 ? N : 0;
    const uint32_t ca = line0 + uint32_t(ia) * a.inner_x, cb = line0 + uint32_t(ib) * a.inner_x;
    const double ma = __ldg(a.src.mean + ca), mb = __ldg(a.src.mean + cb);
    float va[O][O], vb[O][O];   // [l][jv], entry (0, 0) unused
#pragma unroll
    for (int l = 0; l < O; ++l)
#pragma unroll
        for (int v = 0; v < O; ++v) {
            if (l == 0 && v == 0) continue;
            const int J = l * a.ostride + v * a.vstride;
            va[l][v] = ld_hi<OFF32>(a, J, ca);
            vb[l][v] = ld_hi<OFF32>(a, J, cb);
        }
    const double t = mb - ma;
    const float t32 = d2f_fast(t, false);
    float acc[O][O];   // rows jx >= 1
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) acc[x][v] = 0.0f;
    const double abar = __ldg(a.abar + j);   // per v-cell (launch_nodal_abar)
    float a32[kNa32];                         // alpha_q in FP32, then alpha_bar in FP32
    {
        const float4* r = reinterpret_cast<const float4*>(a.na32 + size_t(j) * kNa32);
#pragma unroll
        for (int h = 0; h < (na32_abar(O) + 4) / 4; ++h) {
            const float4 x = __ldg(r + h);
            a32[4 * h] = x.x;
            a32[4 * h + 1] = x.y;
            a32[4 * h + 2] = x.z;
            a32[4 * h + 3] = x.w;
        }
    }
    const float abar32 = a32[na32_abar(O)];
    float ea = 0.0f, eb = 0.0f;
    float dev[O];
#pragma unroll
    for (int q = 0; q < O; ++q) {
        const uint32_t cls = j * O + q;
        float A[O][O], B[O][O];
        load_ab<O>(a.tab, cls, A, B);
        // node values: delta_q of row 0, U_q(l) of the others
        float da = 0.0f, db = 0.0f;
#pragma unroll
        for (int v = 1; v < O; ++v) {
            da = fmaf(va[0][v], a.eval32[q][v], da);
            db = fmaf(vb[0][v], a.eval32[q][v], db);
        }
        float ua[O], ub[O];
#pragma unroll
        for (int l = 1; l < O; ++l) {
            float sa = 0.0f, sb = 0.0f;
#pragma unroll
            for (int v = 0; v < O; ++v) {
                sa = fmaf(va[l][v], a.eval32[q][v], sa);
                sb = fmaf(vb[l][v], a.eval32[q][v], sb);
            }
            ua[l] = sa;
            ub[l] = sb;
        }
        float ga = 0.0f, gb = 0.0f;
#pragma unroll
        for (int l = 1; l < O; ++l) {
            ga = fmaf(A[0][l], ua[l], ga);
            gb = fmaf(A[0][l], ub[l], gb);
        }
        // E(a), E(b): the same operations on each cell's own values
        ea = fmaf(a.wmean32[q], fmaf(-a32[q], da, ga), ea);
        eb = fmaf(a.wmean32[q], fmaf(-a32[q], db, gb), eb);
        dev[q] = fmaf(a32[q], db - da, da) + (ga - gb);
        // rows jx >= 1, the l = 0 term from ua0 - ub0 = -t + da - db
        const float d0 = (da - db) - t32;
#pragma unroll
        for (int x = 1; x < O; ++x) {
            float s = A[x][0] * d0;
#pragma unroll
            for (int l = 1; l < O; ++l) {
                s = fmaf(A[x][l], ua[l], s);
                s = fmaf(B[x][l], ub[l], s);
            }
#pragma unroll
            for (int v = 0; v < O; ++v) acc[x][v] = fmaf(a.back32[v][q], s, acc[x][v]);
        }
    }
    a.dst.mean[c] = fma(abar, t, ma) + (f2d_fast(ea) - f2d_fast(eb));
#pragma unroll
    for (int v = 1; v < O; ++v) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < O; ++q) s = fmaf(a.back32[v][q], fmaf(a32[q] - abar32, t32, dev[q]), s);
        acc[0][v] = s;
    }
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) {
            if (x == 0 && v == 0) continue;
            st_hi<OFF32>(a, x * a.ostride + v * a.vstride, c, acc[x][v]);
        }
}

// The fibre of the cell mean in the mixed store (see the file comment).
template <int K, bool OFF32>
__device__ __forceinline__ void nodal_mean_fibre(const NodalArgs& a, uint32_t c, uint32_t i, uint32_t line0,
                                                 uint32_t j)
{
    constexpr int O = K + 1;
    float acc[O][O];   // rows jx >= 1
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) acc[x][v] = 0.0f;
    double up0[O];
    float va[O][O], vb[O][O];   // [l][jv], entry (0, 0) unused
    double ma = 0.0, mb = 0.0;
    const int32_t N = int32_t(a.N);
    auto load = [&](int32_t sig) {
        int32_t ia = int32_t(i) - sig;
        ia += ia < 0 ? N : 0;
        int32_t ib = ia - 1;
        ib += ib < 0 ? N : 0;
        const uint32_t ca = line0 + uint32_t(ia) * a.inner_x, cb = line0 + uint32_t(ib) * a.inner_x;
        ma = __ldg(a.src.mean + ca);
        mb = __ldg(a.src.mean + cb);
#pragma unroll
        for (int l = 0; l < O; ++l)
#pragma unroll
            for (int v = 0; v < O; ++v) {
                if (l == 0 && v == 0) continue;
                const int J = l * a.ostride + v * a.vstride;
                va[l][v] = ld_hi<OFF32>(a, J, ca);
                vb[l][v] = ld_hi<OFF32>(a, J, cb);
            }
    };
    int32_t sg[O];
    bool same = true;
#pragma unroll
    for (int q = 0; q < O; ++q) {
        sg[q] = __ldg(a.tab.sigma + j * O + q);
        same = same && sg[q] == sg[0];
    }
    if (same) load(sg[0]);
#pragma unroll
    for (int q = 0; q < O; ++q) {
        const uint32_t cls = j * O + q;
        if (!same) load(sg[q]);
        float A[O][O], B[O][O];
        load_ab<O>(a.tab, cls, A, B);
        // node values: row 0 in FP64, the others in FP32
        double ua0 = ma, ub0 = mb;
#pragma unroll
        for (int v = 1; v < O; ++v) {
            ua0 = fma(f2d_fast(va[0][v]), a.eval64[q][v], ua0);
            ub0 = fma(f2d_fast(vb[0][v]), a.eval64[q][v], ub0);
        }
        float ua[O], ub[O];
#pragma unroll
        for (int l = 1; l < O; ++l) {
            float sa = 0.0f, sb = 0.0f;
#pragma unroll
            for (int v = 0; v < O; ++v) {
                sa = fmaf(va[l][v], a.eval32[q][v], sa);
                sb = fmaf(vb[l][v], a.eval32[q][v], sb);
            }
            ua[l] = sa;
            ub[l] = sb;
        }
        // row 0: conservation form with the per-cell FP32 sums
        float ga = 0.0f, gb = 0.0f;
#pragma unroll
        for (int l = 1; l < O; ++l) {
            ga = fmaf(A[0][l], ua[l], ga);
            gb = fmaf(A[0][l], ub[l], gb);
        }
        const double t = ub0 - ua0;
        up0[q] = fma(__ldg(a.tab.alpha + cls), t, ua0) + (f2d_fast(ga) - f2d_fast(gb));
        // rows jx >= 1 in FP32, the l = 0 term from fl32(ua0 - ub0)
        const float dm = d2f_fast(t, true);
#pragma unroll
        for (int x = 1; x < O; ++x) {
            float s = A[x][0] * dm;
#pragma unroll
            for (int l = 1; l < O; ++l) {
                s = fmaf(A[x][l], ua[l], s);
                s = fmaf(B[x][l], ub[l], s);
            }
#pragma unroll
            for (int v = 0; v < O; ++v) acc[x][v] = fmaf(a.back32[v][q], s, acc[x][v]);
        }
    }
    double m = 0.0;
#pragma unroll
    for (int q = 0; q < O; ++q) m = fma(a.wmean[q], up0[q], m);
    a.dst.mean[c] = m;
#pragma unroll
    for (int v = 1; v < O; ++v) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < O; ++q) s = fmaf(a.back32[v][q], d2f_fast(up0[q] - m, false), s);
        acc[0][v] = s;
    }
#pragma unroll
    for (int x = 0; x < O; ++x)
#pragma unroll
        for (int v = 0; v < O; ++v) {
            if (x == 0 && v == 0) continue;
            st_hi<OFF32>(a, x * a.ostride + v * a.vstride, c, acc[x][v]);
        }
}

// Mean's fibre of the mixed store for target c (at x = i of v-cell j).
template <int K, bool OFF32>
__device__ __forceinline__ void nodal_mean_target(const NodalArgs& a, uint32_t c, uint32_t i, uint32_t line0,
                                                  uint32_t j)
{
    constexpr int O = K + 1;
    // the nodes of a v-cell nearly always share sigma
    const int32_t s0 = __ldg(a.tab.sigma + j * O);
    bool same = true;
#pragma unroll
    for (int q = 1; q < O; ++q) same = same && __ldg(a.tab.sigma + j * O + q) == s0;
    if (same)
        nodal_mean_fibre_shared<K, OFF32>(a, c, i, line0, j, s0);
    else
        nodal_mean_fibre<K, OFF32>(a, c, i, line0, j);
}

// Runs of RUN targets of the walk form along x (PARTs 4 and 5): run = inner +
// inner_x (rx + nrunx outer) covers the targets x = rx RUN .. of the x-line
// through the cell inner + inner_x N outer, so neighbouring threads take
// neighbouring lines (x-dimension > 0) or neighbouring runs of one line
// (x-dimension 0).
template <int K, bool OFF32, int RUN>
__device__ __forceinline__ void nodal_run(const NodalArgs& a, uint32_t run, int g)
{
    constexpr int O = K + 1;
    constexpr int FT = nodal_ftw(K);
    const uint32_t t = a.fdInnerX.div(run);
    const uint32_t inn = run - t * a.inner_x;
    const uint32_t outer = a.fdRunX.div(t);
    const uint32_t i0 = (t - outer * a.nrunx) * uint32_t(RUN);
    const int cnt = min(RUN, int(a.N - i0));
    const uint32_t line0 = inn + outer * a.N * a.inner_x;
    const uint32_t ov = a.fdInnerV.div(line0);           // the v-cell is the same along the x-line
    const uint32_t j = ov - a.fdNV.div(ov) * a.NV;
    if (g == 0) {
        for (int r = 0; r < cnt; ++r)
            nodal_mean_target<K, OFF32>(a, line0 + (i0 + uint32_t(r)) * a.inner_x, i0 + uint32_t(r), line0, j);
        return;
    }
    int jb[FT];
#pragma unroll
    for (int u = 0; u < FT; ++u) jb[u] = nodal_fibre_base<O>(a, min(g + u, int(a.nfib2) - 1));
    const int32_t s0 = __ldg(a.tab.sigma + j * O);
    bool same = true;
#pragma unroll
    for (int q = 1; q < O; ++q) same = same && __ldg(a.tab.sigma + j * O + q) == s0;
    if (same) {
        nodal_fp32_walk<K, FT, OFF32, RUN>(a, line0, i0, cnt, j, s0, jb);
    } else {
        for (int r = 0; r < cnt; ++r)
            nodal_fp32_group<K, FT, OFF32>(a, line0 + (i0 + uint32_t(r)) * a.inner_x, i0 + uint32_t(r), line0,
                                           j, jb);
    }
}

// PART 0: every fibre (FP64 store; fibre blockIdx.y); 1: only the mean's
// fibre of the mixed store (two dimensions); 4 and 5: every fibre of the
// mixed store, the blocks of the fibre groups interleaved in a 1D grid (block
// b takes group b % groups), so that blocks of the mean's fibre, bound by the
// FP64 pipe, run beside blocks of FP32 fibres, bound by instruction issue;
// the FP32 fibres take runs of consecutive targets along x.  Part 4 (runs of
// kNodalRun) serves x-dimensions > 0, where the lanes of a warp sit on
// neighbouring x-lines, so that every step of the runs is coalesced (measured
// 8.5% faster than one target per thread along dimension 1 of the 4D store at
// k = 2).  Along dimension 0 the lanes of a run sit RUN cells apart: part 5
// takes runs of kNodalRun0 = 2 there (4652 GB/s against 4090 for one target
// per thread, 3521 and 3169 for runs of 3 and 4, in the 4D store at k = 2).
// Part 1 runs at least 4 blocks of 256 threads per SM (64 registers): in 2D
// 4096^2 at k = 2 it measured 3820 GB/s against 2782 with 2 (96 registers)
// and 3540 with 3.
template <int K, int MODE, int PART>
__global__ void __launch_bounds__(PART >= 4 ? 128 : 256, K == 3 ? 1 : PART >= 4 ? 4 : PART == 1 ? 4 : 2)
    k_sweep_nodal(const NodalArgs a)
{
    constexpr int O = K + 1;
    if constexpr (PART == 4 || PART == 5) {
        constexpr int FT = nodal_ftw(K);
        constexpr int RUN = PART == 4 ? kNodalRun : kNodalRun0;
        // group 0: the mean's fibre; group r >= 1: FP32 fibres 1 + (r - 1) FT ..
        const uint32_t ngroups = 1 + (a.nfib2 - 2) / FT + 1;
        const int r = int(blockIdx.x % ngroups);
        const uint32_t run = (blockIdx.x / ngroups) * blockDim.x + threadIdx.x;
        if (run >= a.nruns) return;
        const int g = r == 0 ? 0 : 1 + (r - 1) * FT;
        if (a.off32)
            nodal_run<K, true, RUN>(a, run, g);
        else
            nodal_run<K, false, RUN>(a, run, g);
        return;
    }
    const int g = int(blockIdx.y);
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.cells) return;
    const uint32_t ox = a.fdInnerX.div(c);
    const uint32_t i = ox - a.fdNX.div(ox) * a.N;        // coordinate along x
    const uint32_t ov = a.fdInnerV.div(c);
    const uint32_t j = ov - a.fdNV.div(ov) * a.NV;       // v-cell
    const uint32_t line0 = c - i * a.inner_x;
    if constexpr (MODE == M_FP64)
        nodal_plain<K, double>(a, c, i, line0, j, nodal_fibre_base<O>(a, g));
    else if (a.off32)
        nodal_mean_target<K, true>(a, c, i, line0, j);
    else
        nodal_mean_target<K, false>(a, c, i, line0, j);
}

template <int K>
cudaError_t nodal_launch(int mode, const NodalArgs& a, int nfib2, cudaStream_t st)
{
    const int block = 256;
    const uint32_t bx = (a.cells + block - 1) / block;
    if (mode == M_FP64) {
        k_sweep_nodal<K, M_FP64, 0><<<dim3(bx, uint32_t(nfib2)), block, 0, st>>>(a);
    } else if (nfib2 == 1) {
        k_sweep_nodal<K, M_F32, 1><<<dim3(bx, 1), block, 0, st>>>(a);
    } else {
        const int run = a.inner_x == 1 ? kNodalRun0 : kNodalRun;
        NodalArgs b = a;
        b.nrunx = (a.N + run - 1) / run;
        b.fdRunX.set(b.nrunx);
        const uint64_t nruns = uint64_t(a.cells / a.N) * b.nrunx;
        if (nruns > 0xffffffffu) return cudaErrorInvalidValue;
        b.nruns = uint32_t(nruns);
        const uint64_t nb = (nruns + 127) / 128 * uint64_t(1 + (nfib2 - 2) / nodal_ftw(K) + 1);
        if (nb > 0x7fffffffu) return cudaErrorInvalidValue;
        if (a.inner_x == 1)
            k_sweep_nodal<K, M_F32, 5><<<uint32_t(nb), 128, 0, st>>>(b);
        else
            k_sweep_nodal<K, M_F32, 4><<<uint32_t(nb), 128, 0, st>>>(b);
    }
    return cudaGetLastError();
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_o from
// the Chebyshev-like start cos(pi (q + 3/4) / (o + 1/2)), ascending.
void gauss_nodes(int o, double* eta, double* w)
{
    for (int q = 0; q < o; ++q) {
        double x = std::cos(M_PI * (q + 0.75) / (o + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int n = 1; n < o; ++n) {
                const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (o == 1) p1 = x, p0 = 1.0;
            dp = o * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        eta[o - 1 - q] = x;
        w[o - 1 - q] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

double legendre_host(int j, double x)
{
    double p0 = 1.0, p1 = x;
    if (j == 0) return 1.0;
    for (int n = 1; n < j; ++n) {
        const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

struct NodalWeights {
    double w[kMaxO];
    float w32[kMaxO];
};

__global__ void k_nodal_abar(const double* __restrict__ alpha, int nv, int o, NodalWeights W,
                             double* __restrict__ abar, float* __restrict__ na32)
{
    const int j = int(blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= nv) return;
    double s = 0.0;
    float s32 = 0.0f;
    float* r = na32 + size_t(j) * kNa32;
    for (int q = 0; q < kNa32; ++q) r[q] = 0.0f;
    for (int q = 0; q < o; ++q) {
        const double al = __ldg(alpha + size_t(j) * o + q);
        s = fma(W.w[q], al, s);
        const float a32 = d2f_fast(al, false);
        s32 = fmaf(W.w32[q], a32, s32);
        r[q] = a32;
    }
    abar[j] = s;
    r[na32_abar(o)] = s32;
}

}  // namespace

cudaError_t launch_nodal_abar(const double* alpha, int nv, int o, const double* wmean, const float* wmean32,
                              double* abar, float* na32, cudaStream_t st)
{
    if (nv <= 0 || o < 1 || o > kMaxO) return cudaErrorInvalidValue;
    NodalWeights W{};
    for (int q = 0; q < o; ++q) {
        W.w[q] = wmean[q];
        W.w32[q] = wmean32[q];
    }
    k_nodal_abar<<<(nv + 127) / 128, 128, 0, st>>>(alpha, nv, o, W, abar, na32);
    return cudaGetLastError();
}

void nodal_setup(int K, double* eta, double* weights, NodalArgs* a)
{
    const int o = K + 1;
    gauss_nodes(o, eta, weights);
    a->O = o;
    for (int q = 0; q < o; ++q)
        for (int v = 0; v < o; ++v) {
            const double p = legendre_host(v, eta[q]);
            a->eval64[q][v] = p;
            a->eval32[q][v] = float(p);
            const double b = 0.5 * (2.0 * v + 1.0) * weights[q] * p;
            a->back64[v][q] = b;
            a->back32[v][q] = float(b);
        }
    // w'_q = w_q / 2 on the grid of 2^-52, the last one completing the sum to
    // exactly 1 (every partial sum is a multiple of 2^-52 below 2, so exact)
    double sum = 0.0;
    for (int q = 0; q + 1 < o; ++q) {
        a->wmean[q] = std::ldexp(std::nearbyint(std::ldexp(0.5 * weights[q], 52)), -52);
        sum += a->wmean[q];
    }
    a->wmean[o - 1] = 1.0 - sum;
    for (int q = 0; q < o; ++q) {
        a->back64[0][q] = a->wmean[q];
        a->wmean32[q] = float(a->wmean[q]);
    }
}

cudaError_t launch_sweep_nodal(int K, int mode, const NodalArgs& a, int nfib2, cudaStream_t st)
{
    if (mode != M_FP64 && mode != M_F32) return cudaErrorInvalidValue;
    switch (K) {
    case 0: return nodal_launch<0>(mode, a, nfib2, st);
    case 1: return nodal_launch<1>(mode, a, nfib2, st);
    case 2: return nodal_launch<2>(mode, a, nfib2, st);
    case 3: return nodal_launch<3>(mode, a, nfib2, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sl
