// sl_aux.cu -- the small kernels around the sweep: shift decomposition and
// construction of A(alpha), B(alpha) per shift class, the FP64 mass
// reduction, encoding/decoding of the split store, and the initial
// projection eq. (cj).
#include "../../include/sl.h"
#include "sl_ab.cuh"
#include "sl_sweep.cuh"

namespace sl {

// ---------------------------------------------------------------- A, B

// The table of a single problem of at most kAbEntryClasses classes: one thread
// per entry of A and B of a class
// (2 o^2 threads per class, each splitting the class's shift itself, the
// shift decomposition and Horner evaluation of sl_ab.cuh's ab_class_k entry
// by entry, so the same bits).  A problem has a few thousand classes at most,
// and one thread per class left one warp per SM running some 800 instructions
// of dependent latency (7.5 us for 512 classes; 4.1-5.0 us this way).  The
// batch, with 10^5 classes, keeps one thread per class (k_batch_ab): there the
// FP64 pipe, not latency, bounds the build.
template <int K>
__global__ void __launch_bounds__(128) k_ab_build_entries(int nclass, uint32_t N, ShiftSource src, PolyTab tab,
                                                          int32_t* __restrict__ sigma, double* __restrict__ alpha,
                                                          double* __restrict__ ab64, float* __restrict__ ab32)
{
    constexpr int O = K + 1;
    constexpr int E = 2 * O * O;
    constexpr int deg = 2 * K + 1;
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = item / E;
    if (c >= nclass) return;
    const int e = item - c * E;
    const double s = shift_of(src, c);
    const double f = floor(s);
    double a = s - f;
    long long sg = (long long)f;
    if (a >= 1.0) {
        sg += 1;
        a = 0.0;
    }
    if (e == 0) {
        long long r = sg % (long long)N;
        if (r < 0) r += N;
        sigma[c] = int32_t(r);
        alpha[c] = a;
    }
    const bool isb = e >= O * O;
    const int jl = isb ? e - O * O : e;
    const int j = jl / O, l = jl - (jl / O) * O;
    double v;
    if (a == 0.0) {
        v = isb ? 0.0 : (j == l ? 1.0 : 0.0);
    } else {
        const double t = a - 0.5;
        const double* pc = isb ? tab.b[j][l] : tab.a[j][l];
        v = pc[deg];
#pragma unroll
        for (int p = deg - 1; p >= 0; --p) v = fma(v, t, pc[p]);
    }
    ab64[size_t(c) * ab_stride64(O) + e] = v;
    ab32[size_t(c) * ab_stride32(O) + e] = __double2float_rn(v);
}

// One thread per class (ab_class_k), in one-warp blocks: for tables of many
// classes, where the per-entry form would repeat the shift split 2 o^2 times
// per class on the FP64 pipe.
template <int K>
__global__ void __launch_bounds__(32) k_ab_build_classes(int nclass, uint32_t N, ShiftSource src, PolyTab tab,
                                                         int32_t* __restrict__ sigma, double* __restrict__ alpha,
                                                         double* __restrict__ ab64, float* __restrict__ ab32)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclass) return;
    ab_class_k<K>(shift_of(src, c), N, tab, c, sigma, alpha, ab64, ab32);
}

// Classes up to which the table takes one thread per entry.
constexpr int kAbEntryClasses = 8192;

cudaError_t launch_ab_build(int K, int nclass, uint32_t N, const ShiftSource& src,
                            const PolyTab& tab, int32_t* sigma, double* alpha, double* ab64,
                            float* ab32, cudaStream_t st)
{
    if (nclass > kAbEntryClasses) {
        const int grid = (nclass + 31) / 32;
        switch (K) {
        case 0: k_ab_build_classes<0><<<grid, 32, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
        case 1: k_ab_build_classes<1><<<grid, 32, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
        case 2: k_ab_build_classes<2><<<grid, 32, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
        case 3: k_ab_build_classes<3><<<grid, 32, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int block = 128;
    const int E = 2 * (K + 1) * (K + 1);
    const int grid = int((int64_t(nclass) * E + block - 1) / block);
    switch (K) {
    case 0: k_ab_build_entries<0><<<grid, block, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
    case 1: k_ab_build_entries<1><<<grid, block, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
    case 2: k_ab_build_entries<2><<<grid, block, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
    case 3: k_ab_build_entries<3><<<grid, block, 0, st>>>(nclass, N, src, tab, sigma, alpha, ab64, ab32); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- mass

constexpr int kMassThreads = 256;
constexpr int kMassMaxBlocks = 1024;

int mass_blocks(uint32_t cells)
{
    int64_t b = (int64_t(cells) + kMassThreads * 8 - 1) / (kMassThreads * 8);
    if (b < 1) b = 1;
    if (b > kMassMaxBlocks) b = kMassMaxBlocks;
    return int(b);
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[kMassThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < kMassThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// Fixed-shape reduction: the grid size depends only on the cell count, each
// thread sums a fixed strided subset, warps reduce by shuffles, blocks write
// partials, and one block sums the partials in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kMassThreads) k_mass_partial(const T* __restrict__ mean,
                                                               uint32_t cells,
                                                               double* __restrict__ partials)
{
    double s = 0.0;
    for (uint32_t c = blockIdx.x * kMassThreads + threadIdx.x; c < cells;
         c += gridDim.x * kMassThreads)
        s += double(mean[c]);
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const double* __restrict__ partials,
                                                             int n, double vol,
                                                             double* __restrict__ out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kMassThreads) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) out[0] = vol * s;
}

cudaError_t launch_mass(const double* mean, uint32_t cells, double* partials, int nblocks,
                        double vol, double* out, cudaStream_t st)
{
    k_mass_partial<double><<<nblocks, kMassThreads, 0, st>>>(mean, cells, partials);
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, vol, out);
    return cudaGetLastError();
}

cudaError_t launch_mass_f32(const float* mean, uint32_t cells, double* partials, int nblocks,
                            double vol, double* out, cudaStream_t st)
{
    k_mass_partial<float><<<nblocks, kMassThreads, 0, st>>>(mean, cells, partials);
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, vol, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- codec

// Coefficient J of a cell in the stores placed by the coefficient map (the
// general split stores and the all-FP32 store): FP64 plane -1 - e or FP32
// plane e of the map entry e, FP32 values rounded to nearest even.
__device__ __forceinline__ void put_mapped(const CodecArgs& c, int J, uint32_t cell, double v)
{
    const int e = c.cmap[J];
    if (e < 0)
        c.p.mean[int64_t(-1 - e) * c.pstride + cell] = v;
    else
        static_cast<float*>(c.p.hi)[int64_t(e) * c.pstride + cell] = __double2float_rn(v);
}
__device__ __forceinline__ double get_mapped(const CodecArgs& c, int J, uint32_t cell)
{
    const int e = c.cmap[J];
    if (e < 0) return c.p.mean[int64_t(-1 - e) * c.pstride + cell];
    return double(static_cast<const float*>(c.p.hi)[int64_t(e) * c.pstride + cell]);
}

template <int MODE>
__device__ void encode_cell(const CodecArgs& c, const double* v, uint32_t cell)
{
    using T = typename St<MODE>::T;
    if constexpr (MODE == M_SPLIT2) {
        for (int J = 0; J < c.ncoef; ++J) put_mapped(c, J, cell, v[J]);
        return;
    }
    c.p.mean[cell] = v[0];
    if constexpr (MODE == M_FP64) {
        for (int J = 1; J < c.ncoef; ++J) *coef_ptr<T>(c, J, cell) = v[J];
    } else if constexpr (MODE == M_F32) {
        for (int J = 1; J < c.ncoef; ++J) *coef_ptr<T>(c, J, cell) = __double2float_rn(v[J]);
    } else {
        double mx = 0.0;
        for (int J = 1; J < c.ncoef; ++J) mx = fmax(mx, fabs(v[J]));
        float s, inv;
        pow2_scale(__double2float_rn(mx), s, inv);
        c.p.scale[cell] = s;
        for (int J = 1; J < c.ncoef; ++J) {
            const double x = v[J] * double(inv);   // exact: inv is a power of two
            T* dst = coef_ptr<T>(c, J, cell);
            if constexpr (MODE == M_BF16)
                *dst = __double2bfloat16(x);
            else
                *dst = __double2half(x);
        }
    }
}

template <int MODE>
__device__ void decode_cell(const CodecArgs& c, uint32_t cell, double* out)
{
    using T = typename St<MODE>::T;
    if constexpr (MODE == M_SPLIT2) {
        for (int J = 0; J < c.ncoef; ++J) out[J] = get_mapped(c, J, cell);
        return;
    }
    out[0] = c.p.mean[cell];
    double s = 1.0;
    if constexpr (St<MODE>::scaled) s = double(c.p.scale[cell]);
    for (int J = 1; J < c.ncoef; ++J) {
        const T raw = *coef_ptr<T>(c, J, cell);
        double x;
        if constexpr (MODE == M_FP64)
            x = raw;
        else if constexpr (MODE == M_F32)
            x = double(raw);
        else if constexpr (MODE == M_BF16)
            x = double(__bfloat162float(raw));
        else
            x = double(__half2float(raw));
        out[J] = x * s;
    }
}

template <int MODE>
__global__ void k_encode(CodecArgs c, const double* __restrict__ aos, uint32_t first,
                         uint32_t count)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    encode_cell<MODE>(c, aos + size_t(t) * c.ncoef, first + t);
}

template <int MODE>
__global__ void k_decode(CodecArgs c, double* __restrict__ aos, uint32_t first, uint32_t count)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    decode_cell<MODE>(c, first + t, aos + size_t(t) * c.ncoef);
}

template <int MODE>
__global__ void k_gather(CodecArgs c, const int64_t* __restrict__ cells, uint32_t count,
                         double* __restrict__ aos)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    decode_cell<MODE>(c, uint32_t(cells[t]), aos + size_t(t) * c.ncoef);
}

#define SL_MODE_SWITCH(mode, CALL)                     \
    switch (mode) {                                    \
    case M_FP64: { constexpr int MD = M_FP64; CALL; } break; \
    case M_F32: { constexpr int MD = M_F32; CALL; } break;   \
    case M_BF16: { constexpr int MD = M_BF16; CALL; } break; \
    case M_FP16: { constexpr int MD = M_FP16; CALL; } break; \
    case M_F32ALL:                                     \
    case M_SPLIT2:                                     \
    case M_SPLIT3: { constexpr int MD = M_SPLIT2; CALL; } break; \
    default: return cudaErrorInvalidValue;             \
    }

cudaError_t launch_encode(const CodecArgs& c, const double* aos, uint32_t first, uint32_t count,
                          cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int b = 128;
    SL_MODE_SWITCH(c.mode, (k_encode<MD><<<(count + b - 1) / b, b, 0, st>>>(c, aos, first, count)));
    return cudaGetLastError();
}

cudaError_t launch_decode(const CodecArgs& c, double* aos, uint32_t first, uint32_t count,
                          cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int b = 128;
    SL_MODE_SWITCH(c.mode, (k_decode<MD><<<(count + b - 1) / b, b, 0, st>>>(c, aos, first, count)));
    return cudaGetLastError();
}

cudaError_t launch_gather(const CodecArgs& c, const int64_t* cells, uint32_t count, double* aos,
                          cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int b = 128;
    SL_MODE_SWITCH(c.mode, (k_gather<MD><<<(count + b - 1) / b, b, 0, st>>>(c, cells, count, aos)));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- projection

__device__ __forceinline__ double legendre_dev(int j, double x)
{
    if (j == 0) return 1.0;
    double pm = 1.0, p = x;
    for (int n = 1; n < j; ++n) {
        const double pn = ((2.0 * n + 1.0) * x * p - n * pm) / (n + 1.0);
        pm = p;
        p = pn;
    }
    return p;
}

// 1D projections of every factor: tab[((t*ndim + m)*nmax + i)*o + j] =
// (2j+1)/2 sum_q w_q g_{t,m}(x_i + h t_q / 2) P_j(t_q)   (eq. (cj)).
__global__ void k_project_1d(ProjectArgs pa, const double* __restrict__ params,
                             double* __restrict__ tab, uint32_t nmax)
{
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t total = uint32_t(pa.nterms) * pa.ndim * nmax;
    if (idx >= total) return;
    const uint32_t i = idx % nmax;
    const uint32_t tm = idx / nmax;
    const int m = int(tm % pa.ndim);
    if (i >= pa.n[m]) return;
    const double* prm = params + size_t(tm) * 4;
    const double xc = pa.lo[m] + (double(i) + 0.5) * pa.h[m];
    const int O = pa.K + 1;
    for (int j = 0; j < O; ++j) {
        double acc = 0.0;
        for (int q = 0; q < pa.nq; ++q) {
            const double x = xc + 0.5 * pa.h[m] * pa.node[q];
            const double d = x - prm[1];
            const double g = exp(-prm[0] * d * d) * cos(prm[2] * x + prm[3]);
            acc += pa.weight[q] * g * legendre_dev(j, pa.node[q]);
        }
        tab[size_t(idx) * O + j] = 0.5 * (2.0 * j + 1.0) * acc;
    }
}

// Coefficient J of a cell: sum_t w_t prod_m tab[t][m][i_m][j_m].
__device__ double project_coef(const ProjectArgs& pa, const double* w, const double* tab,
                               uint32_t nmax, const uint32_t* im, int J)
{
    const int O = pa.K + 1;
    int jm[kMaxDim];
    int r = J;
    for (int m = 0; m < pa.ndim; ++m) {
        jm[m] = r % O;
        r /= O;
    }
    double v = 0.0;
    for (int t = 0; t < pa.nterms; ++t) {
        double p = w[t];
        for (int m = 0; m < pa.ndim; ++m)
            p *= tab[((size_t(t) * pa.ndim + m) * nmax + im[m]) * O + jm[m]];
        v += p;
    }
    return v;
}

template <int MODE>
__global__ void k_project_cells(ProjectArgs pa, const double* __restrict__ w,
                                const double* __restrict__ tab, uint32_t nmax, CodecArgs c,
                                uint32_t cells)
{
    using T = typename St<MODE>::T;
    const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    uint32_t im[kMaxDim];
    uint32_t r = cell;
    for (int m = 0; m < pa.ndim; ++m) {
        im[m] = r % pa.n[m];
        r /= pa.n[m];
    }
    if constexpr (MODE == M_SPLIT2) {
        for (int J = 0; J < c.ncoef; ++J) put_mapped(c, J, cell, project_coef(pa, w, tab, nmax, im, J));
        return;
    }
    c.p.mean[cell] = project_coef(pa, w, tab, nmax, im, 0);
    if constexpr (!St<MODE>::scaled) {
        for (int J = 1; J < c.ncoef; ++J) {
            const double v = project_coef(pa, w, tab, nmax, im, J);
            if constexpr (MODE == M_FP64)
                *coef_ptr<T>(c, J, cell) = v;
            else
                *coef_ptr<T>(c, J, cell) = __double2float_rn(v);
        }
    } else {
        double mx = 0.0;
        for (int J = 1; J < c.ncoef; ++J) mx = fmax(mx, fabs(project_coef(pa, w, tab, nmax, im, J)));
        float s, inv;
        pow2_scale(__double2float_rn(mx), s, inv);
        c.p.scale[cell] = s;
        for (int J = 1; J < c.ncoef; ++J) {
            const double x = project_coef(pa, w, tab, nmax, im, J) * double(inv);
            T* dst = coef_ptr<T>(c, J, cell);
            if constexpr (MODE == M_BF16)
                *dst = __double2bfloat16(x);
            else
                *dst = __double2half(x);
        }
    }
}

cudaError_t launch_project(const ProjectArgs& pa, const double* d_weights, const double* d_params,
                           double* d_tab, uint32_t nmax, const CodecArgs& c, uint32_t cells,
                           cudaStream_t st)
{
    const int b = 128;
    const uint32_t total = uint32_t(pa.nterms) * pa.ndim * nmax;
    if (total > 0) k_project_1d<<<(total + b - 1) / b, b, 0, st>>>(pa, d_params, d_tab, nmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SL_MODE_SWITCH(c.mode, (k_project_cells<MD><<<(cells + b - 1) / b, b, 0, st>>>(
                               pa, d_weights, d_tab, nmax, c, cells)));
    return cudaGetLastError();
}

}  // namespace sl

// ---------------------------------------------------------------- conversion self-test

namespace sl {

// Branch-free forms into the outputs; the branching forms must give the same
// bits (NaN compared as NaN), else the element counts as a mismatch.
__global__ void k_conv_check(const double* __restrict__ din, const float* __restrict__ fin, uint32_t n,
                             float* __restrict__ fout, double* __restrict__ dout,
                             unsigned long long* __restrict__ mism)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float p = d2f_fast(din[i], false), q = d2f_fast(din[i], true);
    const double d = f2d_fast(fin[i]);
    fout[2 * i] = p;
    fout[2 * i + 1] = q;
    dout[i] = d;
    const float pb = d2f_branch(din[i], false), qb = d2f_branch(din[i], true);
    const double db = f2d_branch(fin[i]);
    const bool same = (__float_as_uint(p) == __float_as_uint(pb) || (p != p && pb != pb)) &&
                      (__float_as_uint(q) == __float_as_uint(qb) || (q != q && qb != qb)) &&
                      (__double_as_longlong(d) == __double_as_longlong(db) || (d != d && db != db));
    if (!same) atomicAdd(mism, 1ull);
}

// sub_widened against the FP64 subtraction of the widened operands.
__global__ void k_sub_check(const float* __restrict__ a, const float* __restrict__ b, uint32_t n,
                            double* __restrict__ out, unsigned long long* __restrict__ mism)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = sub_widened(a[i], b[i]);
    const double f = f2d_fast(a[i]) - f2d_fast(b[i]);
    out[i] = r;
    if (!(__double_as_longlong(r) == __double_as_longlong(f) || (r != r && f != f))) atomicAdd(mism, 1ull);
}

// FP64 FMA throughput: C independent dependency chains per thread, so the
// FP64 pipe, not the latency of one chain, sets the rate; the iteration loop
// is unrolled four times so that the loop's own instructions are few.
// x -> a x + b with a = 1 - 2^-20 and b = 2^-30 keeps every value normal and
// bounded.  a and b are read from global memory, so the FMAs take register
// operands: with operands from the constant bank GB300 issued FP64 FMAs at
// 1.68 per clock per SM instead of 2.  The sum is stored only if it is
// negative (never), which keeps the chains live.
template <int C>
__global__ void __launch_bounds__(256) k_fp64_fma(int iters4, const double* __restrict__ coef,
                                                  double* __restrict__ sink)
{
    const double a = coef[0], b = coef[1];
    double x[C];
#pragma unroll
    for (int i = 0; i < C; ++i) x[i] = 0.25 * i + 1e-6 * threadIdx.x + 1e-9 * blockIdx.x;
    for (int it = 0; it < iters4; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < C; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < C; ++i) s += x[i];
    if (s < 0.0) *sink = s;
}

}  // namespace sl

extern "C" sl_status sl_selftest_fp64_rate(int64_t iters, void* cuda_stream, double* flops_per_s)
{
    if (!flops_per_s || iters < 1 || iters > (int64_t(1) << 24)) return SL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) return SL_ECUDA;
    double* buf = nullptr;   // a, b, sink
    if (cudaMalloc(&buf, 3 * sizeof(double)) != cudaSuccess) return SL_ENOMEM;
    const double coef[2] = {1.0 - 0x1.0p-20, 0x1.0p-30};
    e = cudaMemcpyAsync(buf, coef, sizeof(coef), cudaMemcpyHostToDevice, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // the better of 4 and 8 resident blocks of 256 threads per multiprocessor
    double best = 0.0;
    const int iters4 = int((iters + 3) / 4);
    for (int shape = 0; shape < 2 && e == cudaSuccess; ++shape) {
        const unsigned blocks = unsigned(sms) * (shape ? 8u : 4u);
        sl::k_fp64_fma<8><<<blocks, 256, 0, st>>>(iters4 / 8 + 1, buf, buf + 2);   // warm-up
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            sl::k_fp64_fma<8><<<blocks, 256, 0, st>>>(iters4, buf, buf + 2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.0f) {
            const double f = 2.0 * 4.0 * 8.0 * double(iters4) * double(blocks) * 256.0 / (double(ms) * 1e-3);
            if (f > best) best = f;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess || best <= 0.0) return SL_ECUDA;
    *flops_per_s = best;
    return SL_OK;
}

extern "C" sl_status sl_selftest_sub_widened(const float* a, const float* b, int64_t n, double* out,
                                             int64_t* mismatches)
{
    if (!a || !b || !out || !mismatches || n < 1 || n > (int64_t(1) << 26)) return SL_EINVAL;
    const size_t N = size_t(n);
    char* mem = nullptr;
    if (cudaMalloc(&mem, N * (4 + 4 + 8) + 16) != cudaSuccess) return SL_ENOMEM;
    unsigned long long* mism = reinterpret_cast<unsigned long long*>(mem);
    double* dout = reinterpret_cast<double*>(mem + 16);
    float* fa = reinterpret_cast<float*>(dout + N);
    float* fb = fa + N;
    cudaError_t e = cudaMemset(mism, 0, 8);
    if (e == cudaSuccess) e = cudaMemcpy(fa, a, N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fb, b, N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        sl::k_sub_check<<<unsigned((N + 255) / 256), 256>>>(fa, fb, uint32_t(N), dout, mism);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, N * 8, cudaMemcpyDeviceToHost);
    unsigned long long mm = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&mm, mism, 8, cudaMemcpyDeviceToHost);
    *mismatches = int64_t(mm);
    cudaFree(mem);
    return e == cudaSuccess ? SL_OK : SL_ECUDA;
}

extern "C" sl_status sl_selftest_conversions(const double* d_in, const float* f_in, int64_t n, float* f_out,
                                             double* d_out, int64_t* mismatches)
{
    if (!d_in || !f_in || !f_out || !d_out || !mismatches || n < 1 || n > (int64_t(1) << 26)) return SL_EINVAL;
    const size_t N = size_t(n);
    char* mem = nullptr;
    const size_t bytes = N * (8 + 4 + 8 + 8) + 16;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) return SL_ENOMEM;
    unsigned long long* mism = reinterpret_cast<unsigned long long*>(mem);
    double* din = reinterpret_cast<double*>(mem + 16);
    double* dout = din + N;
    float* fout = reinterpret_cast<float*>(dout + N);
    float* fin = fout + 2 * N;
    cudaError_t e = cudaMemset(mism, 0, 8);
    if (e == cudaSuccess) e = cudaMemcpy(din, d_in, N * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fin, f_in, N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        sl::k_conv_check<<<unsigned((N + 255) / 256), 256>>>(din, fin, uint32_t(N), fout, dout, mism);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(f_out, fout, N * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(d_out, dout, N * 8, cudaMemcpyDeviceToHost);
    unsigned long long mm = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&mm, mism, 8, cudaMemcpyDeviceToHost);
    *mismatches = int64_t(mm);
    cudaFree(mem);
    return e == cudaSuccess ? SL_OK : SL_ECUDA;
}
