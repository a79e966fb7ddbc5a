// sl_batch.cu -- device side of the batched sweeps: many independent
// problems of uneven sizes and degrees advance together, one persistent
// launch per split substep.
#include "sl_ab.cuh"
#include "sl_sweep.cuh"

namespace sl {

// Shift tables of every problem for one substep: block row = problem.
__global__ void k_batch_ab(const BatchAB* __restrict__ desc, const PolyTab* __restrict__ tabs,
                           double tau)
{
    const BatchAB d = desc[blockIdx.y];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.nclass) return;
    ShiftSource src{};
    src.kind = d.kind;
    src.data = d.field;
    src.lo = d.lo;
    src.hv = d.hv;
    src.tau = tau;
    src.h = d.h;
    ab_class(d.K, shift_of(src, c), d.N, tabs[d.K], c, d.sigma, d.alpha, d.ab64, d.ab32);
}

cudaError_t launch_batch_ab(const BatchAB* d_desc, const PolyTab* d_tabs, int nprob, int maxclass,
                            double tau, cudaStream_t st)
{
    if (nprob <= 0) return cudaSuccess;
    const int b = 32;   // one warp per block, so the classes spread over the SMs
    dim3 grid((maxclass + b - 1) / b, nprob);
    k_batch_ab<<<grid, b, 0, st>>>(d_desc, d_tabs, tau);
    return cudaGetLastError();
}

// Persistent sweeps over a work list.  Every thread reads its problem's sweep
// geometry straight from the (read-only, L1-cached) argument array, and the
// problem's degree K (0, 1 or 2) and fibres per thread ft (ceil(nfib / nfg),
// at most FTM) select a compiled body, uniform across the block.  Sweeps
// along dimension 0 and along the other dimensions are separate kernels, so
// each has its own register budget.
//
// Along dimension 0 the items are short tiles of equal size, taken
// round-robin (item blockIdx.x, blockIdx.x + gridDim.x, ...).  Along the
// other dimensions the items (tiles of 32 lines of uneven length) are sorted
// by decreasing cost on the host and taken by each warp from a shared
// counter, one atomic per item, so that the long ones start first and no
// warp idles while work remains; a problem's last tile of lines leaves at
// most 31 lanes idle (with tiles of a block's 128 lines, about a tenth of
// the threads of the 256-problem workload were).  Both loops are bounded by
// the item count; no block or warp waits on another.
// One item along dimension 0: reps tiles of kBatchBlock consecutive cells.
// Not inlined, so that each (K, FT) body gets its own register allocation
// and reads the problem's geometry where it needs it.
template <int K, int MODE, int FT>
__device__ __noinline__ void unit_item(const SweepArgs* __restrict__ ap, uint32_t start, int fbase, int reps)
{
    const SweepArgs& a = *ap;
    for (int r = 0; r < reps; ++r) {
        const uint32_t c = start + threadIdx.x + uint32_t(r) * kBatchBlock;
        if (c >= a.cells) break;
        unit_cell<K, MODE, FT>(a, c, fbase);
    }
}

// PC consecutive target cells c .. c + PC - 1 of one line per thread: the
// line, shift class and matrices are set up once, and the PC + 1 source
// cells i - sigma - 1 .. i - sigma + PC - 1 are each loaded once (the source
// i - sigma of one target is the i - sigma - 1 of the next).  A run that
// crosses a line end takes the one-cell form for each cell.
template <int K, int MODE, int FT, bool MEAN, int PC>
__device__ __forceinline__ void unit_run_body(const SweepArgs& a, uint32_t c, uint32_t ls, uint32_t i,
                                              uint32_t cls, int fbase)
{
    constexpr int O = K + 1;
    int jb[FT];
    group_bases<FT>(fbase, a.nfib, O, 1, jb);
    const int32_t N = int32_t(a.N);
    const int32_t sig = __ldg(a.tab.sigma + cls);
    int32_t ib = int32_t(i) - sig - 1;
    ib += ib < 0 ? N : 0;
    ib += ib < 0 ? N : 0;
    Mats<K, MODE> M;
    M.template load<MEAN>(a.tab, cls);
    CellVals<K, MODE, FT> v[PC + 1];
#pragma unroll
    for (int q = 0; q <= PC; ++q) {
        int32_t x = ib + q;
        x -= x >= N ? N : 0;
        load_cell<K, MODE, FT, MEAN>(a.src, a.pstride, ls + uint32_t(x), jb, 1, v[q]);
    }
#pragma unroll
    for (int q = 0; q < PC; ++q) {
        CellVals<K, MODE, FT> out;
        combine<K, MODE, FT, MEAN>(M, v[q + 1], v[q], out);
        store_cell<K, MODE, FT, MEAN>(a.dst, a.pstride, c + q, jb, 1, out);
    }
}

// Element offsets of a fibre group's planes from hi, formed once per work
// item in 32 bits (the problem's planes hold fewer than 2^31 elements), so
// that every access costs one 32-bit add and one address formation instead
// of a 64-bit product per value.
template <int K, int MODE, int FT, bool MEAN>
struct PlaneOffsets {
    using T = typename St<MODE>::T;
    static constexpr int O = K + 1;
    int32_t off[FT][O];   // (J - 1) * pstride of value (u, l); unused for the mean

    __device__ __forceinline__ void init(int64_t pstride, const int (&jb)[FT])
    {
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) off[u][l] = int32_t(int64_t(jb[u] + l - 1) * pstride);
    }
    __device__ __forceinline__ void load(const Planes& p, uint32_t c, CellVals<K, MODE, FT>& cv) const
    {
        const T* hi = static_cast<const T*>(p.hi);
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0) {
                    cv.m = __ldg(p.mean + c);
                    cv.v[0][0] = 0;
                } else {
                    cv.v[u][l] = ld_raw(hi + (off[u][l] + int32_t(c)));
                }
            }
    }
    __device__ __forceinline__ void store(const Planes& p, uint32_t c, const CellVals<K, MODE, FT>& cv) const
    {
        T* hi = static_cast<T*>(p.hi);
#pragma unroll
        for (int u = 0; u < FT; ++u)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                if (MEAN && u == 0 && l == 0)
                    p.mean[c] = cv.m;
                else
                    st_raw(hi + (off[u][l] + int32_t(c)), cv.v[u][l]);
            }
    }
};

// The runs of one work item with the plane offsets formed once (see
// PlaneOffsets); the same arithmetic as unit_run_body, cell for cell.
template <int K, int MODE, int FT, bool MEAN, int PC>
__device__ __forceinline__ void unit_runs_offsets(const SweepArgs& a, uint32_t start, const int (&jb)[FT], int fbase,
                                                  int reps)
{
    PlaneOffsets<K, MODE, FT, MEAN> P;
    P.init(a.pstride, jb);
    const int32_t N = int32_t(a.N);
    for (int r = 0; r < reps; ++r) {
        const uint32_t c = start + PC * (threadIdx.x + uint32_t(r) * kBatchBlock);
        if (c >= a.cells) break;
        const uint32_t line = a.fdN.div(c);
        const uint32_t ls = line * a.N;
        const uint32_t i = c - ls;
        if (i + PC > a.N) {   // the run crosses a line end: one cell at a time
            for (int q = 0; q < PC; ++q)
                if (c + q < a.cells) unit_cell<K, MODE, FT>(a, c + q, fbase);
            continue;
        }
        const uint32_t cls = shift_class(a, 0, line);
        const int32_t sig = __ldg(a.tab.sigma + cls);
        int32_t ib = int32_t(i) - sig - 1;
        ib += ib < 0 ? N : 0;
        ib += ib < 0 ? N : 0;
        Mats<K, MODE> M;
        M.template load<MEAN>(a.tab, cls);
        CellVals<K, MODE, FT> v[PC + 1];
#pragma unroll
        for (int q = 0; q <= PC; ++q) {
            int32_t x = ib + q;
            x -= x >= N ? N : 0;
            P.load(a.src, ls + uint32_t(x), v[q]);
        }
#pragma unroll
        for (int q = 0; q < PC; ++q) {
            CellVals<K, MODE, FT> out;
            combine<K, MODE, FT, MEAN>(M, v[q + 1], v[q], out);
            P.store(a.dst, c + q, out);
        }
    }
}

template <int K, int MODE, int FT, int PC>
__device__ __noinline__ void unit_item_runs(const SweepArgs* __restrict__ ap, uint32_t start, int fbase, int reps)
{
    const SweepArgs& a = *ap;
    if (a.pstride * int64_t(a.nfib * (K + 1)) < (int64_t(1) << 31)) {
        int jb[FT];
        group_bases<FT>(fbase, a.nfib, K + 1, 1, jb);
        if (fbase == 0)
            unit_runs_offsets<K, MODE, FT, true, PC>(a, start, jb, fbase, reps);
        else
            unit_runs_offsets<K, MODE, FT, false, PC>(a, start, jb, fbase, reps);
        return;
    }
    for (int r = 0; r < reps; ++r) {
        const uint32_t c = start + PC * (threadIdx.x + uint32_t(r) * kBatchBlock);
        if (c >= a.cells) break;
        const uint32_t line = a.fdN.div(c);
        const uint32_t ls = line * a.N;
        const uint32_t i = c - ls;
        if (i + PC <= a.N) {
            const uint32_t cls = shift_class(a, 0, line);
            if (fbase == 0)
                unit_run_body<K, MODE, FT, true, PC>(a, c, ls, i, cls, fbase);
            else
                unit_run_body<K, MODE, FT, false, PC>(a, c, ls, i, cls, fbase);
        } else {
            for (int q = 0; q < PC; ++q)
                if (c + q < a.cells) unit_cell<K, MODE, FT>(a, c + q, fbase);
        }
    }
}

// PC cells per thread: 1 (unit_item) or runs of 2 or 4 consecutive ones (unit_item_runs).
template <int K, int MODE, int FT, int PC>
__device__ __forceinline__ void unit_items(const SweepArgs* __restrict__ ap, uint32_t start, int fbase, int reps)
{
    if constexpr (PC == 2 || PC == 4)
        unit_item_runs<K, MODE, FT, PC>(ap, start, fbase, reps);
    else
        unit_item<K, MODE, FT>(ap, start, fbase, reps);
}

// At least 7 resident blocks per SM in the mixed store (at most 72 registers
// per thread, a few spilled: 4940 GB/s on the 256-problem workload against
// 4854 with 6 blocks, 4717 with 8 and 4684 with 5), 6 in the FP64 store (at 7
// its runs spill about 1 KB per thread).
template <int MODE, int FTM, int PC>
__global__ void __launch_bounds__(kBatchBlock, MODE == M_FP64 ? 6 : 7) k_batch_unit(const SweepArgs* __restrict__ args,
                                                            const int32_t* __restrict__ kdeg,
                                                            const BatchItem* __restrict__ items,
                                                            int nitems, int reps)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const SweepArgs* ap = args + item.prob;
        const int K = kdeg[item.prob];
        const int ft = (ap->nfib + ap->nfg - 1) / ap->nfg;
        const int fbase = int(item.grp) * ft;
        switch (K * 4 + ft) {
        case 1: unit_items<0, MODE, 1, PC>(ap, item.start, fbase, reps); break;
        case 5: unit_items<1, MODE, 1, PC>(ap, item.start, fbase, reps); break;
        case 9: unit_items<2, MODE, 1, PC>(ap, item.start, fbase, reps); break;
        case 6:
            if constexpr (FTM >= 2) unit_items<1, MODE, 2, PC>(ap, item.start, fbase, reps);
            break;
        case 10:
            if constexpr (FTM >= 2) unit_items<2, MODE, 2, PC>(ap, item.start, fbase, reps);
            break;
        case 11:
            if constexpr (FTM >= 3) unit_items<2, MODE, 3, PC>(ap, item.start, fbase, reps);
            break;
        default: break;
        }
    }
}

// One item along dimension m > 0: kBatchLines consecutive lines (one per
// lane) walking one chunk of rows (not inlined, as unit_item).
template <int K, int MODE, int FT, int U>
__device__ __noinline__ void strided_item(const SweepArgs* __restrict__ ap, const BatchItem item)
{
    const SweepArgs& a = *ap;
    const LineSetup L = line_setup(a, item.start + (threadIdx.x & 31u), item.grp, item.chunk, FT);
    if (L.active) strided_line<K, MODE, FT, U>(a, L);
}

// Next item of this warp from the launch's counter (lane 0 takes it, every
// lane reads it by shuffle).
__device__ __forceinline__ uint32_t next_item(uint32_t* ctr)
{
    uint32_t it = 0;
    if ((threadIdx.x & 31u) == 0) it = atomicAdd(ctr, 1u);
    return __shfl_sync(0xffffffffu, it, 0);
}

template <int MODE, int FTM, int U>
__global__ void __launch_bounds__(kBatchBlock) k_batch_strided(const SweepArgs* __restrict__ args,
                                                               const int32_t* __restrict__ kdeg,
                                                               const BatchItem* __restrict__ items,
                                                               int nitems, uint32_t* __restrict__ ctr)
{
    for (uint32_t it = next_item(ctr); it < uint32_t(nitems); it = next_item(ctr)) {
        const BatchItem item = items[it];
        const SweepArgs* ap = args + item.prob;
        const int K = kdeg[item.prob];
        const int ft = (ap->nfib + ap->nfg - 1) / ap->nfg;
        switch (K * 4 + ft) {
        case 1: strided_item<0, MODE, 1, U>(ap, item); break;
        case 5: strided_item<1, MODE, 1, U>(ap, item); break;
        case 9: strided_item<2, MODE, 1, U>(ap, item); break;
        case 6:
            if constexpr (FTM >= 2) strided_item<1, MODE, 2, U>(ap, item);
            break;
        case 10:
            if constexpr (FTM >= 2) strided_item<2, MODE, 2, U>(ap, item);
            break;
        default: break;
        }
    }
}

namespace {

template <int MODE, int FTM, int U>
cudaError_t launch_b(const SweepArgs* a, const int32_t* k, const BatchItem* items, int nitems,
                     int unit, int reps, int blocks, uint32_t* ctr, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (unit) {
        k_batch_unit<MODE, FTM, U><<<blocks, kBatchBlock, 0, st>>>(a, k, items, nitems, reps);
    } else {
        cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        k_batch_strided<MODE, FTM, U><<<blocks, kBatchBlock, 0, st>>>(a, k, items, nitems, ctr);
    }
    return cudaGetLastError();
}

template <int MODE, int FTM, int U>
int occ(int unit)
{
    int n = 0;
    cudaError_t e = unit ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_unit<MODE, FTM, U>,
                                                                         kBatchBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_strided<MODE, FTM, U>,
                                                                         kBatchBlock, 0);
    if (e != cudaSuccess) return 1;
    return n < 1 ? 1 : n;
}

}  // namespace

// Compiled shapes: dimension 0 (unit) takes ft 1..3 with unroll (cells per
// thread) 1 or 2, and ft 1..2 with 4; the other dimensions ft 1..2 with
// unroll (cells per walk step) 1, 2 or 4.
bool batch_shape_ok(int unit, int ft, int unroll)
{
    return unit ? (ft >= 1 && ft <= kBatchMaxFtUnit && (unroll == 1 || unroll == 2 || (unroll == 4 && ft <= 2)))
                : (ft >= 1 && ft <= kBatchMaxFtStrided && (unroll == 1 || unroll == 2 || unroll == 4));
}

#define SL_BATCH_SWITCH(CALL)                                                                \
    if (unit) {                                                                              \
        switch (mode * 100 + ft * 10 + unroll) {                                             \
        case M_FP64 * 100 + 11: { constexpr int MD = M_FP64, F = 1, UU = 1; CALL; }            \
        case M_FP64 * 100 + 21: { constexpr int MD = M_FP64, F = 2, UU = 1; CALL; }            \
        case M_FP64 * 100 + 31: { constexpr int MD = M_FP64, F = 3, UU = 1; CALL; }            \
        case M_FP64 * 100 + 12: { constexpr int MD = M_FP64, F = 1, UU = 2; CALL; }            \
        case M_FP64 * 100 + 22: { constexpr int MD = M_FP64, F = 2, UU = 2; CALL; }            \
        case M_FP64 * 100 + 32: { constexpr int MD = M_FP64, F = 3, UU = 2; CALL; }            \
        case M_F32 * 100 + 11: { constexpr int MD = M_F32, F = 1, UU = 1; CALL; }              \
        case M_F32 * 100 + 21: { constexpr int MD = M_F32, F = 2, UU = 1; CALL; }              \
        case M_F32 * 100 + 31: { constexpr int MD = M_F32, F = 3, UU = 1; CALL; }              \
        case M_F32 * 100 + 12: { constexpr int MD = M_F32, F = 1, UU = 2; CALL; }              \
        case M_F32 * 100 + 22: { constexpr int MD = M_F32, F = 2, UU = 2; CALL; }              \
        case M_F32 * 100 + 32: { constexpr int MD = M_F32, F = 3, UU = 2; CALL; }              \
        case M_FP64 * 100 + 14: { constexpr int MD = M_FP64, F = 1, UU = 4; CALL; }            \
        case M_FP64 * 100 + 24: { constexpr int MD = M_FP64, F = 2, UU = 4; CALL; }            \
        case M_F32 * 100 + 14: { constexpr int MD = M_F32, F = 1, UU = 4; CALL; }              \
        case M_F32 * 100 + 24: { constexpr int MD = M_F32, F = 2, UU = 4; CALL; }              \
        default: break;                                                                      \
        }                                                                                    \
    } else {                                                                                 \
        switch (mode * 100 + ft * 10 + unroll) {                                             \
        case M_FP64 * 100 + 11: { constexpr int MD = M_FP64, F = 1, UU = 1; CALL; }            \
        case M_FP64 * 100 + 12: { constexpr int MD = M_FP64, F = 1, UU = 2; CALL; }            \
        case M_FP64 * 100 + 14: { constexpr int MD = M_FP64, F = 1, UU = 4; CALL; }            \
        case M_FP64 * 100 + 21: { constexpr int MD = M_FP64, F = 2, UU = 1; CALL; }            \
        case M_FP64 * 100 + 22: { constexpr int MD = M_FP64, F = 2, UU = 2; CALL; }            \
        case M_FP64 * 100 + 24: { constexpr int MD = M_FP64, F = 2, UU = 4; CALL; }            \
        case M_F32 * 100 + 11: { constexpr int MD = M_F32, F = 1, UU = 1; CALL; }              \
        case M_F32 * 100 + 12: { constexpr int MD = M_F32, F = 1, UU = 2; CALL; }              \
        case M_F32 * 100 + 14: { constexpr int MD = M_F32, F = 1, UU = 4; CALL; }              \
        case M_F32 * 100 + 21: { constexpr int MD = M_F32, F = 2, UU = 1; CALL; }              \
        case M_F32 * 100 + 22: { constexpr int MD = M_F32, F = 2, UU = 2; CALL; }              \
        case M_F32 * 100 + 24: { constexpr int MD = M_F32, F = 2, UU = 4; CALL; }              \
        default: break;                                                                      \
        }                                                                                    \
    }

cudaError_t launch_batch_sweep(int mode, int ft, int unroll, const SweepArgs* d_args,
                               const int32_t* d_kdeg, const BatchItem* d_items, int nitems,
                               int unit, int reps, int blocks, uint32_t* d_ctr, cudaStream_t st)
{
    SL_BATCH_SWITCH(return (launch_b<MD, F, UU>(d_args, d_kdeg, d_items, nitems, unit, reps, blocks, d_ctr, st)))
    return cudaErrorInvalidValue;
}

int batch_sweep_occupancy(int mode, int ft, int unroll, int unit)
{
    SL_BATCH_SWITCH(return (occ<MD, F, UU>(unit)))
    return 1;
}

// Mass of every problem: block = problem, fixed-shape reduction.
constexpr int kBatchMassThreads = 256;

__global__ void __launch_bounds__(kBatchMassThreads) k_batch_mass(const BatchMass* __restrict__ desc,
                                                                  int parity, double* __restrict__ out)
{
    __shared__ double red[kBatchMassThreads / 32];
    const BatchMass d = desc[blockIdx.x];
    const double* mean = d.mean[parity];
    double s = 0.0;
    for (uint32_t c = threadIdx.x; c < d.cells; c += kBatchMassThreads) s += mean[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kBatchMassThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[blockIdx.x] = d.vol * s;
    }
}

cudaError_t launch_batch_mass(const BatchMass* d_desc, int nprob, int parity, double* d_out,
                              cudaStream_t st)
{
    if (nprob <= 0) return cudaSuccess;
    k_batch_mass<<<nprob, kBatchMassThreads, 0, st>>>(d_desc, parity, d_out);
    return cudaGetLastError();
}

}  // namespace sl
