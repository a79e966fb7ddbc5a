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
    const int b = 128;
    dim3 grid((maxclass + b - 1) / b, nprob);
    k_batch_ab<<<grid, b, 0, st>>>(d_desc, d_tabs, tau);
    return cudaGetLastError();
}

// Persistent sweep over a work list: each block takes items blockIdx.x,
// blockIdx.x + gridDim.x, ...; every thread reads the problem's sweep
// geometry straight from the (read-only, L1-cached) argument array, so items
// need no block barrier, and the problem's degree (0, 1 or 2) selects the
// compiled variant (uniform across the block).  The loop is bounded by the
// item count; no block waits on another.  Sweeps along dimension 0 and along
// the other dimensions are separate kernels, so each has its own register
// budget.
template <int MODE, int FT>
__global__ void __launch_bounds__(kBatchBlock) k_batch_unit(const SweepArgs* __restrict__ args,
                                                            const int32_t* __restrict__ kdeg,
                                                            const BatchItem* __restrict__ items,
                                                            int nitems, int reps)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const SweepArgs a = args[item.prob];
        const int K = kdeg[item.prob];
        const int fbase = int(item.grp) * FT;
        // reps tiles of kBatchBlock consecutive cells
        for (int r = 0; r < reps; ++r) {
            const uint32_t c = item.start + threadIdx.x + uint32_t(r) * kBatchBlock;
            if (c >= a.cells) break;
            switch (K) {
            case 0: unit_cell<0, MODE, FT>(a, c, fbase); break;
            case 1: unit_cell<1, MODE, FT>(a, c, fbase); break;
            default: unit_cell<2, MODE, FT>(a, c, fbase); break;
            }
        }
    }
}

template <int MODE, int FT, int U>
__global__ void __launch_bounds__(kBatchBlock) k_batch_strided(const SweepArgs* __restrict__ args,
                                                               const int32_t* __restrict__ kdeg,
                                                               const BatchItem* __restrict__ items,
                                                               int nitems)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const SweepArgs a = args[item.prob];
        const int K = kdeg[item.prob];
        const LineSetup L = line_setup(a, item.start + threadIdx.x, item.grp, item.chunk, FT);
        if (L.active) {
            switch (K) {
            case 0: strided_line<0, MODE, FT, U>(a, L); break;
            case 1: strided_line<1, MODE, FT, U>(a, L); break;
            default: strided_line<2, MODE, FT, U>(a, L); break;
            }
        }
    }
}

namespace {

template <int MODE, int FT, int U>
cudaError_t launch_b(const SweepArgs* a, const int32_t* k, const BatchItem* items, int nitems,
                     int unit, int reps, int blocks, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (unit)
        k_batch_unit<MODE, FT><<<blocks, kBatchBlock, 0, st>>>(a, k, items, nitems, reps);
    else
        k_batch_strided<MODE, FT, U><<<blocks, kBatchBlock, 0, st>>>(a, k, items, nitems);
    return cudaGetLastError();
}

template <int MODE, int FT, int U>
int occ(int unit)
{
    int n = 0;
    cudaError_t e = unit ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_unit<MODE, FT>,
                                                                         kBatchBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_strided<MODE, FT, U>,
                                                                         kBatchBlock, 0);
    if (e != cudaSuccess) return 1;
    return n < 1 ? 1 : n;
}

}  // namespace

#define SL_BATCH_SWITCH(CALL)                                                   \
    switch (mode * 100 + ft * 10 + unroll) {                                    \
    case M_FP64 * 100 + 11: { constexpr int MD = M_FP64, F = 1, UU = 1; CALL; } \
    case M_FP64 * 100 + 14: { constexpr int MD = M_FP64, F = 1, UU = 4; CALL; } \
    case M_FP64 * 100 + 21: { constexpr int MD = M_FP64, F = 2, UU = 1; CALL; } \
    case M_FP64 * 100 + 24: { constexpr int MD = M_FP64, F = 2, UU = 4; CALL; } \
    case M_F32 * 100 + 11: { constexpr int MD = M_F32, F = 1, UU = 1; CALL; }   \
    case M_F32 * 100 + 14: { constexpr int MD = M_F32, F = 1, UU = 4; CALL; }   \
    case M_F32 * 100 + 21: { constexpr int MD = M_F32, F = 2, UU = 1; CALL; }   \
    case M_F32 * 100 + 24: { constexpr int MD = M_F32, F = 2, UU = 4; CALL; }   \
    default: break;                                                             \
    }

cudaError_t launch_batch_sweep(int mode, int ft, int unroll, const SweepArgs* d_args,
                               const int32_t* d_kdeg, const BatchItem* d_items, int nitems,
                               int unit, int reps, int blocks, cudaStream_t st)
{
    SL_BATCH_SWITCH(return (launch_b<MD, F, UU>(d_args, d_kdeg, d_items, nitems, unit, reps, blocks, st)))
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
