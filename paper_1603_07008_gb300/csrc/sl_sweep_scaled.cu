// sl_sweep_scaled.cu -- instantiations and launcher of the sweep kernels for
// the FP64-mean / per-cell-scaled BF16 or FP16 store.  The new scale is the
// maximum over the whole cell, so one thread holds every fibre of its cell
// (up to 16 values) or G threads share it through shared memory; the fibre
// count o^(d-1) is therefore a template parameter.
#include "sl_sweep.cuh"

namespace sl {

namespace {

// Cells are shared by G threads of NF/G fibres each when the launch asks for
// fewer fibres per thread than the cell has (G is a power of o, so it
// divides the fibre count); otherwise one thread holds the whole cell.
template <int K, int MODE, int NF, int G>
cudaError_t launch_coop(const SweepLaunch& L)
{
    const SweepArgs& a = L.args;
    if (a.nfib != NF || a.nfg != 1) return cudaErrorInvalidValue;
    const dim3 block(32, G);
    if (L.unit) {
        k_sweep_unit_coop<K, MODE, NF, G><<<dim3((a.cells + 31) / 32), block, 0, L.stream>>>(a);
    } else {
        const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
        k_sweep_strided_coop<K, MODE, NF, G><<<dim3((a.lines + 31) / 32, nchunk), block, 0, L.stream>>>(a);
    }
    return cudaGetLastError();
}

template <int K, int MODE, int NF>
cudaError_t launch_one(const SweepLaunch& L)
{
    if (L.ft != NF) {
        const int G = NF / (L.ft > 0 ? L.ft : 1);
        if (G * L.ft != NF) return cudaErrorInvalidValue;
        if constexpr (K == 1 && NF == 32) {
            if (G == 2) return launch_coop<K, MODE, NF, 2>(L);
            if (G == 4) return launch_coop<K, MODE, NF, 4>(L);
            if (G == 8) return launch_coop<K, MODE, NF, 8>(L);
        }
        if constexpr (K == 1 && NF == 16) {
            if (G == 2) return launch_coop<K, MODE, NF, 2>(L);
            if (G == 4) return launch_coop<K, MODE, NF, 4>(L);
        }
        if constexpr (K == 2 && NF == 27) {
            if (G == 3) return launch_coop<K, MODE, NF, 3>(L);
            if (G == 9) return launch_coop<K, MODE, NF, 9>(L);
        }
        if constexpr (K == 2 && NF == 9) {
            if (G == 3) return launch_coop<K, MODE, NF, 3>(L);
        }
        if constexpr (K == 3 && NF == 16) {
            if (G == 4) return launch_coop<K, MODE, NF, 4>(L);
        }
        return cudaErrorInvalidValue;
    }
    const SweepArgs& a = L.args;
    if (a.nfib != NF || a.nfg != 1) return cudaErrorInvalidValue;
    if (L.unit) {
        dim3 grid((a.cells + L.block - 1) / L.block, 1);
        k_sweep_unit<K, MODE, NF, false><<<grid, L.block, 0, L.stream>>>(a);
    } else {
        const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
        dim3 grid((a.lines + L.block - 1) / L.block, nchunk);
        // two cells per walk step while the per-thread cell stays small
        constexpr int U = NF * (K + 1) <= 16 ? 2 : 1;
        k_sweep_strided<K, MODE, NF, U><<<grid, L.block, 0, L.stream>>>(a);
    }
    return cudaGetLastError();
}

// Cell-record layout (shapes whose records are nearly full): the sweep
// dimension is a template parameter of the strided kernel.
template <int K, int MODE, int D, int M>
cudaError_t launch_rec_walk(const SweepLaunch& L, dim3 grid)
{
    switch (L.unroll) {
    case 1: k_sweep_strided_rec<K, MODE, D, M, false><<<grid, L.block, 0, L.stream>>>(L.args); break;
    case 2: k_sweep_strided_rec<K, MODE, D, M, true><<<grid, L.block, 0, L.stream>>>(L.args); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Along dimension 0 the cells are either one thread each (chunk 0) or walked
// like the other dimensions (chunk > 0).  unroll: 1 plain, 2 prefetching
// walk.
template <int K, int MODE, int D>
cudaError_t launch_rec(const SweepLaunch& L)
{
    const SweepArgs& a = L.args;
    if (L.block > 128 || L.ndim != D || L.rec != RecShape<K, D>::R || L.dim >= D) return cudaErrorInvalidValue;
    if (L.unit && a.chunk == 0) {
        k_sweep_unit_rec<K, MODE, D><<<(a.cells + L.block - 1) / L.block, L.block, 0, L.stream>>>(a);
        return cudaGetLastError();
    }
    const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
    const dim3 grid((a.lines + L.block - 1) / L.block, nchunk);
    switch (L.dim) {
    case 0: return launch_rec_walk<K, MODE, D, 0>(L, grid);
    case 1: return launch_rec_walk<K, MODE, D, 1>(L, grid);
    case 2: return launch_rec_walk<K, MODE, D, 2>(L, grid);
    case 3:
        if constexpr (D > 3) return launch_rec_walk<K, MODE, D, 3>(L, grid);
        break;
    case 4:
        if constexpr (D > 4) return launch_rec_walk<K, MODE, D, 4>(L, grid);
        break;
    case 5:
        if constexpr (D > 5) return launch_rec_walk<K, MODE, D, 5>(L, grid);
        break;
    }
    return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_mode(const SweepLaunch& L)
{
    if (L.rec) {
        if (L.K == 1 && (L.ndim == 5 || L.ndim == 6) && L.ft == kRecLaneFt) return launch_sweep_rec_lanes(L);
        if (L.K == 1 && L.ndim == 6) return launch_rec<1, MODE, 6>(L);
        if (L.K == 1 && L.ndim == 5) return launch_rec<1, MODE, 5>(L);
        if (L.K == 3 && L.ndim == 3) return launch_rec<3, MODE, 3>(L);
        return cudaErrorInvalidValue;
    }
    const int nf = L.args.nfib;
    switch (L.K) {
    case 0:
        if (nf == 1) return launch_one<0, MODE, 1>(L);
        break;
    case 1:
        switch (nf) {
        case 1: return launch_one<1, MODE, 1>(L);
        case 2: return launch_one<1, MODE, 2>(L);
        case 4: return launch_one<1, MODE, 4>(L);
        case 8: return launch_one<1, MODE, 8>(L);
        case 16: return launch_one<1, MODE, 16>(L);
        case 32: return launch_one<1, MODE, 32>(L);
        }
        break;
    case 2:
        switch (nf) {
        case 1: return launch_one<2, MODE, 1>(L);
        case 3: return launch_one<2, MODE, 3>(L);
        case 9: return launch_one<2, MODE, 9>(L);
        case 27: return launch_one<2, MODE, 27>(L);
        }
        break;
    case 3:
        switch (nf) {
        case 1: return launch_one<3, MODE, 1>(L);
        case 4: return launch_one<3, MODE, 4>(L);
        case 16: return launch_one<3, MODE, 16>(L);
        }
        break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sweep_scaled(const SweepLaunch& L)
{
    if (L.mode == M_BF16) return launch_mode<M_BF16>(L);
    if (L.mode == M_FP16) return launch_mode<M_FP16>(L);
    return cudaErrorInvalidValue;
}

}  // namespace sl
