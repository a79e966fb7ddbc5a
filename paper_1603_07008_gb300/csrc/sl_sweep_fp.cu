// sl_sweep_fp.cu -- instantiations and launcher of the sweep kernels for the
// FP64 store and the mixed FP64-mean / FP32 store.
#include "sl_sweep.cuh"

namespace sl {

namespace {

template <int K, int MODE, int FT>
cudaError_t launch_one(const SweepLaunch& L)
{
    const SweepArgs& a = L.args;
    if (L.unit) {
        dim3 grid((a.cells + L.block - 1) / L.block, a.nfg);
        k_sweep_unit<K, MODE, FT><<<grid, L.block, 0, L.stream>>>(a);
    } else {
        const uint32_t nchunk = (a.N + a.chunk - 1) / a.chunk;
        dim3 grid((a.lines + L.block - 1) / L.block, nchunk * a.nfg);
        k_sweep_strided<K, MODE, FT><<<grid, L.block, 0, L.stream>>>(a);
    }
    return cudaGetLastError();
}

template <int K, int MODE>
cudaError_t launch_ft(const SweepLaunch& L)
{
    switch (L.ft) {
    case 1: return launch_one<K, MODE, 1>(L);
    case 4: return launch_one<K, MODE, 4>(L);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t launch_k(const SweepLaunch& L)
{
    switch (L.K) {
    case 0: return launch_ft<0, MODE>(L);
    case 1: return launch_ft<1, MODE>(L);
    case 2: return launch_ft<2, MODE>(L);
    case 3: return launch_ft<3, MODE>(L);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_sweep_fp(const SweepLaunch& L)
{
    if (L.mode == M_FP64) return launch_k<M_FP64>(L);
    if (L.mode == M_F32) return launch_k<M_F32>(L);
    return cudaErrorInvalidValue;
}

}  // namespace sl
