// sl_sweep_1d.cu -- nsteps sweeps of one short periodic 1D line of the FP64
// store by one thread-block cluster that keeps the line in shared memory.
//
// The 1D advection of Sec. II with a constant shift s (in cells) applies the
// update rule of Sec. II-A, c'_i = A(alpha) c_{i-sigma} + B(alpha)
// c_{i-sigma-1}, at every step.  For a line of a few thousand cells each
// sweep is a few microseconds of launch overhead around well under a
// microsecond of work, so here the cluster's kC blocks hold the line (block r
// cells [r P, (r + 1) P), P = ceil(N / kC)) in two shared-memory copies and
// run all the steps in one launch: at every step each block builds the
// step's A and B from the shift (the same Horner evaluation of the projection
// polynomials as the table kernel, so the same bits), each thread updates its
// target cells reading the two source cells from whichever block holds them
// (distributed shared memory), and a cluster barrier ends the step.  Every
// cell is computed with the same operations in the same order as by the
// one-sweep-per-launch kernels, so the results are the same bits.
#include "sl_sweep.cuh"

#include <cooperative_groups.h>

namespace sl {

namespace {

namespace cg = cooperative_groups;

constexpr int kC1d = 8;     // blocks of the cluster
constexpr int kT1d = 128;   // threads per block

template <int K>
__global__ void __cluster_dims__(kC1d, 1, 1) __launch_bounds__(kT1d)
    k_sweep_1d_cluster(const Planes src, const Planes dst, int64_t pstride, uint32_t N,
                       const double* __restrict__ shift, const PolyTab tab, int nsteps)
{
    constexpr int O = K + 1;
    constexpr int deg = 2 * K + 1;
    extern __shared__ double sm[];   // two copies [O][P] of the block's cells, then A[O][O], B[O][O]
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t P = (N + kC1d - 1) / kC1d;
    const uint32_t c0 = uint32_t(cl.block_rank()) * P;
    const size_t csz = size_t(O) * P;   // copy q of the block's cells at sm + q * csz
    double* tA = sm + 2 * csz;
    double* tB = tA + O * O;
    for (uint32_t q = threadIdx.x; q < P; q += kT1d) {
        const uint32_t i = c0 + q;
        if (i >= N) break;
        sm[q] = src.mean[i];
#pragma unroll
        for (int l = 1; l < O; ++l) sm[size_t(l) * P + q] = plane_ptr<double>(src.hi, pstride, l)[i];
    }
    cl.sync();
    int cur = 0;
    for (int step = 0; step < nsteps; ++step) {
        // this step's shift split and matrices (the table kernel's operations)
        const double s = __ldg(shift);
        const double f = floor(s);
        double alpha = s - f;
        long long sg = (long long)f;
        if (alpha >= 1.0) {
            sg += 1;
            alpha = 0.0;
        }
        long long rr = sg % (long long)N;
        if (rr < 0) rr += N;
        const int32_t sig = int32_t(rr);
        if (threadIdx.x < 2 * O * O) {
            const int e = int(threadIdx.x) % (O * O);
            const int j = e / O, l = e % O;
            const bool isb = int(threadIdx.x) >= O * O;
            double v;
            if (alpha == 0.0) {
                v = isb ? 0.0 : (j == l ? 1.0 : 0.0);
            } else {
                const double t = alpha - 0.5;
                v = isb ? tab.b[j][l][deg] : tab.a[j][l][deg];
#pragma unroll
                for (int p = deg - 1; p >= 0; --p) v = fma(v, t, isb ? tab.b[j][l][p] : tab.a[j][l][p]);
            }
            (isb ? tB : tA)[e] = v;
        }
        __syncthreads();
        Mats<K, M_FP64> M;
#pragma unroll
        for (int j = 0; j < O; ++j)
#pragma unroll
            for (int l = 0; l < O; ++l) {
                M.a[j][l] = tA[j * O + l];
                M.b[j][l] = tB[j * O + l];
            }
#pragma unroll
        for (int l = 0; l < O; ++l) {
            M.a0[l] = tA[l];
            M.aj0[l] = tA[l * O];
        }
        M.alpha = alpha;
        const double* in = sm + cur * csz;
        double* out = sm + (cur ^ 1) * csz;
        for (uint32_t q = threadIdx.x; q < P; q += kT1d) {
            const uint32_t i = c0 + q;
            if (i >= N) break;
            int32_t ia = int32_t(i) - sig;
            ia += ia < 0 ? int32_t(N) : 0;
            int32_t ib = ia - 1;
            ib += ib < 0 ? int32_t(N) : 0;
            const double* pa = cl.map_shared_rank(in, uint32_t(ia) / P) + uint32_t(ia) % P;
            const double* pb = cl.map_shared_rank(in, uint32_t(ib) / P) + uint32_t(ib) % P;
            CellVals<K, M_FP64, 1> va, vb, vo;
            va.m = pa[0];
            vb.m = pb[0];
            va.v[0][0] = 0.0;
            vb.v[0][0] = 0.0;
#pragma unroll
            for (int l = 1; l < O; ++l) {
                va.v[0][l] = pa[size_t(l) * P];
                vb.v[0][l] = pb[size_t(l) * P];
            }
            combine<K, M_FP64, 1, true>(M, va, vb, vo);
            out[q] = vo.m;
#pragma unroll
            for (int l = 1; l < O; ++l) out[size_t(l) * P + q] = vo.v[0][l];
        }
        cl.sync();   // every block's reads of `in` are done before it is written again
        cur ^= 1;
    }
    for (uint32_t q = threadIdx.x; q < P; q += kT1d) {
        const uint32_t i = c0 + q;
        if (i >= N) break;
        const double* fin = sm + cur * csz;
        dst.mean[i] = fin[q];
#pragma unroll
        for (int l = 1; l < O; ++l) plane_ptr_w<double>(dst.hi, pstride, l)[i] = fin[size_t(l) * P + q];
    }
}

template <int K>
cudaError_t launch_1d(const Planes& src, const Planes& dst, int64_t pstride, uint32_t N, const double* shift,
                      const PolyTab& tab, int nsteps, cudaStream_t st)
{
    const size_t smem = sweep_1d_cluster_smem(K, N);
    k_sweep_1d_cluster<K><<<kC1d, kT1d, smem, st>>>(src, dst, pstride, N, shift, tab, nsteps);
    return cudaGetLastError();
}

}  // namespace

size_t sweep_1d_cluster_smem(int K, uint32_t N)
{
    const size_t O = size_t(K) + 1;
    const size_t P = (size_t(N) + kC1d - 1) / kC1d;
    return (2 * O * P + 2 * O * O) * sizeof(double);
}

bool sweep_1d_cluster_ok(int K, uint32_t N)
{
    return K >= 0 && K <= kMaxK && N >= 1 && sweep_1d_cluster_smem(K, N) <= 48 * 1024;
}

cudaError_t launch_sweep_1d_cluster(int K, const Planes& src, const Planes& dst, int64_t pstride, uint32_t N,
                                    const double* shift, const PolyTab& tab, int nsteps, cudaStream_t st)
{
    if (!sweep_1d_cluster_ok(K, N) || nsteps < 1) return cudaErrorInvalidValue;
    switch (K) {
    case 0: return launch_1d<0>(src, dst, pstride, N, shift, tab, nsteps, st);
    case 1: return launch_1d<1>(src, dst, pstride, N, shift, tab, nsteps, st);
    case 2: return launch_1d<2>(src, dst, pstride, N, shift, tab, nsteps, st);
    case 3: return launch_1d<3>(src, dst, pstride, N, shift, tab, nsteps, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sl
