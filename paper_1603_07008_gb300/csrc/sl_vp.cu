// sl_vp.cu -- self-consistent field of the 1+1-dimensional Vlasov equation
// d_t f + v d_x f + E(x) d_v f = 0 (Sec. II), closed by the Poisson equation
// d_x E = rho - rho_bar with rho(x) = int f dv and rho_bar its mean over the
// periodic x-domain.  E is needed at the x-cell centres, where the v-sweep
// takes its shifts.
//
// rho_i = h_v sum_j c0(i, j) is the x-cell average of the density (c0, the
// cell mean, integrates to h_v times itself over a v-cell).  With
// q_i = (rho_i - rho_bar) h_x, the field of the piecewise-constant density at
// the centre of cell i is sum_{j<i} q_j + q_i / 2, up to the constant fixed by
// int E dx = 0, which is subtracted.  Every sum runs in a fixed order that
// depends only on the grid, so the field is the same on every run.
#include "sl_internal.cuh"

#include <cooperative_groups.h>

namespace sl {

namespace {

namespace cg = cooperative_groups;

// The field kernel runs as one cluster of kVpCluster blocks of kVpThreads:
// each block takes a segment of the x-cells, and the blocks exchange their
// segment sums through distributed shared memory.  One block alone is bound
// by its SM's FP64 pipe (about 60 FP64 operations per thread at 2 per clock).
constexpr int kVpCluster = 8;
constexpr int kVpThreads = 512;

// Partial density sums over chunks of v-rows: block (32, 8) over 32 x-cells
// and one chunk of kVpChunk rows; thread (tx, ty) adds rows ty, ty + 8, ...
__global__ void __launch_bounds__(256) k_vp_density(const double* __restrict__ mean, uint32_t nx, uint32_t nv,
                                                    uint32_t sx, uint32_t sv, double* __restrict__ partial)
{
    __shared__ double part[8][32];
    const uint32_t i = blockIdx.x * 32 + threadIdx.x;
    const uint32_t j0 = blockIdx.y * kVpChunk;
    const uint32_t j1 = min(j0 + kVpChunk, nv);
    double s = 0.0;
    if (i < nx)
        for (uint32_t j = j0 + threadIdx.y; j < j1; j += 8) s += mean[size_t(i) * sx + size_t(j) * sv];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && i < nx) {
        double t = 0.0;
#pragma unroll
        for (int y = 0; y < 8; ++y) t += part[y][threadIdx.x];
        partial[size_t(blockIdx.y) * nx + i] = t;
    }
}

// Sum of one value per thread over the block, in a fixed tree order; every
// thread receives the result.
__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int off = kVpThreads / 2; off > 0; off >>= 1) {
        if (int(threadIdx.x) < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Sum over the cluster of one value per block (v on thread 0 of each block),
// in block-rank order, so every block gets the same bits; slot is this
// block's exchange cell.  Every thread of every block receives the sum.
__device__ double cluster_sum(cg::cluster_group& cl, double v, double* slot, double* bcast)
{
    if (threadIdx.x == 0) *slot = v;
    cl.sync();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < kVpCluster; ++r) t += *cl.map_shared_rank(slot, r);
        *bcast = t;
    }
    cl.sync();   // every block has read every slot before the next write
    return *bcast;
}

// Exclusive prefix over the cluster's blocks of one value per block (on
// thread 0), in rank order.
__device__ double cluster_prefix(cg::cluster_group& cl, double v, double* slot, double* bcast)
{
    if (threadIdx.x == 0) *slot = v;
    cl.sync();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < int(cl.block_rank()); ++r) t += *cl.map_shared_rank(slot, r);
        *bcast = t;
    }
    cl.sync();
    return *bcast;
}

// One cluster: density from the partial sums, the field at the cell centres
// into E[nx], and the field energy (1/2) sum E_i^2 h_x into *energy.  Block r
// of the cluster takes the x-cells [r P, (r + 1) P), P = ceil(nx / blocks),
// in thread segments of S cells.
__global__ void __cluster_dims__(kVpCluster, 1, 1) __launch_bounds__(kVpThreads)
    k_vp_field(const double* __restrict__ partial, uint32_t nx, int nchunk, double hx, double hv,
               double* __restrict__ E, double* __restrict__ energy)
{
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double red[kVpThreads];
    __shared__ double seg[kVpThreads];
    __shared__ double slot, bcast;
    const uint32_t P = (nx + kVpCluster - 1) / kVpCluster;
    const uint32_t c0 = min(uint32_t(cl.block_rank()) * P, nx), c1 = min(c0 + P, nx);
    const uint32_t S = (c1 - c0 + kVpThreads - 1) / kVpThreads;   // cells per thread segment
    const uint32_t b0 = min(c0 + threadIdx.x * S, c1), b1 = min(b0 + S, c1);
    // rho_i into E[i]; the block's share of sum rho
    double local = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        double r = 0.0;
        for (int c = 0; c < nchunk; ++c) r += partial[size_t(c) * nx + i];
        r *= hv;
        E[i] = r;
        local += r;
    }
    const double rho_bar = cluster_sum(cl, block_sum(local, red), &slot, &bcast) / double(nx);
    // q_i = (rho_i - rho_bar) h_x and the sum over the thread's segment
    double ssum = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double q = (E[i] - rho_bar) * hx;
        E[i] = q;
        ssum += q;
    }
    // inclusive scan of the segment sums in the block (Hillis-Steele, a fixed
    // order of additions), the blocks before this one, then the exclusive
    // prefix of this thread's segment
    seg[threadIdx.x] = ssum;
    __syncthreads();
    for (int off = 1; off < kVpThreads; off <<= 1) {
        const double add = int(threadIdx.x) >= off ? seg[threadIdx.x - off] : 0.0;
        __syncthreads();
        seg[threadIdx.x] += add;
        __syncthreads();
    }
    const double before = cluster_prefix(cl, seg[kVpThreads - 1], &slot, &bcast);
    double run = threadIdx.x > 0 ? before + seg[threadIdx.x - 1] : before;
    double esum = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double q = E[i];
        const double e = run + 0.5 * q;
        run += q;
        E[i] = e;
        esum += e;
    }
    const double e_bar = cluster_sum(cl, block_sum(esum, red), &slot, &bcast) / double(nx);
    double w = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double e = E[i] - e_bar;
        E[i] = e;
        w += e * e;
    }
    const double W = cluster_sum(cl, block_sum(w, red), &slot, &bcast);
    if (cl.block_rank() == 0 && threadIdx.x == 0 && energy) *energy = 0.5 * hx * W;
}

}  // namespace

int vp_chunks(uint32_t nv) { return int((nv + kVpChunk - 1) / kVpChunk); }

cudaError_t launch_vp_field(const double* mean, uint32_t nx, uint32_t nv, uint32_t sx, uint32_t sv, double hx,
                            double hv, double* partial, double* E, double* energy, cudaStream_t st)
{
    const int nchunk = vp_chunks(nv);
    k_vp_density<<<dim3((nx + 31) / 32, nchunk), dim3(32, 8), 0, st>>>(mean, nx, nv, sx, sv, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_vp_field<<<kVpCluster, kVpThreads, 0, st>>>(partial, nx, nchunk, hx, hv, E, energy);
    return cudaGetLastError();
}

}  // namespace sl
