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

namespace sl {

namespace {

constexpr int kVpThreads = 1024;

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

// One block: density from the partial sums, the field at the cell centres
// into E[nx], and the field energy (1/2) sum E_i^2 h_x into *energy.
__global__ void __launch_bounds__(kVpThreads) k_vp_field(const double* __restrict__ partial, uint32_t nx,
                                                         int nchunk, double hx, double hv, double* __restrict__ E,
                                                         double* __restrict__ energy)
{
    __shared__ double red[kVpThreads];
    __shared__ double seg[kVpThreads];
    const uint32_t S = (nx + kVpThreads - 1) / kVpThreads;   // cells per thread segment
    const uint32_t b0 = threadIdx.x * S, b1 = min(b0 + S, nx);
    // rho_i into E[i]; the thread's share of sum rho
    double local = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        double r = 0.0;
        for (int c = 0; c < nchunk; ++c) r += partial[size_t(c) * nx + i];
        r *= hv;
        E[i] = r;
        local += r;
    }
    const double rho_bar = block_sum(local, red) / double(nx);
    // q_i = (rho_i - rho_bar) h_x and the sum over the thread's segment
    double ssum = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double q = (E[i] - rho_bar) * hx;
        E[i] = q;
        ssum += q;
    }
    // inclusive scan of the segment sums (Hillis-Steele, a fixed order of
    // additions), then the exclusive prefix of this thread's segment
    seg[threadIdx.x] = ssum;
    __syncthreads();
    for (int off = 1; off < kVpThreads; off <<= 1) {
        const double add = int(threadIdx.x) >= off ? seg[threadIdx.x - off] : 0.0;
        __syncthreads();
        seg[threadIdx.x] += add;
        __syncthreads();
    }
    double run = threadIdx.x > 0 ? seg[threadIdx.x - 1] : 0.0;
    double esum = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double q = E[i];
        const double e = run + 0.5 * q;
        run += q;
        E[i] = e;
        esum += e;
    }
    const double e_bar = block_sum(esum, red) / double(nx);
    double w = 0.0;
    for (uint32_t i = b0; i < b1; ++i) {
        const double e = E[i] - e_bar;
        E[i] = e;
        w += e * e;
    }
    const double W = block_sum(w, red);
    if (threadIdx.x == 0 && energy) *energy = 0.5 * hx * W;
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
    k_vp_field<<<1, kVpThreads, 0, st>>>(partial, nx, nchunk, hx, hv, E, energy);
    return cudaGetLastError();
}

}  // namespace sl
