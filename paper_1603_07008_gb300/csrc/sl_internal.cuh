// sl_internal.cuh -- structures shared by the sLdG device kernels and the host
// side of libsl.so.  Not part of the public ABI (include/sl.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sl {

// Storage modes, numerically equal to sl_storage.  M_F32ALL keeps every
// coefficient in FP32 ("# double" = 0 of Sec. III-A); M_SPLIT2 / M_SPLIT3 keep
// the coefficients whose every per-dimension index is below 2 / 3 in FP64 and
// the rest in FP32 ("# double" = 2, 3).
enum Mode : int { M_FP64 = 0, M_F32 = 1, M_BF16 = 2, M_FP16 = 3, M_F32ALL = 4, M_SPLIT2 = 5, M_SPLIT3 = 6 };

// FP64 indices per dimension ("# double") of a store of the split family
// below (-1 for the other stores).
__host__ __device__ constexpr int split_q(int mode)
{
    return mode == M_F32ALL ? 0 : mode == M_SPLIT2 ? 2 : mode == M_SPLIT3 ? 3 : -1;
}
// Stores whose coefficient planes are placed by a coefficient map (below).
__host__ __device__ constexpr bool is_split_family(int mode)
{
    return mode == M_F32ALL || mode == M_SPLIT2 || mode == M_SPLIT3;
}

constexpr int kMaxDim = 6;
constexpr int kMaxK = 3;
constexpr int kMaxO = kMaxK + 1;
constexpr int kMaxPolyDeg = 2 * kMaxK + 1;   // entries of A(alpha), B(alpha) are polynomials of this degree
constexpr int kMaxScaledCoef = 128;          // o^d limit of the per-cell-scaled modes (registers per thread)
constexpr int kMaxQuad = 32;

// Unsigned 32-bit division by a run-time constant d >= 1 with a multiply-high
// and a shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up variant): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l.
// The sum is formed in 64 bits, so the identity holds for every 32-bit n.
struct FastDiv {
    uint32_t d, m, l;
    FastDiv() : d(1), m(1), l(0) {}
    explicit FastDiv(uint32_t div) { set(div); }
    void set(uint32_t div)
    {
        d = div;
        l = 0;
        while ((uint64_t(1) << l) < div) ++l;
        m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - div)) / div + 1);
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const
    {
#ifdef __CUDA_ARCH__
        uint32_t t = __umulhi(n, m);
#else
        uint32_t t = uint32_t((uint64_t(n) * m) >> 32);
#endif
        return uint32_t((uint64_t(t) + n) >> l);
    }
    __host__ __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

// One split copy of the state: FP64 mean plane, low-precision planes for the
// other o^d - 1 coefficients (coefficient J >= 1 lives at hi + (J-1)*pstride),
// and the per-cell FP32 scale plane of the scaled modes.
// The general split stores (M_SPLIT2, M_SPLIT3) hold a block of FP64 planes at
// `mean` (plane 0 is the cell mean) and a block of FP32 planes at `hi`, the
// plane of coefficient J given by the coefficient map: map[J] = e >= 0 for FP32
// plane e, map[J] = -1 - e for FP64 plane e.  The all-FP32 store (M_F32ALL)
// has no FP64 plane (mean = nullptr); its o^d FP32 planes start one plane
// before `hi`, so that coefficient J is at hi + (J-1)*pstride for every J >= 0
// as in the mixed stores.
struct Planes {
    double* mean;
    void* hi;
    float* scale;
};

// Per shift class: sigma reduced into [0, N), alpha in [0,1), and the
// matrices A (first o*o) and B (next o*o), row-major, in FP64 and FP32.
// Each class's record is padded to a multiple of 16 bytes so that the sweep
// kernels read it with vector loads.
__host__ __device__ constexpr int ab_stride32(int O) { return (2 * O * O + 3) / 4 * 4; }
__host__ __device__ constexpr int ab_stride64(int O) { return (2 * O * O + 1) / 2 * 2; }

struct ShiftTable {
    const int32_t* sigma;
    const double* alpha;
    const double* ab64;   // [class][ab_stride64(o)]: A then B
    const float* ab32;    // [class][ab_stride32(o)]: A then B
};

// Geometry of one sweep along dimension `dim` of the flattened grid viewed as
// [outer][N][inner]: a line is an (outer, inner) pair, its cells are
// base + i*inner, base = outer*N*inner + inner_index.
struct SweepArgs {
    Planes src, dst;
    ShiftTable tab;
    uint32_t cells;      // < 2^31
    uint32_t N;          // extent along the sweep dimension
    uint32_t inner;      // prod_{q<dim} n_q
    uint32_t lines;      // cells / N
    int64_t pstride;     // elements between coefficient planes
    FastDiv fdN;         // divides by N   (unit-stride kernel: cell -> line)
    FastDiv fdInner;     // divides by inner (strided kernel: line -> outer)
    FastDiv fdCls;       // line coordinate -> shift class: (x / cdiv) % cmod
    FastDiv fdClsMod;
    int cls_src;         // 0: one class, 1: from the inner index, 2: from the outer index
    int ostride;         // o^dim
    int nfib;            // o^(d-1) fibres per cell
    int nfg;             // fibre groups (gridDim.y = nfg * nchunk for the strided kernel)
    uint32_t chunk;      // cells per thread along the line (strided kernel)
    const int32_t* cmap; // coefficient map of the general split stores (see Planes)
};

// Coefficient plane pointer helpers.
template <typename T>
__host__ __device__ __forceinline__ const T* plane_ptr(const void* hi, int64_t pstride, int J)
{
    return static_cast<const T*>(hi) + int64_t(J - 1) * pstride;
}
template <typename T>
__host__ __device__ __forceinline__ T* plane_ptr_w(void* hi, int64_t pstride, int J)
{
    return static_cast<T*>(hi) + int64_t(J - 1) * pstride;
}

// Launch request handed from the host side to the per-family launchers.
struct SweepLaunch {
    SweepArgs args;
    int K;
    int mode;
    int unit;            // 1: sweep along dimension 0
    int ft;              // fibres per thread (non-scaled modes)
    int unroll;          // cells per walk step of the strided kernel
    int pipeline;        // > 0: strided kernel with a cp.async ring of this many rows
    int block;           // threads per block
    int dim;             // sweep dimension
    int ndim;            // grid dimensions
    int rec;             // > 0: scaled store in cell records of this many slots
    int occ;             // > 0: the strided register walk runs at most this many blocks per SM
    cudaStream_t stream;
};

cudaError_t launch_sweep_f64(const SweepLaunch& L);      // M_FP64
cudaError_t launch_sweep_f32(const SweepLaunch& L);      // M_F32
cudaError_t launch_sweep_f32all(const SweepLaunch& L);   // M_F32ALL
cudaError_t launch_sweep_split(const SweepLaunch& L);    // M_SPLIT2, M_SPLIT3
// The stores with FP32 planes (M_F32, M_F32ALL, M_SPLIT2, M_SPLIT3) with
// every row in FP64 arithmetic; one fibre per thread (nfg = nfib).
cudaError_t launch_sweep_wide(const SweepLaunch& L);
cudaError_t launch_sweep_scaled(const SweepLaunch& L);   // M_BF16, M_FP16
// Cell records of degree 1 in 5 or 6 dimensions with G = R/16 lanes per cell,
// 16 slots (8 fibres) each (selected by fibres_per_thread == kRecLaneFt).
constexpr int kRecLaneFt = 8;
cudaError_t launch_sweep_rec_lanes(const SweepLaunch& L);

// Self-consistent field of a grid with one x and one v dimension: the
// density partial sums over chunks of kVpChunk v-rows, then E at the x-cell
// centres (and, if energy != nullptr, (1/2) sum E^2 h_x).  The cell with
// x-index i and v-index j is i * sx + j * sv.  partial holds
// vp_chunks(nv) * nx doubles.
constexpr uint32_t kVpChunk = 256;
int vp_chunks(uint32_t nv);
cudaError_t launch_vp_field(const double* mean, uint32_t nx, uint32_t nv, uint32_t sx, uint32_t sv, double hx,
                            double hv, double* partial, double* E, double* energy, cudaStream_t st);

// Coefficients of the entries of A(alpha) and B(alpha) as polynomials in
// alpha, exact rationals rounded once to FP64: a[j][l][p] alpha^p.
struct PolyTab {
    double a[kMaxO][kMaxO][kMaxPolyDeg + 1];
    double b[kMaxO][kMaxO][kMaxPolyDeg + 1];
};
void build_poly_table(int K, PolyTab* out);   // host, exact rational arithmetic

// nsteps sweeps with one shift (*shift, device) of a 1D line of N cells of the
// FP64 store by one thread-block cluster holding the line in shared memory
// (sl_sweep_1d.cu): reads src, writes the state after the last step to dst
// (src itself allowed).  sweep_1d_cluster_ok: the line fits.
size_t sweep_1d_cluster_smem(int K, uint32_t N);
bool sweep_1d_cluster_ok(int K, uint32_t N);
cudaError_t launch_sweep_1d_cluster(int K, const Planes& src, const Planes& dst, int64_t pstride, uint32_t N,
                                    const double* shift, const PolyTab& tab, int nsteps, cudaStream_t st);

// Where the shift of class c comes from.
struct ShiftSource {
    int kind;            // 0: shifts[c]; 1: (lo + (c+1/2) hv) * tau / h; 2: field[c] * tau / h
    const double* data;  // shifts (kind 0) or field samples (kind 2)
    double lo, hv, tau, h;
};

cudaError_t launch_ab_build(int K, int nclass, uint32_t N, const ShiftSource& src,
                            const PolyTab& tab, int32_t* sigma, double* alpha, double* ab64,
                            float* ab32, cudaStream_t st);

cudaError_t launch_mass(const double* mean, uint32_t cells, double* partials, int nblocks,
                        double vol, double* out, cudaStream_t st);
// The same reduction over an FP32 mean plane (the all-FP32 store).
cudaError_t launch_mass_f32(const float* mean, uint32_t cells, double* partials, int nblocks,
                            double vol, double* out, cudaStream_t st);
int mass_blocks(uint32_t cells);

struct CodecArgs {
    Planes p;
    int64_t pstride;
    int ncoef;
    int mode;
    int rec;             // > 0: higher coefficients in cell records of rec slots (slot J = coefficient J)
    const int32_t* cmap; // general split and all-FP32 stores: coefficient map, with p.hi the
                         // start of the FP32 block (see Planes)
};

// Address of coefficient J >= 1 of a cell, planar or in records.
template <typename T>
__host__ __device__ __forceinline__ T* coef_ptr(const CodecArgs& c, int J, uint32_t cell)
{
    return c.rec ? static_cast<T*>(c.p.hi) + size_t(cell) * c.rec + J
                 : static_cast<T*>(c.p.hi) + int64_t(J - 1) * c.pstride + cell;
}
cudaError_t launch_encode(const CodecArgs& c, const double* aos, uint32_t first, uint32_t count,
                          cudaStream_t st);
cudaError_t launch_decode(const CodecArgs& c, double* aos, uint32_t first, uint32_t count,
                          cudaStream_t st);
cudaError_t launch_gather(const CodecArgs& c, const int64_t* cells, uint32_t count, double* aos,
                          cudaStream_t st);

struct ProjectArgs {
    int ndim, K, nq, nterms;
    uint32_t n[kMaxDim];
    double lo[kMaxDim], h[kMaxDim];
    double node[kMaxQuad], weight[kMaxQuad];
};
cudaError_t launch_project(const ProjectArgs& pa, const double* d_weights, const double* d_params,
                           double* d_tab, uint32_t nmax, const CodecArgs& c, uint32_t cells,
                           cudaStream_t st);

// ---------------------------------------------------------------- batches

// One work item of a batched sweep: a block's threads cover `reps` tiles of
// `kBatchBlock` consecutive cells (sweep along dimension 0), or a warp's
// lanes `kBatchLines` consecutive lines walking one chunk of rows (other
// dimensions), starting at `start` of problem `prob`, for fibre group `grp`.
constexpr int kBatchBlock = 128;
constexpr int kBatchLines = 32;
constexpr int kBatchMaxK = 2;          // degrees compiled into the batched sweep
constexpr int kBatchMaxFtUnit = 3;     // fibres per thread compiled along dimension 0
constexpr int kBatchMaxFtStrided = 2;  // ... and along the other dimensions
struct BatchItem {
    uint32_t prob;
    uint32_t start;
    uint32_t grp;
    uint32_t chunk;
};

// Per (problem, sweep dimension): where the shifts of its classes come from
// and where its table goes.
struct BatchAB {
    int K;
    uint32_t N;
    int nclass;
    int kind;              // 1: cell-centre velocity of a v-dimension, 2: field samples
    const double* field;
    double lo, hv, h;
    int32_t* sigma;
    double* alpha;
    double* ab64;
    float* ab32;
};

struct BatchMass {
    const double* mean[2];   // mean plane of each copy
    uint32_t cells;
    double vol;
};

cudaError_t launch_batch_ab(const BatchAB* d_desc, const PolyTab* d_tabs, int nprob, int maxclass,
                            double tau, cudaStream_t st);
// unit = 1: sweep along dimension 0, each item covering reps * kBatchBlock
// cells.  ft is the most fibres per thread (each problem's own is
// ceil(nfib / nfg) of its arguments).  Along the other dimensions the warps
// take items from *d_ctr, which the launch first sets to zero.
cudaError_t launch_batch_sweep(int mode, int ft, int unroll, const SweepArgs* d_args,
                               const int32_t* d_kdeg, const BatchItem* d_items, int nitems,
                               int unit, int reps, int blocks, uint32_t* d_ctr, cudaStream_t st);
bool batch_shape_ok(int unit, int ft, int unroll);
// Resident blocks per SM of the batched sweep kernel for (mode, ft, unroll).
int batch_sweep_occupancy(int mode, int ft, int unroll, int unit);
cudaError_t launch_batch_mass(const BatchMass* d_desc, int nprob, int parity, double* d_out,
                              cudaStream_t st);

}  // namespace sl
