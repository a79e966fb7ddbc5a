// sl_host.h -- host-side internals of libsl.so shared by the single-problem
// API (sl_api.cu) and the batched API (sl_batch_api.cu).  Not part of the
// public ABI (include/sl.h is).
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sl.h"
#include "sl_internal.cuh"

// One problem: its grid, store, ping-pong state, shift tables and launch shapes.
struct sl_ctx {
    sl_grid g{};
    int K = 0, O = 1, ndim = 1;
    sl::Mode mode = sl::M_FP64;
    cudaStream_t st = nullptr;
    int64_t cells = 0, ncoef = 1, pstride = 0, nfib = 1;
    int rec = 0;                // > 0: scaled store in cell records of rec 16-bit slots
    int sm_count = 0;           // multiprocessors of the context's device
    size_t elem = 8;            // bytes of a low-precision (hi) element
    int64_t nlo = 1, nhi = 0;   // FP64 planes (the mean's block) and hi planes of one copy
    int32_t* d_cmap = nullptr;  // coefficient map of the stores that use one (see sl::Planes)
    int64_t state_bytes = 0;

    void* mem = nullptr;
    size_t mem_bytes = 0;
    // canaries: guard bands after every array of the allocation, and the
    // padding of the owned planes past `cells` (offsets into mem)
    struct Band {
        size_t off, pitch, width, height;   // height rows of width bytes, pitch apart
    };
    std::vector<Band> bands;
    sl::Planes planes[2]{};
    bool external = false;      // planes owned by the caller (sl_create_external)
    int cur = 0;

    // shift tables, one per sweep dimension m with ncls[m] classes (the
    // extent of the largest other dimension, at least 1: a line's shift
    // depends on one orthogonal coordinate), so that the tables of a split
    // step can be built ahead of their sweeps
    int ncls[SL_MAX_DIM] = {0};
    int maxcls = 1;             // max over m: host shifts staged in d_shifts
    int32_t* d_sigma[SL_MAX_DIM] = {nullptr};
    double* d_alpha[SL_MAX_DIM] = {nullptr};
    double* d_ab64[SL_MAX_DIM] = {nullptr};
    float* d_ab32[SL_MAX_DIM] = {nullptr};
    // side stream of the v-dimensions' table builds, forked from and joined
    // back to st by the two events within every split step
    cudaStream_t st_tab = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double* d_shifts = nullptr;
    double* d_fields = nullptr;
    int64_t nfields = 0;
    bool fields_set = false;
    // self-consistent field (one x and one v dimension): the field of the
    // v-sweep is computed from the state before every v-sweep
    bool poisson = false;
    int vp_x = -1, vp_v = -1;
    double* d_vp = nullptr;     // [chunks][n_x] partial sums, E scratch [n_x], energy [1]
    // x-sweeps with the velocity at the Gauss nodes of every v-cell
    bool nodal = false;
    // every row of the sweeps in FP64 arithmetic (sl_set_arithmetic)
    bool wide = false;
    void* d_nodal = nullptr;    // node velocities per x-dimension, then the node tables
    int64_t nodal_vel_off[SL_MAX_DIM] = {0};
    int nodal_maxcls = 0;
    int32_t* d_nsig = nullptr;
    double* d_nalpha = nullptr;
    double* d_nab64 = nullptr;
    float* d_nab32 = nullptr;
    double* d_nabar = nullptr;  // alpha_bar per v-cell of the node table (mixed store)
    float* d_nna32 = nullptr;   // per v-cell FP32 record of the node table (kNa32 floats)
    double* d_partials = nullptr;
    double* d_mass = nullptr;
    int mass_nblk = 1;
    double* h_mass = nullptr;   // pinned

    double* d_stage = nullptr;  // lazily allocated AoS staging for set/get
    int64_t stage_cells = 0;
    double* d_proj = nullptr;   // lazily allocated projection workspace
    size_t proj_bytes = 0;

    sl::PolyTab poly{};

    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    double* d_gshifts = nullptr;   // shifts owned by a captured advect graph
    int64_t gshifts_n = 0;
    int graph_start = -1;       // copy index the first graph starts from
    int graph_flip = 0;         // sweeps per graph mod 2
    bool capturing = false;

    bool prof = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used;
    std::vector<int> ev_dim;
    int64_t prof_launches = 0;
    int64_t last_dim_launches[SL_MAX_DIM] = {0};
    double last_dim_ms[SL_MAX_DIM] = {0};

    struct Tune {
        int block = 256;
        int ft = 1;
        int unroll = 1;
        uint32_t chunk = 0;
        int pipeline = 0;
        int occ = 0;   // resident blocks per SM the walk is limited to (0: no limit)
    } tune[SL_MAX_DIM];

    std::string err;
};

namespace sl {
namespace host {

sl_status fail(sl_ctx* c, sl_status s, const char* fmt, ...);
sl_status fail_to(std::string* err, sl_status s, const char* fmt, ...);
sl_status cuda_fail(sl_ctx* c, cudaError_t e, const char* what);
// cudaMalloc / cudaMallocHost behind the allocation-failure test hook
// (sl_debug_fail_alloc): every device or pinned allocation the library makes.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t pinned_malloc(void** p, size_t bytes);
cudaError_t vp_field(sl_ctx* c, double* E, double* energy);
sl_status check_grid(const sl_grid* g, int degree, int storage, sl_ctx* c);
bool is_scaled(const sl_ctx* c);
bool is_split(const sl_ctx* c);   // the general split stores (# double = 2, 3)
// FP64 and hi planes per copy of (ndim, degree, storage).
void plane_counts(int ndim, int degree, int storage, int64_t* nlo, int64_t* nhi);
// Start of a copy's hi block (its first plane), whatever the kernels' convention.
void* hi_block(const sl_ctx* c, int parity);
int64_t fibre_groups(const sl_ctx* c, int ft);
// lanes: threads per line (G of the lane-group record form, else 1)
uint32_t chunk_for(const sl_ctx* c, int m, int ft, int lanes);
// Cell records of degree 1 in 5 or 6 dimensions offer the lane-group form,
// selected by fibres_per_thread == kRecLaneFt.
bool rec_lanes_ok(const sl_ctx* c);
bool rec_lanes(const sl_ctx* c, int ft);
double cell_width(const sl_grid& g, int m);
int64_t ipow(int64_t b, int e);
// Sweep geometry along `dim`, reading copy `parity` and writing the other.
SweepArgs make_args_parity(sl_ctx* c, int dim, int shift_dim, int parity);
int natural_shift_dim(const sl_ctx* c, int m);
int64_t field_offset(const sl_ctx* c, int xdim);

struct SubStep {
    int dim;
    double frac;
};
std::vector<SubStep> plan_of(const sl_ctx* c, sl_splitting sp);

}  // namespace host
}  // namespace sl

#define SL_CUDA(ctx, call)                                                 \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return sl::host::cuda_fail((ctx), e_, #call); \
    } while (0)
